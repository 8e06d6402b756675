// finom_kv_log_noalloc: the stabilised product log(diag(e^{a/eps}) K diag(e^{b/eps}) 1)
// for callers that may not allocate device memory.
//
// Some programs that embed this library cannot call cudaMalloc on the hot
// path: their device memory is owned by a fixed pool or another allocator,
// they run under a strict memory budget, or they must not take the
// allocator's locks or implicit synchronisation.  This entry point allocates
// nothing.  Its working memory (the tile maps, the tile carries and the
// last-CTA ticket of the scan) lives in one file-scope device array of
// kNoAllocBytes bytes that every GPU loading the library keeps until the
// process exits; the caller passes only inputs and outputs, and the plan's
// own tables were allocated when the plan was made.
//
// The product is computed in one pass with the caller's a as the frame
// (finom_kv_log refines the frame in a second pass; with absorption vectors
// that vary smoothly between neighbouring points the two agree to float32
// precision).
#include <cuda_runtime.h>

#include <mutex>

#include "apply.cuh"
#include "finom_internal.h"

namespace finom {
namespace {

constexpr int kNoAllocMaxTiles = 4096;   // N + M <= 4096 * kTile merged points
constexpr size_t kNoAllocMaps = 6 * (size_t)kNoAllocMaxTiles * sizeof(double);
constexpr size_t kNoAllocCarries = 4 * (size_t)kNoAllocMaxTiles * sizeof(double);
constexpr size_t kNoAllocBytes = kNoAllocMaps + kNoAllocCarries + 256;

// The shared scratch.  Host code must not take this symbol's address as a
// device pointer: the address is obtained once per device with
// cudaGetSymbolAddress and passed to the kernels.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

finom_status scratch_for_device(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("finom_kv_log_noalloc: device index out of range");
    return FINOM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return FINOM_OK;
}

struct RawArgs {
  const uint32_t* tbits;
  const void* gap;
  const int32_t* tile_x0;
  int64_t L;
  int C;
  int o_is_x;
  const double* aO;   // O-side absorption (cost units): the frame
  const double* bW;   // W-side absorption (cost units, may be -inf)
  double scale;       // 1 / (eps ln 2)
  double* out;        // ln of the product at the O points
  void* maps;         // 6 * C tile maps (plan precision)
  void* carries;      // 4 * C tile carries
  int32_t* ticket;
};

template <class R>
__device__ __forceinline__ void to_pot(double v, float2& p) {
  const float hi = (float)v;
  p = make_float2(hi, (float)(v - (double)hi));
}
template <class R>
__device__ __forceinline__ void to_pot(double v, double& p) {
  p = v;
}

template <class R, bool kAggOnly>
__global__ void __launch_bounds__(kThreads) k_apply_raw(RawArgs a) {
  using T = Tr<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem<R>& sm = *reinterpret_cast<TileSmem<R>*>(smem_raw);
  const int tid = threadIdx.x, tile = blockIdx.x;
  const int64_t k0 = (int64_t)tile * kTile;
  const int64_t kend = min(k0 + (int64_t)kTile, a.L);
  const int x0 = a.tile_x0[tile], x1 = a.tile_x0[tile + 1];
  const int y0 = (int)(k0 - x0), y1 = (int)(kend - x1);
  const int o_start = a.o_is_x ? x0 : y0;
  const int n_o = a.o_is_x ? (x1 - x0) : (y1 - y0);
  const int w_start = a.o_is_x ? y0 : x0;
  const int n_w = a.o_is_x ? (y1 - y0) : (x1 - x0);
  const int wofs = n_o + 1;
  const int64_t seg = k0 + (int64_t)tid * kElems;
  uint32_t vmask = 0;
  if (seg < a.L) {
    const int64_t nv = a.L - seg;
    vmask = nv >= kElems ? ((1u << kElems) - 1u) : ((1u << nv) - 1u);
  }
  const uint32_t bits = (seg < a.L) ? ((a.tbits[seg >> 5] >> (seg & 31)) & ((1u << kElems) - 1u)) : 0u;
  const uint32_t xmask = bits & vmask, ymask = (~bits) & vmask;
  const uint32_t omask = a.o_is_x ? xmask : ymask;
  const uint32_t wmask = a.o_is_x ? ymask : xmask;
  R g[kElems];
  load_gaps<R>(static_cast<const R*>(a.gap), seg, g);
  // stage the caller's absorption vectors as frames / weights
  for (int i = tid; i < n_o + 1; i += kThreads) {
    const int gi = max(o_start - 1 + i, 0);
    to_pot<R>(a.aO[gi] * a.scale, sm.pot[i]);
    sm.mass[i] = (typename T::Mass)1;
  }
  for (int i = tid; i < n_w + 1; i += kThreads) {
    const int gi = max(w_start - 1 + i, 0);
    const double b = a.bW[gi];
    const bool fin = b > -INFINITY;
    to_pot<R>(fin ? b * a.scale : 0.0, sm.pot[wofs + i]);
    sm.mass[wofs + i] = fin ? (typename T::Mass)1 : (typename T::Mass)0;
  }
  const int o_before = block_exclusive_sum<kThreads>(__popc(omask), sm.iscan);
  const int w_before = min((int)(seg - k0) - o_before, n_w);

  R D[kElems], PB[kElems], L1[kElems], L2[kElems], mt[kElems], MF, MB;
  Agg<R> mapF, mapB;
  seg_terms<R>(omask, wmask, g, sm.pot, o_before, sm.pot + wofs, sm.mass + wofs, w_before + 1, R(0),
               D, PB, L1, L2, mt);
  const bool fast = seg_maps<R>(D, PB, L1, L2, mt, mapF, mapB, MF, MB);
  R* maps = static_cast<R*>(a.maps);
  R* carries = static_cast<R*>(a.carries);
  put_map(sm.tf, tid, mapF);
  put_map(sm.tb, tid, mapB);
  __syncthreads();

  if constexpr (kAggOnly) {
    if (tid < 64) rake_reduce<R>(sm, maps + 6 * tile);
    if (last_cta<R>(a.ticket, a.C, sm)) {
      carry_scan<R>(maps, carries, a.C, sm);
      if (tid == 0) *a.ticket = 0;
    }
    return;
  }

  if (tid < 64) {
    const R* c = carries + 4 * tile;
    rake_scan<R>(sm, LS<R>{c[0], c[1]}, LS<R>{c[2], c[3]});
  }
  __syncthreads();
  const LS<R> ef = {sm.tf[1][slot(tid)], sm.tf[2][slot(tid)]};
  const LS<R> eb = {sm.tb[1][slot(tid)], sm.tb[2][slot(tid)]};
  const R ebm = eb.m + PB[kElems - 1];
  R lam[kElems];
  if (fast) {
    R qsuf[kElems];
    R acc = R(0);
#pragma unroll
    for (int e = kElems - 1; e >= 0; --e) {
      qsuf[e] = acc;
      acc += L2[e];
    }
    const R lf1 = (ef.s > R(0)) ? ef.m : T::kNegBig;
    const R LF = fmax(lf1, MF);
    const R cF0 = ef.s * T::ex2(lf1 - LF), cF1 = T::ex2(MF - LF);
    const R lb1 = (eb.s > R(0)) ? ebm : T::kNegBig;
    const R LB = fmax(lb1, MB);
    const R cB0 = eb.s * T::ex2(lb1 - LB), cB1 = T::ex2(MB - LB);
    R pf = R(0);
#pragma unroll
    for (int e = 0; e < kElems; ++e) {
      pf += L1[e];
      const R sf = fma(cF1, pf, cF0), sb = fma(cB1, qsuf[e], cB0);
      const R a1 = (sf > R(0)) ? LF + D[e] : T::kNegBig;
      const R a2 = (sb > R(0)) ? LB - PB[e] : T::kNegBig;
      const R M = fmax(a1, a2);
      lam[e] = M + T::lg2(fma(sf, T::ex2(a1 - M), sb * T::ex2(a2 - M)));
    }
  } else {
    R fm[kElems], fs[kElems];
    R m = ef.m, sv = ef.s;
#pragma unroll
    for (int e = 0; e < kElems; ++e) {
      if (mt[e] > R(0)) ls_add_fast(m, sv, L1[e], mt[e]);
      fm[e] = m;
      fs[e] = sv;
    }
    m = ebm;
    sv = eb.s;
#pragma unroll
    for (int e = kElems - 1; e >= 0; --e) {
      LS<R> s2 = ls_add(fm[e] + D[e], fs[e], m - PB[e], sv);
      lam[e] = s2.m + T::lg2(s2.s);
      if (mt[e] > R(0)) ls_add_fast(m, sv, L2[e], mt[e]);
    }
  }
  int oi = o_before;
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    if ((omask >> e) & 1u) {
      ++oi;
      a.out[o_start + oi - 1] = 0.69314718055994530942 * (double)lam[e];
    }
  }
}

template <class R>
finom_status run_raw(finom_plan_s* p, bool transpose, const double* a, const double* b, double* out,
                     unsigned char* scratch, cudaStream_t s) {
  RawArgs r{};
  r.tbits = p->tbits;
  r.gap = p->gap;
  r.tile_x0 = p->tile_x0;
  r.L = p->L;
  r.C = (int)p->C;
  r.o_is_x = transpose ? 0 : 1;
  r.aO = transpose ? b : a;
  r.bW = transpose ? a : b;
  r.scale = 1.0 / (p->eps * 0.69314718055994530942);
  r.out = out;
  r.maps = scratch;
  r.carries = scratch + kNoAllocMaps;
  r.ticket = reinterpret_cast<int32_t*>(scratch + kNoAllocMaps + kNoAllocCarries);
  // the ticket must start at zero; the rest is fully rewritten by every call
  cudaError_t e = cudaMemsetAsync(r.ticket, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(noalloc ticket)");
  const size_t smem = sizeof(TileSmem<R>);
  k_apply_raw<R, true><<<r.C, kThreads, smem, s>>>(r);
  k_apply_raw<R, false><<<r.C, kThreads, smem, s>>>(r);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "k_apply_raw launch");
  return FINOM_OK;
}

finom_status noalloc_dispatch(finom_plan_t p, bool transpose, const double* a, const double* b,
                              double* out, void* stream) {
  if (!p || !a || !b || !out) {
    set_error("finom_kv_log_noalloc: null argument");
    return FINOM_EINVAL;
  }
  if (p->dim != 1 || p->B > 0) {
    set_error("finom_kv_log_noalloc: single 1D plans only");
    return FINOM_ENOTSUP;
  }
  if (p->C > kNoAllocMaxTiles) {
    set_error("finom_kv_log_noalloc: N + M exceeds the static scratch (at most " +
              std::to_string((long long)kNoAllocMaxTiles * kTile) + " merged points)");
    return FINOM_EINVAL;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != p->device) cudaSetDevice(p->device);
  unsigned char* scratch = nullptr;
  finom_status rc = scratch_for_device(p->device, &scratch);
  if (rc == FINOM_OK) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = p->prec == FINOM_F32_LOG ? run_raw<float>(p, transpose, a, b, out, scratch, s)
                                  : run_raw<double>(p, transpose, a, b, out, scratch, s);
  }
  if (prev >= 0 && prev != p->device) cudaSetDevice(prev);
  return rc;
}

}  // namespace
}  // namespace finom

extern "C" finom_status finom_kv_log_noalloc(finom_plan_t plan, const double* a, const double* b,
                                             double* out, void* stream) {
  return finom::noalloc_dispatch(plan, false, a, b, out, stream);
}
