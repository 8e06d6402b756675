// finom_kv_log_noalloc: the stabilised product log(diag(e^{a/eps}) K diag(e^{b/eps}) 1)
// for callers that may not allocate device memory.
//
// Some programs that embed this library cannot call cudaMalloc on the hot
// path: their device memory is owned by a fixed pool or another allocator,
// they run under a strict memory budget, or they must not take the
// allocator's locks or implicit synchronisation.  This entry point allocates
// nothing.  Its working memory (the tile aggregates, the tile carries and the
// last-CTA ticket of the scan) lives in one file-scope device array of
// kNoAllocBytes bytes that every GPU loading the library keeps until the
// process exits; the caller passes only inputs and outputs, and the plan's
// own tables were allocated when the plan was made.
//
// The product runs the half-step kernel (half.cuh) in its product mode with
// the levels formed inside the kernel from the caller's float64 vectors and
// the plan's positions, so it needs no converted copies; its result is the
// one finom_kv_log computes, to the same precision, for any a and b.
#include <cuda_runtime.h>

#include <mutex>

#include "finom_internal.h"
#include "half.cuh"

namespace finom {

template <class R>
finom_status half_launch(const HalfArgs<R>&, int, int, cudaStream_t);

namespace {

constexpr int kNoAllocMaxTiles = 4096;   // tiles of the plan (N + M <= 4096 * 2048 at 8 points per thread)
constexpr size_t kNoAllocPerTile = 4 * sizeof(double);   // one tile's two log-sum states (largest precision)
constexpr size_t kNoAllocMaps = kNoAllocPerTile * kNoAllocMaxTiles;
constexpr size_t kNoAllocCarries = kNoAllocPerTile * kNoAllocMaxTiles;
constexpr size_t kNoAllocBytes = kNoAllocMaps + kNoAllocCarries + 256;
static_assert(2 * HT<float>::kSt * sizeof(float) <= kNoAllocPerTile &&
                  2 * HT<double>::kSt * sizeof(double) <= kNoAllocPerTile,
              "per-tile scratch");

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

template <class R>
finom_status run_raw(finom_plan_s* p, bool transpose, const double* a, const double* b, double* out,
                     unsigned char* scratch, cudaStream_t s) {
  HalfArgs<R> r{};
  r.tbits = p->tbits;
  r.tile_x0 = p->tile_x0e;
  r.L = p->L;
  r.C = (int)p->Ce;
  r.o_is_x = transpose ? 0 : 1;
  r.rawO = transpose ? b : a;
  r.rawW = transpose ? a : b;
  r.posO = transpose ? p->y : p->x;
  r.posW = transpose ? p->x : p->y;
  r.scale = 1.0 / (p->eps * 0.69314718055994530942);
  r.inv_eps = 1.0 / p->eps;
  r.out = out;
  r.agg_out = reinterpret_cast<R*>(scratch);
  r.carry_out = reinterpret_cast<R*>(scratch + kNoAllocMaps);
  r.ctrl = reinterpret_cast<int32_t*>(scratch + kNoAllocMaps + kNoAllocCarries);
  // the ticket and the done flag must start at zero; the rest is fully
  // rewritten by every call
  cudaError_t e = cudaMemsetAsync(r.ctrl, 0, 8 * sizeof(int32_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(noalloc ticket)");
  r.carry_in = nullptr;
  finom_status rc = half_launch<R>(r, kHalfRawAgg, p->elems, s);
  if (rc != FINOM_OK) return rc;
  r.carry_in = r.carry_out;
  return half_launch<R>(r, kHalfRawLog, p->elems, s);
}

finom_status noalloc_dispatch(finom_plan_t p, bool transpose, const double* a, const double* b,
                              double* out, void* stream) {
  if (!p || !a || !b || !out) {
    set_error("finom_kv_log_noalloc: null argument");
    return FINOM_EINVAL;
  }
  if (p->dim != 1 || p->nd || p->B > 0) {
    set_error("finom_kv_log_noalloc: single 1D plans only");
    return FINOM_ENOTSUP;
  }
  if (p->Ce > kNoAllocMaxTiles) {
    set_error("finom_kv_log_noalloc: the plan has more tiles than the static scratch holds (at most " +
              std::to_string(kNoAllocMaxTiles) + " tiles, i.e. N + M <= " +
              std::to_string((long long)kNoAllocMaxTiles * kTile) + " merged points at 8 points per thread)");
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
