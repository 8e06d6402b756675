// float64 transport cost <C, Gamma> and marginal error of given potentials.
//
// Gamma_ij = u_i v_j 2^{Px_i + Py_j - G_ij}, G_ij = |x_i - y_j| / (eps ln 2)
// (Sec. 2.1: Gamma = diag(phi) K diag(psi)).  For every y point j the kernel
// computes, in the frame Py_j,
//     S_j = sum_i u_i 2^{Px_i + Py_j - G_ij}       (column sum / v_j)
//     T_j = sum_i u_i G_ij 2^{Px_i + Py_j - G_ij}   (cost-weighted column sum)
// with the same forward/backward recurrences as the half step, augmented by
// a distance moment: moving by a gap g turns (s, t) into 2^A (s, t + g s).
// Then err = sum_j |v_j S_j - v_j| (Algorithm 1 loop head) and
// <C, Gamma> = eps ln 2 sum_j v_j T_j (objective of eq. w1Definition).
#include <cuda_runtime.h>

#include <algorithm>

#include "dev_common.cuh"
#include "finom_internal.h"

namespace finom {

namespace {

struct LSM {
  double m, s, t;
};
struct AggM {
  double D, G, m, s, t;
};

__device__ __forceinline__ LSM lsm_add(double ma, double sa, double ta, double mb, double sb,
                                       double tb) {
  double d = mb - ma;
  bool bmax = d > 0.0;
  double e = exp2(-fabs(d));
  LSM r;
  r.m = bmax ? mb : ma;
  r.s = bmax ? fma(sa, e, sb) : fma(sb, e, sa);
  r.t = bmax ? fma(ta, e, tb) : fma(tb, e, ta);
  if (r.s >= 2.0) {
    r.s *= 0.5;
    r.t *= 0.5;
    r.m += 1.0;
  }
  return r;
}

// w = mant 2^e with mant in [1, 2) (w = 0: mant = 0, e a very negative level)
__device__ __forceinline__ void split_mass(double w, double& e, double& mant) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(w);
  const int ex = (int)((b >> 52) & 0x7ffull);
  const bool z = ex == 0;
  e = z ? -1.0e300 : (double)(ex - 1023);
  mant = z ? 0.0 : __longlong_as_double((long long)((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
}

// the kElems gaps of a thread's merged points (16-byte loads; the gap array
// is padded to whole tiles)
__device__ __forceinline__ void load_gaps(const double* gap, int64_t seg, double (&g)[kElems]) {
  const double2* p = reinterpret_cast<const double2*>(gap + seg);
#pragma unroll
  for (int q = 0; q < kElems / 2; ++q) {
    const double2 v = __ldg(p + q);
    g[2 * q] = v.x;
    g[2 * q + 1] = v.y;
  }
}

__device__ __forceinline__ AggM aggm_identity() { return {0.0, 0.0, -1.0e300, 0.0, 0.0}; }

__device__ __forceinline__ AggM aggm_then(const AggM& a, const AggM& b) {
  LSM r = lsm_add(a.m + b.D, a.s, fma(b.G, a.s, a.t), b.m, b.s, b.t);
  return {a.D + b.D, a.G + b.G, r.m, r.s, r.t};
}

__device__ __forceinline__ LSM aggm_apply(const AggM& a, LSM st) {
  return lsm_add(st.m + a.D, st.s, fma(a.G, st.s, st.t), a.m, a.s, a.t);
}

__device__ __forceinline__ AggM shfl_aggm(const AggM& a, int o, bool up) {
  AggM r;
  if (up) {
    r.D = __shfl_up_sync(0xffffffffu, a.D, o); r.G = __shfl_up_sync(0xffffffffu, a.G, o);
    r.m = __shfl_up_sync(0xffffffffu, a.m, o); r.s = __shfl_up_sync(0xffffffffu, a.s, o);
    r.t = __shfl_up_sync(0xffffffffu, a.t, o);
  } else {
    r.D = __shfl_down_sync(0xffffffffu, a.D, o); r.G = __shfl_down_sync(0xffffffffu, a.G, o);
    r.m = __shfl_down_sync(0xffffffffu, a.m, o); r.s = __shfl_down_sync(0xffffffffu, a.s, o);
    r.t = __shfl_down_sync(0xffffffffu, a.t, o);
  }
  return r;
}

template <bool kReverse>
__device__ AggM scan_m(AggM x, AggM* sh, AggM& total) {
  constexpr int NW = kThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  AggM inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    AggM t = shfl_aggm(inc, o, !kReverse);
    if (!kReverse ? (lane >= o) : (lane + o < 32)) inc = aggm_then(t, inc);
  }
  AggM exc = shfl_aggm(inc, 1, !kReverse);
  if (kReverse ? (lane == 31) : (lane == 0)) exc = aggm_identity();
  if (kReverse ? (lane == 0) : (lane == 31)) sh[warp] = inc;
  __syncthreads();
  AggM wp = aggm_identity(), tot = aggm_identity();
  if (!kReverse) {
    for (int w = 0; w < NW; ++w) {
      if (w < warp) wp = aggm_then(wp, sh[w]);
      tot = aggm_then(tot, sh[w]);
    }
  } else {
    for (int w = NW - 1; w >= 0; --w) {
      if (w > warp) wp = aggm_then(wp, sh[w]);
      tot = aggm_then(tot, sh[w]);
    }
  }
  __syncthreads();
  total = tot;
  return aggm_then(wp, exc);
}

struct CostArgs {
  const uint32_t* tbits;
  const double* gap;
  const int32_t* tile_x0;
  int64_t L;
  int C;              // tiles
  const double* px;   // W side (x): smooth potentials (log2 units)
  const double* py;   // O side (y): smooth potentials (frames)
  const double* u;    // W side: masses
  const double* v;    // O side: masses
  double* agg;        // 10 per tile
  double* carry;      // 6 per tile
  double* part;       // 2 per tile
  double* out;        // [0] err [1] sum v T
  int32_t* ticket;
};

struct CostSmem {
  double pot[kTile + 2];
  double mass[kTile + 2];
  AggM scan[kThreads / 32];
  double red[2][kThreads / 32];
  int iscan[kThreads / 32];
  int last;
};

// Points: O = y (outputs), W = x (weights).  Per merged point e: Af / Ab
// the exponent a forward / backward state moves by (frame change minus the
// gap), and for a W point its log2 level Bl, mantissa Bs and moment Bt (0).
__device__ __forceinline__ void cost_terms(uint32_t omask, uint32_t wmask, const double (&g)[kElems],
                                           const double* po, int o0, const double* pw,
                                           const double* mw, int w0, double (&Af)[kElems],
                                           double (&Ab)[kElems], double (&Bl)[kElems],
                                           double (&Bs)[kElems], double (&Bt)[kElems]) {
  double cprev = po[o0];
  int oi = o0 + 1, wi = w0;
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    double dc = 0.0;
    if ((omask >> e) & 1u) {
      double c = po[oi++];
      dc = c - cprev;
      cprev = c;
    }
    Af[e] = dc - g[e];
    Ab[e] = -dc - g[e];
    Bl[e] = -1.0e300;
    Bs[e] = 0.0;
    Bt[e] = 0.0;
    if ((wmask >> e) & 1u) {
      double ex, mt;
      split_mass(mw[wi], ex, mt);
      if (mt > 0.0) {
        Bl[e] = (cprev + pw[wi]) + ex;
        Bs[e] = mt;
      }
      ++wi;
    }
  }
}

__device__ __forceinline__ AggM fwd_mapm(const double (&Af)[kElems], const double (&g)[kElems],
                                         const double (&Bl)[kElems], const double (&Bs)[kElems],
                                         const double (&Bt)[kElems], uint32_t wmask) {
  AggM a = aggm_identity();
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    a.D += Af[e];
    a.G += g[e];
    a.m += Af[e];
    a.t = fma(g[e], a.s, a.t);
    if ((wmask >> e) & 1u) {
      LSM r = lsm_add(a.m, a.s, a.t, Bl[e], Bs[e], Bt[e]);
      a.m = r.m; a.s = r.s; a.t = r.t;
    }
  }
  return a;
}

__device__ __forceinline__ AggM bwd_mapm(const double (&Ab)[kElems], const double (&g)[kElems],
                                         const double (&Bl)[kElems], const double (&Bs)[kElems],
                                         const double (&Bt)[kElems], uint32_t wmask) {
  AggM a = aggm_identity();
#pragma unroll
  for (int e = kElems - 1; e >= 0; --e) {
    if ((wmask >> e) & 1u) {
      LSM r = lsm_add(a.m, a.s, a.t, Bl[e], Bs[e], Bt[e]);
      a.m = r.m; a.s = r.s; a.t = r.t;
    }
    a.t = fma(g[e], a.s, a.t);
    a.m += Ab[e];
    a.D += Ab[e];
    a.G += g[e];
  }
  return a;
}

__device__ __forceinline__ AggM load_aggm(const double* o) {
  return AggM{__ldcg(o), __ldcg(o + 1), __ldcg(o + 2), __ldcg(o + 3), __ldcg(o + 4)};
}

template <bool kMaps>
__global__ void __launch_bounds__(kThreads) k_cost(CostArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CostSmem& sm = *reinterpret_cast<CostSmem*>(smem_raw);
  const int tid = threadIdx.x;
  const int C = a.C;
  const int tile = (int)blockIdx.x;
  const int64_t k0 = (int64_t)tile * kTile;
  const int64_t kend = min(k0 + (int64_t)kTile, a.L);
  const int x0 = a.tile_x0[tile], x1 = a.tile_x0[tile + 1];
  const int y0 = (int)(k0 - x0), y1 = (int)(kend - x1);
  const int n_o = y1 - y0, n_w = x1 - x0, wofs = n_o + 1;
  const int64_t seg = k0 + (int64_t)tid * kElems;
  uint32_t vmask = 0;
  if (seg < a.L) {
    int64_t nv = a.L - seg;
    vmask = nv >= kElems ? ((1u << kElems) - 1u) : ((1u << nv) - 1u);
  }
  uint32_t bits = (seg < a.L) ? ((a.tbits[seg >> 5] >> (seg & 31)) & ((1u << kElems) - 1u)) : 0u;
  const uint32_t wmask = bits & vmask, omask = (~bits) & vmask;
  double g[kElems];
  load_gaps(a.gap, seg, g);
  const int o_before = block_exclusive_sum<kThreads>(__popc(omask), sm.iscan);
  // threads past the end of the sequence own no points; keep their index in range
  const int w_before = min((int)(seg - k0) - o_before, n_w);
  for (int i = tid; i < n_o + 1; i += kThreads) {
    const int64_t gi = max(y0 - 1 + i, 0);
    sm.pot[i] = a.py[gi];
    sm.mass[i] = a.v[gi];
  }
  for (int i = tid; i < n_w + 1; i += kThreads) {
    const int64_t gi = max(x0 - 1 + i, 0);
    sm.pot[wofs + i] = a.px[gi];
    sm.mass[wofs + i] = a.u[gi];
  }
  __syncthreads();
  double Af[kElems], Ab[kElems], Bl[kElems], Bs[kElems], Bt[kElems];
  cost_terms(omask, wmask, g, sm.pot, o_before, sm.pot + wofs, sm.mass + wofs, w_before + 1,
                    Af, Ab, Bl, Bs, Bt);
  AggM tf, tb;
  if (kMaps) {
    (void)scan_m<false>(fwd_mapm(Af, g, Bl, Bs, Bt, wmask), sm.scan, tf);
    (void)scan_m<true>(bwd_mapm(Ab, g, Bl, Bs, Bt, wmask), sm.scan, tb);
    if (tid == 0) {
      double* o = a.agg + 10 * (int64_t)blockIdx.x;
      o[0] = tf.D; o[1] = tf.G; o[2] = tf.m; o[3] = tf.s; o[4] = tf.t;
      o[5] = tb.D; o[6] = tb.G; o[7] = tb.m; o[8] = tb.s; o[9] = tb.t;
    }
  } else {
    AggM pre = scan_m<false>(fwd_mapm(Af, g, Bl, Bs, Bt, wmask), sm.scan, tf);
    const double* c = a.carry + 6 * (int64_t)blockIdx.x;
    LSM st = aggm_apply(pre, LSM{c[0], c[1], c[2]});
    double fm[kElems], fs[kElems], ft[kElems];
#pragma unroll
    for (int e = 0; e < kElems; ++e) {
      st.m += Af[e];
      st.t = fma(g[e], st.s, st.t);
      if ((wmask >> e) & 1u) st = lsm_add(st.m, st.s, st.t, Bl[e], Bs[e], Bt[e]);
      fm[e] = st.m; fs[e] = st.s; ft[e] = st.t;
    }
    pre = scan_m<true>(bwd_mapm(Ab, g, Bl, Bs, Bt, wmask), sm.scan, tb);
    st = aggm_apply(pre, LSM{c[3], c[4], c[5]});
    int oi = o_before + __popc(omask);
    double err = 0.0, wt = 0.0;
#pragma unroll
    for (int e = kElems - 1; e >= 0; --e) {
      if ((omask >> e) & 1u) {
        const LSM s2 = lsm_add(fm[e], fs[e], ft[e], st.m, st.s, st.t);
        const double sc = exp2(s2.m);
        const double vj = sm.mass[oi];
        err += fabs(vj * (s2.s * sc) - vj);
        wt += vj * (s2.t * sc);
        --oi;
      }
      if ((wmask >> e) & 1u) st = lsm_add(st.m, st.s, st.t, Bl[e], Bs[e], Bt[e]);
      st.t = fma(g[e], st.s, st.t);
      st.m += Ab[e];
    }
    err = warp_sum(err);
    wt = warp_sum(wt);
    if ((tid & 31) == 0) {
      sm.red[0][tid >> 5] = err;
      sm.red[1][tid >> 5] = wt;
    }
    __syncthreads();
    if (tid == 0) {
      double se = 0.0, sw = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) { se += sm.red[0][w]; sw += sm.red[1][w]; }
      a.part[2 * (int64_t)blockIdx.x] = se;
      a.part[2 * (int64_t)blockIdx.x + 1] = sw;
    }
  }
  // ticket
  const int total = C;
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    sm.last = (atomicAdd(a.ticket, 1) == total - 1);
  }
  __syncthreads();
  if (!sm.last) return;
  __threadfence();
  if (kMaps) {
    // scan the tile maps into carries (same layout as carry_scan, 3 values per state)
    const int per = (C + kThreads - 1) / kThreads;
    const int t0 = min(C, tid * per), t1 = min(C, t0 + per);
    AggM loc = aggm_identity();
    for (int t = t0; t < t1; ++t) loc = aggm_then(loc, load_aggm(a.agg + 10 * t));
    AggM tot;
    AggM pre = scan_m<false>(loc, sm.scan, tot);
    LSM st = aggm_apply(pre, LSM{-1.0e300, 0.0, 0.0});
    for (int t = t0; t < t1; ++t) {
      a.carry[6 * t + 0] = st.m; a.carry[6 * t + 1] = st.s; a.carry[6 * t + 2] = st.t;
      st = aggm_apply(load_aggm(a.agg + 10 * t), st);
    }
    loc = aggm_identity();
    for (int t = t1 - 1; t >= t0; --t) loc = aggm_then(loc, load_aggm(a.agg + 10 * t + 5));
    pre = scan_m<true>(loc, sm.scan, tot);
    st = aggm_apply(pre, LSM{-1.0e300, 0.0, 0.0});
    for (int t = t1 - 1; t >= t0; --t) {
      a.carry[6 * t + 3] = st.m; a.carry[6 * t + 4] = st.s; a.carry[6 * t + 5] = st.t;
      st = aggm_apply(load_aggm(a.agg + 10 * t + 5), st);
    }
  } else {
    double se = 0.0, sw = 0.0;
    for (int t = tid; t < total; t += kThreads) {
      se += __ldcg(a.part + 2 * t);
      sw += __ldcg(a.part + 2 * t + 1);
    }
    se = warp_sum(se);
    sw = warp_sum(sw);
    __syncthreads();
    if ((tid & 31) == 0) {
      sm.red[0][tid >> 5] = se;
      sm.red[1][tid >> 5] = sw;
    }
    __syncthreads();
    if (tid == 0) {
      se = 0.0;
      sw = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) { se += sm.red[0][w]; sw += sm.red[1][w]; }
      a.out[0] = se;
      a.out[1] = sw;
    }
  }
  if (tid == 0) *a.ticket = 0;
}

finom_status run_cost(const CostArgs& a, cudaStream_t s) {
  const size_t smem = sizeof(CostSmem);
  // once per process (a function-local static: thread-safe initialisation)
  static const cudaError_t attr = [smem]() {
    cudaError_t e = cudaFuncSetAttribute(k_cost<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_cost<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
  }();
  FINOM_CUDA(attr);
  k_cost<true><<<(unsigned)a.C, kThreads, smem, s>>>(a);
  k_cost<false><<<(unsigned)a.C, kThreads, smem, s>>>(a);
  FINOM_CUDA(cudaGetLastError());
  return FINOM_OK;
}

CostArgs cost_args(const finom_plan_s* p, double* scratch, int32_t* ticket) {
  CostArgs a{};
  a.tbits = p->tbits;
  a.gap = p->gap64;
  a.tile_x0 = p->tile_x0;
  a.L = p->L;
  a.C = (int)p->C;
  const size_t T = (size_t)p->C;
  a.agg = scratch;
  a.carry = scratch + 10 * T;
  a.part = scratch + 16 * T;
  a.out = scratch + 18 * T;
  a.ticket = ticket;
  return a;
}

}  // namespace

// Float64 evaluation of (err, <C,Gamma>) for smooth potentials px, py (log2
// units, float64) and masses u, v (float64, normalised).  Synchronous.
finom_status cost64(finom_plan_s* p, const double* px, const double* py, const double* u,
                    const double* v, double* err, double* w1, cudaStream_t s) {
  const size_t T = (size_t)p->C;
  double* scratch = nullptr;
  int32_t* ticket = nullptr;
  FINOM_CUDA(cudaMallocAsync(&scratch, sizeof(double) * (18 * T + 2), s));
  FINOM_CUDA(cudaMallocAsync(&ticket, sizeof(int32_t), s));
  FINOM_CUDA(cudaMemsetAsync(ticket, 0, sizeof(int32_t), s));
  CostArgs a = cost_args(p, scratch, ticket);
  a.px = px; a.py = py; a.u = u; a.v = v;
  finom_status rc = run_cost(a, s);
  if (rc != FINOM_OK) return rc;
  double h[2];
  FINOM_CUDA(cudaMemcpyAsync(h, a.out, sizeof(h), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  cudaFreeAsync(scratch, s);
  cudaFreeAsync(ticket, s);
  *err = h[0];
  *w1 = h[1] * p->eps * 0.69314718055994530942;
  return FINOM_OK;
}

}  // namespace finom
