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

#include "apply.cuh"

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

// How the weights and frames of a cost pass are given.
enum : int {
  C_ZERO_FRAME = 1,  // O side has no potentials: frame 0 (the first 2D pass)
  C_LEVELS = 2,      // W side gives (log2 level, moment ratio) instead of (potential, mass)
  C_INTER = 4,       // write log2 S and T/S per O point instead of reducing (err, sum v T)
};

struct CostArgs {
  const uint32_t* tbits;
  const double* gap;
  const int32_t* tile_x0;
  int64_t L;
  int C;              // tiles per line
  int lines;
  int64_t o_ls, o_es; // O-side arrays: offset between lines, stride between points
  int64_t w_ls, w_es; // W-side arrays
  const double* px;   // W side: smooth potentials (log2 units) or log2 levels (C_LEVELS)
  const double* py;   // O side: smooth potentials (frames)
  const double* u;    // W side: masses, or moment ratios T/S (C_LEVELS)
  const double* v;    // O side: masses
  double* z1;         // C_INTER outputs: log2 S, T/S
  double* z2;
  int64_t z_ls, z_es;
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

// Points: O = y (outputs), W = x (weights).  Exponents as in point_terms;
// Bt is the moment a weight brings with it (C_LEVELS).
template <int kMode>
__device__ __forceinline__ void cost_terms(uint32_t omask, uint32_t wmask, const double (&g)[kElems],
                                           const double* po, int o0, const double* pw,
                                           const double* mw, int w0, double (&Af)[kElems],
                                           double (&Ab)[kElems], double (&Bl)[kElems],
                                           double (&Bs)[kElems], double (&Bt)[kElems]) {
  double cprev = (kMode & C_ZERO_FRAME) ? 0.0 : po[o0];
  int oi = o0 + 1, wi = w0;
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    double dc = 0.0;
    if (!(kMode & C_ZERO_FRAME) && ((omask >> e) & 1u)) {
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
      if (kMode & C_LEVELS) {
        const double lv = pw[wi];
        if (lv > -1.0e290) {
          Bl[e] = cprev + lv;
          Bs[e] = 1.0;
          Bt[e] = mw[wi];
        }
      } else {
        double ex, mt;
        Tr<double>::split(mw[wi], ex, mt);
        if (mt > 0.0) {
          Bl[e] = (cprev + pw[wi]) + ex;
          Bs[e] = mt;
        }
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

template <bool kMaps, int kMode>
__global__ void __launch_bounds__(kThreads) k_cost(CostArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CostSmem& sm = *reinterpret_cast<CostSmem*>(smem_raw);
  const int tid = threadIdx.x;
  const int C = a.C;
  const int line = (int)(blockIdx.x / (unsigned)C);
  const int tile = (int)blockIdx.x - line * C;
  const int64_t ob = (int64_t)line * a.o_ls, wb = (int64_t)line * a.w_ls;
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
  load_gaps<double>(a.gap, seg, g);
  const int o_before = block_exclusive_sum<kThreads>(__popc(omask), sm.iscan);
  // threads past the end of the sequence own no points; keep their index in range
  const int w_before = min((int)(seg - k0) - o_before, n_w);
  for (int i = tid; i < n_o + 1; i += kThreads) {
    const int64_t gi = ob + (int64_t)max(y0 - 1 + i, 0) * a.o_es;
    sm.pot[i] = (kMode & C_ZERO_FRAME) ? 0.0 : a.py[gi];
    sm.mass[i] = (kMode & C_INTER) ? 0.0 : a.v[gi];
  }
  for (int i = tid; i < n_w + 1; i += kThreads) {
    const int64_t gi = wb + (int64_t)max(x0 - 1 + i, 0) * a.w_es;
    sm.pot[wofs + i] = a.px[gi];
    sm.mass[wofs + i] = a.u[gi];
  }
  __syncthreads();
  double Af[kElems], Ab[kElems], Bl[kElems], Bs[kElems], Bt[kElems];
  cost_terms<kMode>(omask, wmask, g, sm.pot, o_before, sm.pot + wofs, sm.mass + wofs, w_before + 1,
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
        LSM s2 = lsm_add(fm[e], fs[e], ft[e], st.m, st.s, st.t);
        if (kMode & C_INTER) {
          const bool pos = s2.s > 0.0;
          const int64_t zi = (int64_t)line * a.z_ls + (int64_t)(y0 + oi - 1) * a.z_es;
          a.z1[zi] = pos ? s2.m + log2(s2.s) : -1.0e300;
          a.z2[zi] = pos ? s2.t / s2.s : 0.0;
        } else {
          double sc = exp2(s2.m);
          double vj = sm.mass[oi];
          err += fabs(vj * (s2.s * sc) - vj);
          wt += vj * (s2.t * sc);
        }
        --oi;
      }
      if ((wmask >> e) & 1u) st = lsm_add(st.m, st.s, st.t, Bl[e], Bs[e], Bt[e]);
      st.t = fma(g[e], st.s, st.t);
      st.m += Ab[e];
    }
    if (!(kMode & C_INTER)) {
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
  }
  // ticket
  const int total = a.lines * C;
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    sm.last = (atomicAdd(a.ticket, 1) == total - 1);
  }
  __syncthreads();
  if (!sm.last) return;
  __threadfence();
  if (kMaps && a.lines > 1) {
    // line batches: one thread per line scans its few tiles; lines start empty
    for (int l = tid; l < a.lines; l += kThreads) {
      const int64_t b = (int64_t)l * C;
      LSM st = LSM{-1.0e300, 0.0, 0.0};
      for (int t = 0; t < C; ++t) {
        double* cw = a.carry + 6 * (b + t);
        cw[0] = st.m; cw[1] = st.s; cw[2] = st.t;
        st = aggm_apply(load_aggm(a.agg + 10 * (b + t)), st);
      }
      st = LSM{-1.0e300, 0.0, 0.0};
      for (int t = C - 1; t >= 0; --t) {
        double* cw = a.carry + 6 * (b + t);
        cw[3] = st.m; cw[4] = st.s; cw[5] = st.t;
        st = aggm_apply(load_aggm(a.agg + 10 * (b + t) + 5), st);
      }
    }
  } else if (kMaps) {
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
  } else if (!(kMode & C_INTER)) {
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

template <int kMode>
finom_status run_cost(const CostArgs& a, cudaStream_t s) {
  const size_t smem = sizeof(CostSmem);
  static bool attr = false;
  if (!attr) {
    FINOM_CUDA(cudaFuncSetAttribute(k_cost<true, kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FINOM_CUDA(cudaFuncSetAttribute(k_cost<false, kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  const unsigned grid = (unsigned)((int64_t)a.C * a.lines);
  k_cost<true, kMode><<<grid, kThreads, smem, s>>>(a);
  k_cost<false, kMode><<<grid, kThreads, smem, s>>>(a);
  FINOM_CUDA(cudaGetLastError());
  return FINOM_OK;
}

CostArgs cost_args(const finom_plan_s* p, int lines, double* scratch, int32_t* ticket) {
  CostArgs a{};
  a.tbits = p->tbits;
  a.gap = p->gap64;
  a.tile_x0 = p->tile_x0;
  a.L = p->L;
  a.C = (int)p->C;
  a.lines = lines;
  a.o_es = 1;
  a.w_es = 1;
  const size_t T = (size_t)p->C * lines;
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
  CostArgs a = cost_args(p, 1, scratch, ticket);
  a.px = px; a.py = py; a.u = u; a.v = v;
  finom_status rc = run_cost<0>(a, s);
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

// The same for a 2D plan (Sec. 3, Appendix A).  pa: smooth potentials of the
// first grid, row-major (i + M k); pb: of the second grid, column-major
// (l + N j); u, v: masses in the same layouts.  The separable cost
// |x1_k - x2_l| + |y1_i - y2_j| is carried as a moment through both passes:
//   pass y (rows k of the first grid): S'(k, j) = sum_i phi(k,i) Ky(i,j),
//       T'(k, j) = sum_i phi(k,i) Ky(i,j) Gy(i,j)
//   pass x (columns j): S(l, j) = sum_k Kx(k,l) S'(k,j),
//       T(l, j) = sum_k Kx(k,l) (T'(k,j) + Gx(k,l) S'(k,j))
// so that err = sum v |S psi - 1| and <C, Gamma> = eps ln2 sum v T psi.
finom_status cost64_2d(finom_plan_s* p, const double* pa, const double* pb, const double* u,
                       const double* v, double* err, double* w1, cudaStream_t s) {
  finom_plan_s* ax = p->ax;
  finom_plan_s* ay = p->ay;
  const int64_t N = ax->N, M = ay->N;
  const size_t T = std::max((size_t)ax->C * M, (size_t)ay->C * N);
  double* scratch = nullptr;
  int32_t* ticket = nullptr;
  FINOM_CUDA(cudaMallocAsync(&scratch, sizeof(double) * (18 * T + 2), s));
  FINOM_CUDA(cudaMallocAsync(&ticket, sizeof(int32_t), s));
  FINOM_CUDA(cudaMemsetAsync(ticket, 0, sizeof(int32_t), s));
  double* z1 = p->st.z;
  double* z2 = p->st.z + N * M;
  // pass y: lines = rows k of the first grid (W = y1, weights phi), outputs
  // on y2 with frame 0, written column-major (k + N j)
  CostArgs a = cost_args(ay, (int)N, scratch, ticket);
  a.px = pa; a.u = u; a.w_ls = M; a.w_es = 1;
  a.z1 = z1; a.z2 = z2; a.z_ls = 1; a.z_es = N;
  finom_status rc = run_cost<C_ZERO_FRAME | C_INTER>(a, s);
  if (rc != FINOM_OK) return rc;
  // pass x: lines = columns j (W = x1 with the moments of pass y, O = x2)
  CostArgs b = cost_args(ax, (int)M, scratch, ticket);
  b.px = z1; b.u = z2; b.w_ls = N; b.w_es = 1;
  b.py = pb; b.v = v; b.o_ls = N; b.o_es = 1;
  rc = run_cost<C_LEVELS>(b, s);
  if (rc != FINOM_OK) return rc;
  double h[2];
  FINOM_CUDA(cudaMemcpyAsync(h, b.out, sizeof(h), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  cudaFreeAsync(scratch, s);
  cudaFreeAsync(ticket, s);
  *err = h[0];
  *w1 = h[1] * p->eps * 0.69314718055994530942;
  return FINOM_OK;
}

}  // namespace finom
