// Fused FINOM half step on the merged order of the two meshes.
//
// One CTA owns one tile of kTile merged points; thread t walks kElems
// consecutive points.  For the application with output side O and weight
// side W (O = x: K psi; O = y: K^T phi) a thread
//   1. forms, for each of its points, the forward and backward exponents
//      A_k, A'_k and the log2 weight B_k of W points (frame: the absorbed
//      potential of the O side, carried across W points -- Remark
//      log-domain-stabilization);
//   2. runs the forward recurrence (eq. p by dynamic programming) and the
//      backward recurrence (eq. q by dynamic programming) over its points,
//      each as: local map -> block scan of maps -> carry from the tile carry
//      -> second local pass that emits the state at O points;
//   3. at O points adds p and q (eq. decompose to p+q) and performs the
//      Sinkhorn division of eq. iteration in the log domain: the absorbed
//      potential drops by log2 of the stabilised sum;
//   4. on request adds v_j |S_j - 1| to the marginal error (Algorithm 1
//      loop head; Sec. 4), and computes the tile's forward and backward maps
//      for the NEXT application (roles swapped, new potentials), so that the
//      next launch finds its tile carries ready;
//   5. the last CTA to finish (ticket) scans the tile maps into per-tile
//      carries, reduces the error in float64 and updates the loop control.
#pragma once

#include "dev_common.cuh"
#include "finom_internal.h"

namespace finom {

enum : int {
  F_OUT_POT = 1,     // write new O potentials
  F_OUT_LIN = 2,     // write S (linear, float64) per O point
  F_OUT_LOG = 4,     // write log S (natural log, float64) per O point
  F_ERR = 8,         // marginal error + convergence flag
  F_NEXT = 16,       // aggregates of the next application (roles swapped)
  F_ITER_END = 32,   // this launch ends a Sinkhorn iteration
  F_CHECK_DONE = 64, // exit at once when the loop is done
};

template <class R>
struct ApplyArgs {
  using Pot = typename Tr<R>::Pot;
  using Mass = typename Tr<R>::Mass;
  const uint32_t* tbits;
  const R* gap;
  const int32_t* tile_x0;
  int64_t L;
  int C;
  int o_is_x;
  const Pot* pO;      // O-side absorbed potentials (the frame), log2 units
  const Mass* mO;     // O-side masses
  Pot* pO_out;        // O-side new potentials
  double* out;        // optional per-O-point output (F_OUT_LIN / F_OUT_LOG)
  const Pot* pW;      // W-side absorbed potentials
  const Mass* mW;     // W-side masses
  R w_uniform;        // > 0: every W point has potential 0 and mass w_uniform
  R o_scale;          // > 0: the error uses psi = o_scale instead of mass * 2^P
  const R* carry_in;  // 4*C: forward (m, s) | backward (m, s) state entering each tile
  R* agg_out;         // 6*C: tile maps of the target application
  R* carry_out;       // 4*C: carries of the target application (last CTA)
  double* part;       // C partial error sums
  double* scal;       // [0] error of the last check
  int32_t* ctrl;      // [0] ticket [1] done [2] iteration [3] iterations at exit [4] converged
  double tol;
  int64_t maxit;
  int flags;
};

template <class R>
struct TileSmem {
  using Pot = typename Tr<R>::Pot;
  using Mass = typename Tr<R>::Mass;
  Pot pot[kTile + 2];
  Mass mass[kTile + 2];
  Agg<R> scan[kThreads / 32];
  double red[kThreads / 32];
  int iscan[kThreads / 32];
  int last;
};

// exclusive block sum of one int per thread
template <int NT>
__device__ __forceinline__ int block_exclusive_sum(int v, int* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  int wp = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w)
    if (w < warp) wp += sh[w];
  __syncthreads();
  return wp + inc - v;
}

// Per-point exponents of one application.  omask/wmask: which of the thread's
// points are O / W points.  Frames come from po[] (po[o0] = the O point before
// the thread's first point, then one entry per O point); weights from pw[],
// mw[] starting at index w0.
template <class R>
__device__ __forceinline__ void point_terms(uint32_t omask, uint32_t wmask, const R (&g)[kElems],
                                            const typename Tr<R>::Pot* po, int o0,
                                            const typename Tr<R>::Pot* pw,
                                            const typename Tr<R>::Mass* mw, int w0, R w_uniform,
                                            R (&Af)[kElems], R (&Ab)[kElems], R (&Bl)[kElems],
                                            R (&Bs)[kElems]) {
  using T = Tr<R>;
  typename T::Pot cprev = po[o0];
  int oi = o0 + 1, wi = w0;
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    R dc = R(0);
    if ((omask >> e) & 1u) {
      typename T::Pot c = po[oi++];
      dc = T::diff(c, cprev);
      cprev = c;
    }
    Af[e] = dc - g[e];
    Ab[e] = -dc - g[e];
    Bl[e] = T::kNegBig;
    Bs[e] = R(0);
    if ((wmask >> e) & 1u) {
      typename T::Pot pwv = (w_uniform > R(0)) ? T::zero() : pw[wi];
      typename T::Mass wv = (w_uniform > R(0)) ? (typename T::Mass)w_uniform : mw[wi];
      ++wi;
      R ex, mt;
      T::split(wv, ex, mt);
      if (mt > R(0)) {
        Bl[e] = T::sum(cprev, pwv, ex);
        Bs[e] = mt;
      }
    }
  }
}

template <class R>
__device__ __forceinline__ Agg<R> fwd_map(const R (&Af)[kElems], const R (&Bl)[kElems],
                                          const R (&Bs)[kElems], uint32_t wmask) {
  Agg<R> a = agg_identity<R>();
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    a.D += Af[e];
    a.m += Af[e];
    if ((wmask >> e) & 1u) {
      LS<R> t = ls_add(a.m, a.s, Bl[e], Bs[e]);
      a.m = t.m;
      a.s = t.s;
    }
  }
  return a;
}

template <class R>
__device__ __forceinline__ Agg<R> bwd_map(const R (&Ab)[kElems], const R (&Bl)[kElems],
                                          const R (&Bs)[kElems], uint32_t wmask) {
  Agg<R> a = agg_identity<R>();
#pragma unroll
  for (int e = kElems - 1; e >= 0; --e) {
    if ((wmask >> e) & 1u) {
      LS<R> t = ls_add(a.m, a.s, Bl[e], Bs[e]);
      a.m = t.m;
      a.s = t.s;
    }
    a.m += Ab[e];
    a.D += Ab[e];
  }
  return a;
}

// Last CTA: scan the tile maps agg[6*C] into carries[4*C].
template <class R>
__device__ void carry_scan(const R* agg, R* carry, int C, TileSmem<R>& sm) {
  const int tid = threadIdx.x;
  const int per = (C + kThreads - 1) / kThreads;
  const int t0 = min(C, tid * per), t1 = min(C, t0 + per);
  // forward
  Agg<R> loc = agg_identity<R>();
  for (int t = t0; t < t1; ++t) {
    Agg<R> a = {__ldcg(agg + 6 * t + 0), __ldcg(agg + 6 * t + 1), __ldcg(agg + 6 * t + 2)};
    loc = agg_then(loc, a);
  }
  Agg<R> tot;
  Agg<R> pre = block_exclusive_scan<R, kThreads, false>(loc, sm.scan, tot);
  LS<R> st = agg_apply(pre, ls_empty<R>());
  for (int t = t0; t < t1; ++t) {
    carry[4 * t + 0] = st.m;
    carry[4 * t + 1] = st.s;
    Agg<R> a = {__ldcg(agg + 6 * t + 0), __ldcg(agg + 6 * t + 1), __ldcg(agg + 6 * t + 2)};
    st = agg_apply(a, st);
  }
  // backward: tiles right to left
  loc = agg_identity<R>();
  for (int t = t1 - 1; t >= t0; --t) {
    Agg<R> a = {__ldcg(agg + 6 * t + 3), __ldcg(agg + 6 * t + 4), __ldcg(agg + 6 * t + 5)};
    loc = agg_then(loc, a);
  }
  pre = block_exclusive_scan<R, kThreads, true>(loc, sm.scan, tot);
  st = agg_apply(pre, ls_empty<R>());
  for (int t = t1 - 1; t >= t0; --t) {
    carry[4 * t + 2] = st.m;
    carry[4 * t + 3] = st.s;
    Agg<R> a = {__ldcg(agg + 6 * t + 3), __ldcg(agg + 6 * t + 4), __ldcg(agg + 6 * t + 5)};
    st = agg_apply(a, st);
  }
}

template <class R>
__device__ __forceinline__ void load_gaps(const R* gap, int64_t seg, int64_t L, R (&g)[kElems]);

template <>
__device__ __forceinline__ void load_gaps<float>(const float* gap, int64_t seg, int64_t L,
                                                 float (&g)[kElems]) {
  // gap arrays are padded to whole tiles, so the two vector loads stay in bounds
  const float4* p = reinterpret_cast<const float4*>(gap + seg);
  float4 a = __ldg(p), b = __ldg(p + 1);
  g[0] = a.x; g[1] = a.y; g[2] = a.z; g[3] = a.w;
  g[4] = b.x; g[5] = b.y; g[6] = b.z; g[7] = b.w;
  (void)L;
}

template <>
__device__ __forceinline__ void load_gaps<double>(const double* gap, int64_t seg, int64_t L,
                                                  double (&g)[kElems]) {
  const double2* p = reinterpret_cast<const double2*>(gap + seg);
#pragma unroll
  for (int q = 0; q < kElems / 2; ++q) {
    double2 a = __ldg(p + q);
    g[2 * q] = a.x;
    g[2 * q + 1] = a.y;
  }
  (void)L;
}

// Tile maps of one application (used by the aggregate-only launch and by the
// F_NEXT epilogue).  Thread 0 writes the tile's forward/backward maps.
template <class R>
__device__ __forceinline__ void tile_maps(uint32_t omask, uint32_t wmask, const R (&g)[kElems],
                                          const typename Tr<R>::Pot* po, int o0,
                                          const typename Tr<R>::Pot* pw,
                                          const typename Tr<R>::Mass* mw, int w0, R w_uniform,
                                          R* agg_out, int tile, TileSmem<R>& sm) {
  R Af[kElems], Ab[kElems], Bl[kElems], Bs[kElems];
  point_terms<R>(omask, wmask, g, po, o0, pw, mw, w0, w_uniform, Af, Ab, Bl, Bs);
  Agg<R> f = fwd_map<R>(Af, Bl, Bs, wmask);
  Agg<R> b = bwd_map<R>(Ab, Bl, Bs, wmask);
  Agg<R> tf = block_reduce<R, kThreads, false>(f, sm.scan);
  Agg<R> tb = block_reduce<R, kThreads, true>(b, sm.scan);
  if (threadIdx.x == 0) {
    R* a = agg_out + 6 * tile;
    a[0] = tf.D; a[1] = tf.m; a[2] = tf.s;
    a[3] = tb.D; a[4] = tb.m; a[5] = tb.s;
  }
}

// Ticket: returns true in the last CTA to finish (all others' writes visible).
template <class R>
__device__ __forceinline__ bool last_cta(int32_t* ticket, int C, TileSmem<R>& sm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    int t = atomicAdd(ticket, 1);
    sm.last = (t == C - 1);
  }
  __syncthreads();
  if (sm.last) __threadfence();
  return sm.last != 0;
}

template <class R, bool kAggOnly>
__global__ void __launch_bounds__(kThreads) k_apply(ApplyArgs<R> a) {
  using T = Tr<R>;
  using Pot = typename T::Pot;
  using Mass = typename T::Mass;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem<R>& sm = *reinterpret_cast<TileSmem<R>*>(smem_raw);

  if ((a.flags & F_CHECK_DONE) && *(volatile int32_t*)(a.ctrl + 1)) return;

  const int tid = threadIdx.x;
  const int tile = blockIdx.x;
  const int64_t k0 = (int64_t)tile * kTile;
  const int64_t kend = min(k0 + (int64_t)kTile, a.L);
  const int x0 = a.tile_x0[tile], x1 = a.tile_x0[tile + 1];
  const int y0 = (int)(k0 - x0), y1 = (int)(kend - x1);
  const int o_start = a.o_is_x ? x0 : y0;
  const int n_o = a.o_is_x ? (x1 - x0) : (y1 - y0);
  const int w_start = a.o_is_x ? y0 : x0;
  const int n_w = a.o_is_x ? (y1 - y0) : (x1 - x0);
  const int wofs = n_o + 1;   // smem index of the W point before the tile

  // this thread's points
  const int64_t seg = k0 + (int64_t)tid * kElems;
  uint32_t vmask = 0;
  if (seg < a.L) {
    int64_t nv = a.L - seg;
    vmask = nv >= kElems ? ((1u << kElems) - 1u) : ((1u << nv) - 1u);
  }
  uint32_t bits = (seg < a.L) ? ((a.tbits[seg >> 5] >> (seg & 31)) & ((1u << kElems) - 1u)) : 0u;
  const uint32_t xmask = bits & vmask, ymask = (~bits) & vmask;
  const uint32_t omask = a.o_is_x ? xmask : ymask;
  const uint32_t wmask = a.o_is_x ? ymask : xmask;
  R g[kElems];
  load_gaps<R>(a.gap, seg, a.L, g);

  const int o_before = block_exclusive_sum<kThreads>(__popc(omask), sm.iscan);
  // threads past the end of the sequence own no points; keep their index in range
  const int w_before = min((int)(seg - k0) - o_before, n_w);   // valid for threads with seg < L

  // stage the tile's O and W data (plus the point before the tile) in shared memory
  for (int i = tid; i < n_o + 1; i += kThreads) {
    int gi = max(o_start - 1 + i, 0);
    sm.pot[i] = a.pO[gi];
    sm.mass[i] = a.mO[gi];
  }
  if (a.w_uniform <= R(0) || (a.flags & F_NEXT)) {
    for (int i = tid; i < n_w + 1; i += kThreads) {
      int gi = max(w_start - 1 + i, 0);
      sm.pot[wofs + i] = a.pW[gi];
      sm.mass[wofs + i] = a.mW[gi];
    }
  }
  __syncthreads();

  if (kAggOnly) {
    tile_maps<R>(omask, wmask, g, sm.pot, o_before, sm.pot + wofs, sm.mass + wofs, w_before + 1,
                 a.w_uniform, a.agg_out, tile, sm);
    if (last_cta<R>(a.ctrl, a.C, sm)) {
      carry_scan<R>(a.agg_out, a.carry_out, a.C, sm);
      if (tid == 0) a.ctrl[0] = 0;
    }
    return;
  }

  R Af[kElems], Ab[kElems], Bl[kElems], Bs[kElems];
  point_terms<R>(omask, wmask, g, sm.pot, o_before, sm.pot + wofs, sm.mass + wofs, w_before + 1,
                 a.w_uniform, Af, Ab, Bl, Bs);

  // forward recurrence: local map, block scan, carried second pass
  Agg<R> tot;
  Agg<R> pre = block_exclusive_scan<R, kThreads, false>(fwd_map<R>(Af, Bl, Bs, wmask), sm.scan, tot);
  LS<R> st = agg_apply(pre, LS<R>{__ldg(a.carry_in + 4 * tile + 0), __ldg(a.carry_in + 4 * tile + 1)});
  R fm[kElems], fs[kElems];
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    st.m += Af[e];
    if ((wmask >> e) & 1u) st = ls_add(st.m, st.s, Bl[e], Bs[e]);
    fm[e] = st.m;
    fs[e] = st.s;
  }
  // backward recurrence
  pre = block_exclusive_scan<R, kThreads, true>(bwd_map<R>(Ab, Bl, Bs, wmask), sm.scan, tot);
  st = agg_apply(pre, LS<R>{__ldg(a.carry_in + 4 * tile + 2), __ldg(a.carry_in + 4 * tile + 3)});
  int oi = o_before + __popc(omask);   // smem index of this thread's last O point
  R err = R(0);
#pragma unroll
  for (int e = kElems - 1; e >= 0; --e) {
    if ((omask >> e) & 1u) {
      LS<R> s2 = ls_add(fm[e], fs[e], st.m, st.s);   // p + q (eq. decompose to p+q)
      R l2 = s2.m + T::lg2(s2.s);                      // log2 of the stabilised sum
      Pot c = sm.pot[oi];
      if (a.flags & F_OUT_POT) sm.pot[oi] = T::sub(c, l2);
      if (a.flags & (F_OUT_LIN | F_OUT_LOG)) {
        double v;
        if (a.flags & F_OUT_LIN) v = (double)s2.s * exp2((double)s2.m);
        else v = 0.69314718055994530942 * ((double)s2.m + log2((double)s2.s));
        a.out[o_start + oi - 1] = v;
      }
      if (a.flags & F_ERR) {
        R mo = (R)sm.mass[oi];
        if (a.o_scale > R(0)) {
          err += fabs(a.o_scale * T::ex2(l2) - mo);
        } else {
          // S - 1 without the cancellation of ex2(l2) - 1 near l2 = 0
          R x = l2 * R(0.69314718055994530942);
          R sm1 = (fabs(x) < R(0.03)) ? x * (R(1) + x * (R(0.5) + x * (R(1.0 / 6) + x * R(1.0 / 24))))
                                      : T::ex2(l2) - R(1);
          err += mo * fabs(sm1);
        }
      }
      --oi;
    }
    if ((wmask >> e) & 1u) st = ls_add(st.m, st.s, Bl[e], Bs[e]);
    st.m += Ab[e];
  }

  if (a.flags & F_ERR) {
    double e64 = warp_sum((double)err);
    if ((tid & 31) == 0) sm.red[tid >> 5] = e64;
  }
  __syncthreads();
  if ((a.flags & F_ERR) && tid == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += sm.red[w];
    a.part[tile] = s;
  }
  if (a.flags & F_OUT_POT) {
    for (int i = tid; i < n_o; i += kThreads) a.pO_out[o_start + i] = sm.pot[1 + i];
  }
  if (a.flags & F_NEXT) {
    // next application: O' = current W (frames = current W potentials),
    // W' = current O (new potentials, same masses)
    tile_maps<R>(wmask, omask, g, sm.pot + wofs, w_before, sm.pot, sm.mass, o_before + 1, R(0),
                 a.agg_out, tile, sm);
  }

  if (last_cta<R>(a.ctrl, a.C, sm)) {
    if (a.flags & F_NEXT) carry_scan<R>(a.agg_out, a.carry_out, a.C, sm);
    if (tid == 0) {
      int32_t* c = a.ctrl;
      if (a.flags & F_ERR) {
        double s = 0.0;
        for (int t = 0; t < a.C; ++t) s += __ldcg(a.part + t);
        a.scal[0] = s;
        if (s <= a.tol) {
          c[1] = 1;
          c[3] = c[2];
          c[4] = 1;
        }
      }
      if ((a.flags & F_ITER_END) && !c[1]) {
        c[2] += 1;
        if ((int64_t)c[2] >= a.maxit) {
          c[1] = 1;
          c[3] = c[2];
        }
      }
      c[0] = 0;
    }
  }
}

}  // namespace finom
