// Fused FINOM half step on the merged order of the two meshes.
//
// One CTA owns one tile of kTile merged points; thread t walks kElems
// consecutive points.  For the application with output side O and weight
// side W (O = x: K psi; O = y: K^T phi) the stabilised sums (Remark
// log-domain-stabilization) are carried in log2 form relative to a frame:
// at an O point its own absorbed potential, at a W point the frame of the O
// point before it.  Between consecutive points the lower-block recurrence
// (eq. p by dynamic programming) moves by A_k = (c_k - c_{k-1}) - g_k and the
// upper-block one (eq. q) by A'_k = -(c_k - c_{k-1}) - g_k (g = gap in bits);
// both are small once the frame tracks the potential, so their prefix sums
// D, PB over a thread's points stay precise in float32.  A thread
//   1. forms its prefix sums D, PB, its weight levels B (frame + potential +
//      log2 mass) and the maps of both recurrences over its points (each a
//      log-sum of its weights against their maximum);
//   2. gets its entry states from a scan of the 256 maps of the tile (two
//      warps, one per direction) seeded with the tile's carries;
//   3. at each O point adds p and q (eq. decompose to p+q) and performs the
//      Sinkhorn division of eq. iteration in the log domain: the absorbed
//      potential drops by log2 of the stabilised sum;
//   4. on request adds v_j |S_j - 1| to the marginal error (Algorithm 1 loop
//      head; Sec. 4) and forms the tile maps of the NEXT application (roles
//      swapped, new potentials), so the next launch finds its carries ready;
//   5. the last CTA to finish (ticket) scans the tile maps into per-tile
//      carries, reduces the error in float64 and updates the loop control.
//
// Line batches (the 2D application of Appendix A): the grid is lines x tiles;
// every line is one merged sequence of the same axis plan, with its own
// offset (and element stride) into the O- and W-side arrays.  The first pass
// of a 2D application has no O-side potentials (the paper's a_x = 0): its
// frames are taken from the W side (F_FRAME_W) and it writes log2 of the sums
// (F_QOUT); the second pass takes those as W potentials of unit mass
// (F_WVALID) and performs the division.
#pragma once

#include "dev_common.cuh"
#include "finom_internal.h"

namespace finom {

enum : int {
  F_OUT_POT = 1,     // write new O potentials
  F_OUT_LIN = 2,     // write S (linear, float64) per O point
  F_OUT_LOG = 4,     // write ln S (float64) per O point
  F_ERR = 8,         // marginal error + convergence flag
  F_NEXT = 16,       // maps of the next application (roles swapped)
  F_ITER_END = 32,   // this launch ends a Sinkhorn iteration
  F_CHECK_DONE = 64, // exit at once when the loop is done
  F_AGG_ONLY = 128,  // only the tile maps of this application (no outputs)
  F_FRAME_W = 256,   // O frames: minus the potential of the last W point before (no O data)
  F_WVALID = 512,    // W masses: 1 where the W potential is finite, else 0 (no W masses)
  F_QOUT = 1024,     // write log2 of the sums at the O points to q_out (no division)
};

// the launch kinds (compile-time flag sets)
constexpr int kModeHalfY = F_OUT_POT | F_ERR | F_NEXT | F_CHECK_DONE;      // psi <- v / K^T phi
constexpr int kModeHalfX = F_OUT_POT | F_NEXT | F_ITER_END | F_CHECK_DONE; // phi <- u / K psi
constexpr int kModeCheck = F_ERR;                                           // loop-head check only
constexpr int kModeLin = F_OUT_LIN;
constexpr int kModeLog = F_OUT_LOG;
constexpr int kModeAgg = F_AGG_ONLY;
// passes of the 2D application (line batches)
constexpr int kMode2Inner = F_QOUT | F_FRAME_W | F_CHECK_DONE;            // first pass: Q
constexpr int kMode2HalfB = F_OUT_POT | F_ERR | F_WVALID | F_CHECK_DONE;   // psi update + check
constexpr int kMode2HalfA = F_OUT_POT | F_WVALID | F_ITER_END | F_CHECK_DONE;
constexpr int kMode2Check = F_ERR | F_WVALID;
constexpr int kMode2InnerP = F_QOUT | F_FRAME_W;                            // products
constexpr int kMode2Log = F_OUT_LOG | F_WVALID;
constexpr int kMode2Lin = F_OUT_LIN | F_WVALID;
constexpr int kMode2AggInner = F_AGG_ONLY | F_FRAME_W;
constexpr int kMode2AggOuter = F_AGG_ONLY | F_WVALID;

template <class R>
struct ApplyArgs {
  using Pot = typename Tr<R>::Pot;
  using Mass = typename Tr<R>::Mass;
  const uint32_t* tbits;
  const R* gap;
  const int32_t* tile_x0;
  int64_t L;
  int C;              // tiles per line
  int lines;          // lines in the batch (1 for a 1D plan)
  int o_is_x;
  int64_t o_ls, o_es; // O-side arrays: offset between lines, stride between points
  int64_t w_ls, w_es; // W-side arrays: the same
  const int32_t* fw;  // F_FRAME_W: per tile, the W point whose potential frames the O point before it
  const Pot* pO;      // O-side absorbed potentials (the frame), log2 units
  const Mass* mO;     // O-side masses
  Pot* pO_out;        // O-side new potentials
  double* out;        // optional per-O-point output (F_OUT_LIN / F_OUT_LOG)
  Pot* q_out;         // F_QOUT: log2 sums at the O points
  int64_t q_ls, q_es; // F_QOUT: offset between lines, stride between points
  const Pot* pW;      // W-side absorbed potentials
  const Mass* mW;     // W-side masses
  R w_uniform;        // > 0: every W point has potential 0 and mass w_uniform
  R o_scale;          // > 0: the error uses psi = o_scale instead of mass * 2^P
  const R* carry_in;  // 4 per tile: forward (m, s) | backward (m, s) entering it; NULL = none
  R* agg_out;         // 6 per tile: tile maps of the target application
  R* carry_out;       // 4 per tile: carries of the target application (last CTA)
  double* part;       // one partial error sum per tile
  double* scal;       // [0] error of the last check
  int32_t* ctrl;      // [0] ticket [1] done [2] iteration [3] iterations at exit [4] converged
  double tol;
  int64_t maxit;
  int flags;
};

// padded index of a per-thread slot: conflict-free both for the threads that
// fill the slots and for the raking warp that reads 8 consecutive slots per lane
__device__ __forceinline__ int slot(int t) { return t + (t >> 5); }
constexpr int kSlots = kThreads + kThreads / 32;
constexpr int kPer = kThreads / 32;   // slots raked per lane

template <class R>
struct TileSmem {
  using Pot = typename Tr<R>::Pot;
  using Mass = typename Tr<R>::Mass;
  Pot pot[kTile + 2];
  Mass mass[kTile + 2];
  R tf[3][kSlots];   // per-thread forward maps (D, m, s); after the rake: carries (m, s)
  R tb[3][kSlots];   // per-thread backward maps; after the rake: carries
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

template <class R>
__device__ __forceinline__ void put_map(R (*arr)[kSlots], int t, const Agg<R>& a) {
  const int i = slot(t);
  arr[0][i] = a.D;
  arr[1][i] = a.m;
  arr[2][i] = a.s;
}
template <class R>
__device__ __forceinline__ Agg<R> get_map(R (*arr)[kSlots], int t) {
  const int i = slot(t);
  return {arr[0][i], arr[1][i], arr[2][i]};
}

// Warps 0 and 1: turn the 256 per-thread maps into per-thread entry states.
// Warp 0, forward: state entering thread t = threads 0..t-1 applied to cf.
// Warp 1, backward: state entering thread t from its right = threads
// 255..t+1 applied to cb.  Slots are overwritten with (m, s) of those states.
template <class R>
__device__ __forceinline__ void rake_scan(TileSmem<R>& sm, LS<R> cf, LS<R> cb) {
  const int lane = threadIdx.x & 31;
  const bool fwd = threadIdx.x < 32;
  R (*arr)[kSlots] = fwd ? sm.tf : sm.tb;
  Agg<R> f = agg_identity<R>();
  if (fwd) {
#pragma unroll
    for (int k = 0; k < kPer; ++k) f = agg_then(f, get_map(arr, lane * kPer + k));
  } else {
#pragma unroll
    for (int k = kPer - 1; k >= 0; --k) f = agg_then(f, get_map(arr, lane * kPer + k));
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    if (fwd) {
      Agg<R> t = shfl_up_agg(f, o);
      if (lane >= o) f = agg_then(t, f);
    } else {
      Agg<R> t = shfl_down_agg(f, o);
      if (lane + o < 32) f = agg_then(t, f);
    }
  }
  Agg<R> ex = fwd ? shfl_up_agg(f, 1) : shfl_down_agg(f, 1);
  if (fwd ? lane == 0 : lane == 31) ex = agg_identity<R>();
  LS<R> st = agg_apply(ex, fwd ? cf : cb);
#pragma unroll
  for (int kk = 0; kk < kPer; ++kk) {
    const int k = fwd ? kk : kPer - 1 - kk;
    const int t = lane * kPer + k;
    Agg<R> a = get_map(arr, t);
    arr[1][slot(t)] = st.m;
    arr[2][slot(t)] = st.s;
    st = agg_apply(a, st);
  }
}

// Warps 0 and 1: ordered composition of the 256 per-thread maps (warp 0
// forward, warp 1 backward); lane 0 of each writes its half of the tile map.
template <class R>
__device__ __forceinline__ void rake_reduce(TileSmem<R>& sm, R* out) {
  const int lane = threadIdx.x & 31;
  const bool fwd = threadIdx.x < 32;
  R (*arr)[kSlots] = fwd ? sm.tf : sm.tb;
  Agg<R> f = agg_identity<R>();
  if (fwd) {
#pragma unroll
    for (int k = 0; k < kPer; ++k) f = agg_then(f, get_map(arr, lane * kPer + k));
  } else {
#pragma unroll
    for (int k = kPer - 1; k >= 0; --k) f = agg_then(f, get_map(arr, lane * kPer + k));
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    Agg<R> t = shfl_down_agg(f, o);
    // forward: lane l gathers lanes l..l+2o-1 in order; backward: lanes l+2o-1..l
    if (lane + o < 32) f = fwd ? agg_then(f, t) : agg_then(t, f);
  }
  if (lane == 0) {
    R* o = out + (fwd ? 0 : 3);
    o[0] = f.D; o[1] = f.m; o[2] = f.s;
  }
}


#ifndef FINOM_CPASYNC
#define FINOM_CPASYNC 1
#endif

// asynchronous global -> shared copies (LDGSTS): every load of the tile is in
// flight at once and nothing passes through registers
template <class T>
__device__ __forceinline__ void cp_async(T* smem, const T* gmem) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8 || sizeof(T) == 16, "cp.async size");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(T) == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
  else if constexpr (sizeof(T) == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit_wait() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Terms of one application over the thread's points.  Frames come from po[]
// (po[o0] = the O point before the thread's first point, then one entry per
// O point); weights from pw[], mw[] starting at w0.  Outputs per point e:
//   D[e]  = A_0 + ... + A_e     (forward, frame-compensated log decays)
//   PB[e] = A'_0 + ... + A'_e   (backward)
//   L1[e] = B_e - D[e], L2[e] = B_e + PB[e]   (weight levels carried to the
//           segment start; kNegBig for points without weight)
//   mt[e] = mass mantissa in [1, 2) (0 for points without weight)
template <class R, bool kWValid = false>
__device__ __forceinline__ void seg_terms(uint32_t omask, uint32_t wmask, const R (&g)[kElems],
                                          const typename Tr<R>::Pot* po, int o0,
                                          const typename Tr<R>::Pot* pw,
                                          const typename Tr<R>::Mass* mw, int w0, R w_uniform,
                                          R (&D)[kElems], R (&PB)[kElems], R (&L1)[kElems],
                                          R (&L2)[kElems], R (&mt)[kElems]) {
  using T = Tr<R>;
  typename T::Pot cprev = po[o0];
  int oi = o0 + 1, wi = w0;
  R d = R(0), pb = R(0);
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    R dc = R(0);
    if ((omask >> e) & 1u) {
      const typename T::Pot c = po[oi++];
      dc = T::diff(c, cprev);
      cprev = c;
    }
    d += dc - g[e];
    pb -= dc + g[e];
    D[e] = d;
    PB[e] = pb;
    L1[e] = T::kNegBig;
    L2[e] = T::kNegBig;
    mt[e] = R(0);
    if ((wmask >> e) & 1u) {
      const typename T::Pot pv = (w_uniform > R(0)) ? T::zero() : pw[wi];
      typename T::Mass mv;
      if constexpr (kWValid) mv = (T::hi(pv) > T::kNegBig * R(0.5)) ? R(1) : R(0);
      else mv = (w_uniform > R(0)) ? (typename T::Mass)w_uniform : mw[wi];
      ++wi;
      R ex, mn;
      T::split(mv, ex, mn);
      if (mn > R(0)) {
        const R B = T::sum(cprev, pv, ex);
        L1[e] = B - d;
        L2[e] = B + pb;
        mt[e] = mn;
      }
    }
  }
}

// Maxima and spread of the levels; when the spread allows (fast path) the
// levels are replaced in place by the scaled terms mt 2^{L - M}.  Returns the
// maps of both recurrences over the thread's points:
//   forward  (D_last,  MF + D_last, sum tF),  backward (PB_last, MB, sum tB).
template <class R>
__device__ __forceinline__ bool seg_maps(const R (&D)[kElems], const R (&PB)[kElems],
                                         R (&L1)[kElems], R (&L2)[kElems], const R (&mt)[kElems],
                                         Agg<R>& mapF, Agg<R>& mapB, R& MF, R& MB) {
  using T = Tr<R>;
  MF = T::kNegBig;
  MB = T::kNegBig;
  R mnF = R(1e30), mnB = R(1e30);
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    MF = fmax(MF, L1[e]);
    MB = fmax(MB, L2[e]);
    if (mt[e] > R(0)) {
      mnF = fmin(mnF, L1[e]);
      mnB = fmin(mnB, L2[e]);
    }
  }
  // the fast path sums scaled terms; a term more than 60 bits below the
  // maximum would underflow while it may still matter at an earlier point
  const bool fast = fmax(MF - mnF, MB - mnB) <= R(60);
  R sF = R(0), sB = R(0);
  if (fast) {
#pragma unroll
    for (int e = 0; e < kElems; ++e) {
      L1[e] = mt[e] * T::ex2(L1[e] - MF);
      L2[e] = mt[e] * T::ex2(L2[e] - MB);
      sF += L1[e];
      sB += L2[e];
    }
    R m1 = MF + D[kElems - 1];
    renorm(m1, sF);
    R m2 = MB;
    renorm(m2, sB);
    mapF = {D[kElems - 1], m1, sF};
    mapB = {PB[kElems - 1], m2, sB};
  } else {
    R m1 = T::kNegBig, m2 = T::kNegBig;
#pragma unroll
    for (int e = 0; e < kElems; ++e) {
      if (mt[e] > R(0)) {
        ls_add_fast(m1, sF, L1[e], mt[e]);
        ls_add_fast(m2, sB, L2[e], mt[e]);
      }
    }
    m1 += D[kElems - 1];
    renorm(m1, sF);
    renorm(m2, sB);
    mapF = {D[kElems - 1], m1, sF};
    mapB = {PB[kElems - 1], m2, sB};
  }
  return fast;
}

template <class R>
__device__ __forceinline__ void load_gaps(const R* gap, int64_t seg, R (&g)[kElems]);

template <>
__device__ __forceinline__ void load_gaps<float>(const float* gap, int64_t seg, float (&g)[kElems]) {
  // gap arrays are padded to whole tiles, so the vector loads stay in bounds
  static_assert(kElems % 4 == 0 && kElems <= 16, "kElems");
  const float4* p = reinterpret_cast<const float4*>(gap + seg);
#pragma unroll
  for (int q = 0; q < kElems / 4; ++q) {
    float4 v = __ldg(p + q);
    g[4 * q] = v.x; g[4 * q + 1] = v.y; g[4 * q + 2] = v.z; g[4 * q + 3] = v.w;
  }
}

template <>
__device__ __forceinline__ void load_gaps<double>(const double* gap, int64_t seg, double (&g)[kElems]) {
  const double2* p = reinterpret_cast<const double2*>(gap + seg);
#pragma unroll
  for (int q = 0; q < kElems / 2; ++q) {
    double2 a = __ldg(p + q);
    g[2 * q] = a.x;
    g[2 * q + 1] = a.y;
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

// Last CTA: scan the tile maps agg[6*C] into carries[4*C] (all threads).
template <class R>
__device__ void carry_scan(const R* agg, R* carry, int C, TileSmem<R>& sm) {
  const int tid = threadIdx.x;
  const int per = (C + kThreads - 1) / kThreads;
  const int t0 = min(C, tid * per), t1 = min(C, t0 + per);
  Agg<R> f = agg_identity<R>(), b = agg_identity<R>();
  for (int t = t0; t < t1; ++t)
    f = agg_then(f, Agg<R>{__ldcg(agg + 6 * t + 0), __ldcg(agg + 6 * t + 1), __ldcg(agg + 6 * t + 2)});
  for (int t = t1 - 1; t >= t0; --t)
    b = agg_then(b, Agg<R>{__ldcg(agg + 6 * t + 3), __ldcg(agg + 6 * t + 4), __ldcg(agg + 6 * t + 5)});
  put_map(sm.tf, tid, f);
  put_map(sm.tb, tid, b);
  __syncthreads();
  if (tid < 64) rake_scan<R>(sm, ls_empty<R>(), ls_empty<R>());
  __syncthreads();
  LS<R> st = {sm.tf[1][slot(tid)], sm.tf[2][slot(tid)]};
  for (int t = t0; t < t1; ++t) {
    carry[4 * t + 0] = st.m;
    carry[4 * t + 1] = st.s;
    st = agg_apply(Agg<R>{__ldcg(agg + 6 * t + 0), __ldcg(agg + 6 * t + 1), __ldcg(agg + 6 * t + 2)}, st);
  }
  st = {sm.tb[1][slot(tid)], sm.tb[2][slot(tid)]};
  for (int t = t1 - 1; t >= t0; --t) {
    carry[4 * t + 2] = st.m;
    carry[4 * t + 3] = st.s;
    st = agg_apply(Agg<R>{__ldcg(agg + 6 * t + 3), __ldcg(agg + 6 * t + 4), __ldcg(agg + 6 * t + 5)}, st);
  }
}

// Last CTA, line batches: each thread scans the tile maps of whole lines
// (a line holds a few tiles) into their carries; lines start empty.
template <class R>
__device__ void carry_scan_lines(const R* agg, R* carry, int lines, int C) {
  for (int l = threadIdx.x; l < lines; l += kThreads) {
    const int64_t b = (int64_t)l * C;
    LS<R> st = ls_empty<R>();
    for (int t = 0; t < C; ++t) {
      carry[4 * (b + t) + 0] = st.m;
      carry[4 * (b + t) + 1] = st.s;
      const R* q = agg + 6 * (b + t);
      st = agg_apply(Agg<R>{__ldcg(q), __ldcg(q + 1), __ldcg(q + 2)}, st);
    }
    st = ls_empty<R>();
    for (int t = C - 1; t >= 0; --t) {
      carry[4 * (b + t) + 2] = st.m;
      carry[4 * (b + t) + 3] = st.s;
      const R* q = agg + 6 * (b + t) + 3;
      st = agg_apply(Agg<R>{__ldcg(q), __ldcg(q + 1), __ldcg(q + 2)}, st);
    }
  }
}

// Last CTA: float64 sum of the C per-tile partial sums (all threads).
template <class R>
__device__ double sum_parts(const double* part, int C, TileSmem<R>& sm) {
  double s = 0.0;
  for (int t = threadIdx.x; t < C; t += kThreads) s += __ldcg(part + t);
  s = warp_sum(s);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = s;
  __syncthreads();
  double tot = 0.0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) tot += sm.red[w];
  return tot;
}

template <class R, int kFlags>
#ifndef FINOM_MINB
#define FINOM_MINB 4
#endif
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? FINOM_MINB : 1) k_apply(ApplyArgs<R> a) {
  constexpr bool kAggOnly = (kFlags & F_AGG_ONLY) != 0;
  constexpr bool kFrameW = (kFlags & F_FRAME_W) != 0;
  constexpr bool kWValid = (kFlags & F_WVALID) != 0;
  using T = Tr<R>;
  using Pot = typename T::Pot;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem<R>& sm = *reinterpret_cast<TileSmem<R>*>(smem_raw);

  if ((kFlags & F_CHECK_DONE) && *(volatile int32_t*)(a.ctrl + 1)) return;

  const int tid = threadIdx.x;
  const int C = a.C;
  const int line = (int)(blockIdx.x / (unsigned)C);
  const int tile = (int)blockIdx.x - line * C;
  const int64_t ob = (int64_t)line * a.o_ls, wb = (int64_t)line * a.w_ls;
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
  load_gaps<R>(a.gap, seg, g);

  // stage the tile's O and W data (plus the point before the tile) in shared memory
  if (!kFrameW) {
    for (int i = tid; i < n_o + 1; i += kThreads) {
      const int64_t gi = ob + (int64_t)max(o_start - 1 + i, 0) * a.o_es;
#if FINOM_CPASYNC
      cp_async(&sm.pot[i], &a.pO[gi]);
      cp_async(&sm.mass[i], &a.mO[gi]);
#else
      sm.pot[i] = a.pO[gi];
      sm.mass[i] = a.mO[gi];
#endif
    }
  }
  if (a.w_uniform <= R(0) || (kFlags & F_NEXT)) {
    for (int i = tid; i < n_w + 1; i += kThreads) {
      const int64_t gi = wb + (int64_t)max(w_start - 1 + i, 0) * a.w_es;
#if FINOM_CPASYNC
      cp_async(&sm.pot[wofs + i], &a.pW[gi]);
      if (!kWValid) cp_async(&sm.mass[wofs + i], &a.mW[gi]);
#else
      sm.pot[wofs + i] = a.pW[gi];
      if (!kWValid) sm.mass[wofs + i] = a.mW[gi];
#endif
    }
  }
  const int o_before = block_exclusive_sum<kThreads>(__popc(omask), sm.iscan);
  // threads past the end of the sequence own no points; keep their index in range
  const int w_before = min((int)(seg - k0) - o_before, n_w);
#if FINOM_CPASYNC
  cp_async_commit_wait();
  __syncthreads();
#endif

  if constexpr (kFrameW) {
    // frame of an O point: minus the potential of the last W point before it
    // (of the line's first W point when there is none); the O point before the
    // tile gets the frame its own tile gave it
    const bool uni = a.w_uniform > R(0);
    int oi = o_before, wl = w_before;
#pragma unroll
    for (int e = 0; e < kElems; ++e) {
      if ((omask >> e) & 1u) {
        ++oi;
        sm.pot[oi] = uni ? T::zero() : T::neg(sm.pot[wofs + wl]);
      }
      if ((wmask >> e) & 1u) ++wl;
    }
    if (tid == 0) sm.pot[0] = uni ? T::zero() : T::neg(a.pW[wb + (int64_t)a.fw[tile] * a.w_es]);
    __syncthreads();
  }

  R D[kElems], PB[kElems], L1[kElems], L2[kElems], mt[kElems], MF, MB;
  Agg<R> mapF, mapB;
  seg_terms<R, kWValid>(omask, wmask, g, sm.pot, o_before, sm.pot + wofs, sm.mass + wofs, w_before + 1,
                        a.w_uniform, D, PB, L1, L2, mt);
  const bool fast = seg_maps<R>(D, PB, L1, L2, mt, mapF, mapB, MF, MB);

  if constexpr (kAggOnly) {
    put_map(sm.tf, tid, mapF);
    put_map(sm.tb, tid, mapB);
    __syncthreads();
    if (tid < 64) rake_reduce<R>(sm, a.agg_out + 6 * (int64_t)blockIdx.x);
    if (last_cta<R>(a.ctrl, a.lines * C, sm)) {
      if (a.lines == 1) carry_scan<R>(a.agg_out, a.carry_out, C, sm);
      else carry_scan_lines<R>(a.agg_out, a.carry_out, a.lines, C);
      if (tid == 0) a.ctrl[0] = 0;
    }
    return;
  }

  // entry states of the thread's points: forward (from the left) and
  // backward (from the right, in the frame of the thread's last point)
  LS<R> ef, eb;
  {
    LS<R> cf = ls_empty<R>(), cb = ls_empty<R>();
    if (a.carry_in) {
      const R* c = a.carry_in + 4 * (int64_t)blockIdx.x;
      cf = {__ldg(c + 0), __ldg(c + 1)};
      cb = {__ldg(c + 2), __ldg(c + 3)};
    }
    put_map(sm.tf, tid, mapF);
    put_map(sm.tb, tid, mapB);
    __syncthreads();
    if (tid < 64) rake_scan<R>(sm, cf, cb);
    __syncthreads();
    ef = {sm.tf[1][slot(tid)], sm.tf[2][slot(tid)]};
    eb = {sm.tb[1][slot(tid)], sm.tb[2][slot(tid)]};
  }

  // lam_e = log2 S_e in the point's own frame (S = p + q, eq. decompose to p+q):
  //   p_e = D_e + log2(entry_f (+) weights t <= e),  q_e = -PB_e + log2(entry_b' (+) weights t > e)
  // with entry_b' = the backward entry state carried to the segment start.
  R lam[kElems];
  const R ebm = eb.m + PB[kElems - 1];
  if (fast) {
    R qsuf[kElems];
    R acc = R(0);
#pragma unroll
    for (int e = kElems - 1; e >= 0; --e) {
      qsuf[e] = acc;         // backward terms strictly after e
      acc += L2[e];
    }
    // fold each entry state into its local sum once per thread; a part with
    // no weight must not set the level
    const R lf1 = (ef.s > R(0)) ? ef.m : T::kNegBig;
    const R LF = fmax(lf1, MF);
    const R cF0 = ef.s * T::ex2(lf1 - LF), cF1 = T::ex2(MF - LF);
    const R lb1 = (eb.s > R(0)) ? ebm : T::kNegBig;
    const R LB = fmax(lb1, MB);
    const R cB0 = eb.s * T::ex2(lb1 - LB), cB1 = T::ex2(MB - LB);
    R pf = R(0);
#pragma unroll
    for (int e = 0; e < kElems; ++e) {
      pf += L1[e];           // forward terms up to e
      const R sf = fma(cF1, pf, cF0), sb = fma(cB1, qsuf[e], cB0);
      const R a1 = (sf > R(0)) ? LF + D[e] : T::kNegBig;
      const R a2 = (sb > R(0)) ? LB - PB[e] : T::kNegBig;
      const R M = fmax(a1, a2);
      lam[e] = M + T::lg2(fma(sf, T::ex2(a1 - M), sb * T::ex2(a2 - M)));
    }
  } else {
    // levels spread over more than 60 bits: running-max log-sums
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

  // outputs at the O points: the division of eq. iteration in the log domain
  int oi = o_before;   // smem index of the O point before the current one
  R err = R(0);
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    if ((omask >> e) & 1u) {
      ++oi;
      const R l2 = lam[e];
      if constexpr ((kFlags & F_OUT_POT) != 0) sm.pot[oi] = T::sub(sm.pot[oi], l2);
      if constexpr ((kFlags & F_QOUT) != 0) {
        // an empty sum (no weight on the line) stays empty
        sm.pot[oi] = (l2 > T::kNegBig * R(0.5)) ? T::sub(sm.pot[oi], l2) : T::neg(T::none());
      }
      if constexpr ((kFlags & (F_OUT_LIN | F_OUT_LOG)) != 0) {
        double v;
        if constexpr ((kFlags & F_OUT_LIN) != 0) v = exp2((double)l2);
        else v = 0.69314718055994530942 * (double)l2;
        a.out[ob + (int64_t)(o_start + oi - 1) * a.o_es] = v;
      }
      if constexpr ((kFlags & F_ERR) != 0) {
        const R mo = (R)sm.mass[oi];
        if (a.o_scale > R(0)) {
          err += fabs(a.o_scale * T::ex2(l2) - mo);
        } else {
          // S - 1 without the cancellation of ex2(l2) - 1 near l2 = 0
          const R x = l2 * R(0.69314718055994530942);
          const R sm1 = (fabs(x) < R(0.03))
                            ? x * (R(1) + x * (R(0.5) + x * (R(1.0 / 6) + x * R(1.0 / 24))))
                            : T::ex2(l2) - R(1);
          err += mo * fabs(sm1);
        }
      }
    }
  }

  if (kFlags & F_ERR) {
    double e64 = warp_sum((double)err);
    if ((tid & 31) == 0) sm.red[tid >> 5] = e64;
  }
  __syncthreads();
  if ((kFlags & F_ERR) && tid == 0) {
    double tot = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) tot += sm.red[w];
    a.part[blockIdx.x] = tot;
  }
  if constexpr ((kFlags & F_OUT_POT) != 0) {
    for (int i = tid; i < n_o; i += kThreads) a.pO_out[ob + (int64_t)(o_start + i) * a.o_es] = sm.pot[1 + i];
  }
  if constexpr ((kFlags & F_QOUT) != 0) {
    const int64_t qb = (int64_t)line * a.q_ls;
    for (int i = tid; i < n_o; i += kThreads) a.q_out[qb + (int64_t)(o_start + i) * a.q_es] = T::neg(sm.pot[1 + i]);
  }
  if (kFlags & F_NEXT) {
    // next application: O' = current W (frames = current W potentials),
    // W' = current O (new potentials, same masses); same gaps
    seg_terms<R>(wmask, omask, g, sm.pot + wofs, w_before, sm.pot, sm.mass, o_before + 1, R(0), D,
                 PB, L1, L2, mt);
    (void)seg_maps<R>(D, PB, L1, L2, mt, mapF, mapB, MF, MB);
    put_map(sm.tf, tid, mapF);
    put_map(sm.tb, tid, mapB);
    __syncthreads();
    if (tid < 64) rake_reduce<R>(sm, a.agg_out + 6 * (int64_t)blockIdx.x);
  }

  if (last_cta<R>(a.ctrl, a.lines * C, sm)) {
    if (kFlags & F_NEXT) carry_scan<R>(a.agg_out, a.carry_out, C, sm);
    double errsum = 0.0;
    if (kFlags & F_ERR) errsum = sum_parts<R>(a.part, a.lines * C, sm);
    if (tid == 0) {
      int32_t* c = a.ctrl;
      if (kFlags & F_ERR) {
        a.scal[0] = errsum;
        if (errsum <= a.tol) {
          c[1] = 1;
          c[3] = c[2];
          c[4] = 1;
        }
      }
      if ((kFlags & F_ITER_END) && !c[1]) {
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
