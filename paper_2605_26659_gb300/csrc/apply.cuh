// Fused FINOM half step on the merged order of the two meshes.
//
// One CTA owns one tile of E * kThreads merged points; thread t walks E
// consecutive points (E = kElems = 8 for 2D lines and batches; a 1D plan may
// use 1, 2 or 4 to spread small problems over more SMs).  For the application with output side O and weight
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

#include <cstddef>

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
  F_BATCH = 2048,    // units are the tiles of a batch of independent 1D instances
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
// batches of 1D instances: per-instance carries, errors and retirement come
// from k_batch_end, launched after each of these
constexpr int kModeBHalfY = F_OUT_POT | F_NEXT | F_ERR | F_CHECK_DONE | F_BATCH;
constexpr int kModeBHalfX = F_OUT_POT | F_NEXT | F_CHECK_DONE | F_BATCH;
constexpr int kModeBAgg = F_AGG_ONLY | F_BATCH;
constexpr int kModeBCheck = F_ERR | F_BATCH;

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
  // F_BATCH: units are global tiles; instance b owns tiles itile[b] .. itile[b+1]-1,
  // its points x[ioffx[b] ..), y[ioffy[b] ..) of the packed arrays, and C_b + 1
  // entries of tile_x0 from itile[b] + b.  Gaps and type bits are packed per tile.
  const int32_t* tinst;   // per tile: its instance
  const int32_t* itile;   // B + 1
  const int64_t* ioffx;   // B + 1
  const int64_t* ioffy;   // B + 1
  const int32_t* idone;   // per instance: nonzero once retired
  const int32_t* alist;   // the tiles of the active instances (rebuilt after each half step) ...
  const int32_t* acount;  // ... and their number; units index this list
  const R* iuni;          // per instance: (1/n_W, 1/n_O) while the start phi, psi apply, else NULL
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
  int elems;          // points per thread of the launch (the plan's tile / kThreads)
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
  Agg<R> wf[kThreads / 32];   // warp totals (block scans at the end of a launch)
  double red[kThreads / 32];
  int iscan[kThreads / 32];
  int last;
};
// the last CTA reuses pot and mass as one scratch area (carry_scan)
static_assert(offsetof(TileSmem<float>, mass) == sizeof(float2) * (kTile + 2), "layout");
static_assert(offsetof(TileSmem<double>, mass) == sizeof(double) * (kTile + 2), "layout");

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
template <class R, bool kWValid = false, int E = kElems>
__device__ __forceinline__ void seg_terms(uint32_t omask, uint32_t wmask, const R (&g)[E],
                                          const typename Tr<R>::Pot* po, int o0,
                                          const typename Tr<R>::Pot* pw,
                                          const typename Tr<R>::Mass* mw, int w0, R w_uniform,
                                          R (&D)[E], R (&PB)[E], R (&L1)[E],
                                          R (&L2)[E], R (&mt)[E]) {
  using T = Tr<R>;
  typename T::Pot cprev = po[o0];
  int oi = o0 + 1, wi = w0;
  R d = R(0), pb = R(0);
#pragma unroll
  for (int e = 0; e < E; ++e) {
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
template <class R, int E = kElems>
__device__ __forceinline__ bool seg_maps(const R (&D)[E], const R (&PB)[E],
                                         R (&L1)[E], R (&L2)[E], const R (&mt)[E],
                                         Agg<R>& mapF, Agg<R>& mapB, R& MF, R& MB) {
  using T = Tr<R>;
  MF = T::kNegBig;
  MB = T::kNegBig;
  R mnF = R(1e30), mnB = R(1e30);
#pragma unroll
  for (int e = 0; e < E; ++e) {
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
    for (int e = 0; e < E; ++e) {
      L1[e] = mt[e] * T::ex2(L1[e] - MF);
      L2[e] = mt[e] * T::ex2(L2[e] - MB);
      sF += L1[e];
      sB += L2[e];
    }
    R m1 = MF + D[E - 1];
    renorm(m1, sF);
    R m2 = MB;
    renorm(m2, sB);
    mapF = {D[E - 1], m1, sF};
    mapB = {PB[E - 1], m2, sB};
  } else {
    R m1 = T::kNegBig, m2 = T::kNegBig;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (mt[e] > R(0)) {
        ls_add_fast(m1, sF, L1[e], mt[e]);
        ls_add_fast(m2, sB, L2[e], mt[e]);
      }
    }
    m1 += D[E - 1];
    renorm(m1, sF);
    renorm(m2, sB);
    mapF = {D[E - 1], m1, sF};
    mapB = {PB[E - 1], m2, sB};
  }
  return fast;
}

// the E gaps of a thread's points (seg is a multiple of E; gap arrays are
// padded to whole tiles, so the vector loads stay in bounds)
template <class R, int E = kElems>
__device__ __forceinline__ void load_gaps(const R* gap, int64_t seg, R (&g)[E]) {
  static_assert(E == 1 || E == 2 || E == 4 || E == 8 || E == 16, "points per thread");
  if constexpr (sizeof(R) == 4 && E >= 4) {
    const float4* p = reinterpret_cast<const float4*>(gap + seg);
#pragma unroll
    for (int q = 0; q < E / 4; ++q) {
      float4 v = __ldg(p + q);
      g[4 * q] = v.x; g[4 * q + 1] = v.y; g[4 * q + 2] = v.z; g[4 * q + 3] = v.w;
    }
  } else if constexpr (sizeof(R) == 4 && E == 2) {
    float2 v = __ldg(reinterpret_cast<const float2*>(gap + seg));
    g[0] = v.x; g[1] = v.y;
  } else if constexpr (sizeof(R) == 8 && E >= 2) {
    const double2* p = reinterpret_cast<const double2*>(gap + seg);
#pragma unroll
    for (int q = 0; q < E / 2; ++q) {
      double2 v = __ldg(p + q);
      g[2 * q] = v.x; g[2 * q + 1] = v.y;
    }
  } else {
    g[0] = __ldg(gap + seg);
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

template <class R>
__device__ __forceinline__ Agg<R> ld_map(const R* p) {
  return {__ldcg(p), __ldcg(p + 1), __ldcg(p + 2)};
}

// Exclusive scan of one per-thread map per thread over the block, in one
// direction, seeded with cin: the state entering thread t from the left
// (forward) or from the right (backward).  Shuffle scans inside each warp,
// warp totals through shared memory; *total receives the block's map.
template <class R, bool kBackward>
__device__ __forceinline__ LS<R> block_scan_dir(TileSmem<R>& sm, Agg<R> f, LS<R> cin, Agg<R>* total) {
  // only the end of a launch runs this: loops stay rolled (small code, few
  // instruction-cache misses on the SM that runs it)
  constexpr int NW = kThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 1
  for (int o = 1; o < 32; o <<= 1) {
    const Agg<R> t = kBackward ? shfl_down_agg(f, o) : shfl_up_agg(f, o);
    if (kBackward ? (lane + o < 32) : (lane >= o)) f = agg_then(t, f);
  }
  __syncthreads();   // the warp-total slots may still be read by a previous scan
  if (kBackward ? lane == 0 : lane == 31) sm.wf[warp] = f;
  Agg<R> fx = kBackward ? shfl_down_agg(f, 1) : shfl_up_agg(f, 1);
  if (kBackward ? lane == 31 : lane == 0) fx = agg_identity<R>();
  __syncthreads();
  LS<R> st = cin;
  Agg<R> tot = agg_identity<R>();
  if (!kBackward) {
#pragma unroll 1
    for (int w = 0; w < NW; ++w) {
      if (w < warp) st = agg_apply(sm.wf[w], st);
      tot = agg_then(tot, sm.wf[w]);
    }
  } else {
#pragma unroll 1
    for (int w = NW - 1; w >= 0; --w) {
      if (w > warp) st = agg_apply(sm.wf[w], st);
      tot = agg_then(tot, sm.wf[w]);
    }
  }
  if (total) *total = tot;
  return agg_apply(fx, st);
}

// Last CTA: scan the tile maps agg[6*C] into carries[4*C] (all threads).
// One direction at a time, a chunk of tiles at a time: the chunk's maps are
// copied with coalesced loads into the (now free) staging arrays, each thread
// composes a run of them, a block scan gives every run its entry state, the
// runs are replayed into carries in shared memory, and those are stored with
// coalesced writes.  The state leaving a chunk enters the next one.
template <class R>
__device__ void carry_scan(const R* agg, R* carry, int C, TileSmem<R>& sm) {
  R* buf = reinterpret_cast<R*>(sm.pot);   // pot and mass are adjacent: one scratch area
  constexpr int kBytes = sizeof(sm.pot) + sizeof(sm.mass);
  constexpr int kPerT = (kBytes / (int)sizeof(R)) / (5 * kThreads);   // tiles per thread per chunk
  static_assert(kPerT >= 1, "scratch");
  constexpr int kQ = kPerT * kThreads;                               // tiles per chunk
  R* cbuf = buf + 3 * kQ;                                            // 2 carry values per tile
  const int tid = threadIdx.x;
#pragma unroll 1
  for (int dir = 0; dir < 2; ++dir) {
    LS<R> run = ls_empty<R>();   // state entering the next chunk
    const int nch = (C + kQ - 1) / kQ;
#pragma unroll 1
    for (int ci = 0; ci < nch; ++ci) {
      const int ch = dir == 0 ? ci : nch - 1 - ci;
      const int c0 = ch * kQ, nq = min(kQ, C - c0);
      __syncthreads();
      for (int i = tid; i < 3 * nq; i += kThreads) {
        const int j = i / 3, d = i - 3 * j;
        buf[i] = __ldcg(agg + 6 * (int64_t)(c0 + j) + 3 * dir + d);
      }
      __syncthreads();
      const int j0 = tid * kPerT;
      Agg<R> f = agg_identity<R>();
      if (dir == 0) {
#pragma unroll 1
        for (int k = 0; k < kPerT; ++k)
          if (j0 + k < nq) f = agg_then(f, Agg<R>{buf[3 * (j0 + k)], buf[3 * (j0 + k) + 1], buf[3 * (j0 + k) + 2]});
      } else {
#pragma unroll 1
        for (int k = kPerT - 1; k >= 0; --k)
          if (j0 + k < nq) f = agg_then(f, Agg<R>{buf[3 * (j0 + k)], buf[3 * (j0 + k) + 1], buf[3 * (j0 + k) + 2]});
      }
      Agg<R> tot;
      LS<R> st = dir == 0 ? block_scan_dir<R, false>(sm, f, run, &tot) : block_scan_dir<R, true>(sm, f, run, &tot);
      if (dir == 0) {
#pragma unroll 1
        for (int k = 0; k < kPerT; ++k) {
          if (j0 + k < nq) {
            cbuf[2 * (j0 + k)] = st.m;
            cbuf[2 * (j0 + k) + 1] = st.s;
            st = agg_apply(Agg<R>{buf[3 * (j0 + k)], buf[3 * (j0 + k) + 1], buf[3 * (j0 + k) + 2]}, st);
          }
        }
      } else {
#pragma unroll 1
        for (int k = kPerT - 1; k >= 0; --k) {
          if (j0 + k < nq) {
            cbuf[2 * (j0 + k)] = st.m;
            cbuf[2 * (j0 + k) + 1] = st.s;
            st = agg_apply(Agg<R>{buf[3 * (j0 + k)], buf[3 * (j0 + k) + 1], buf[3 * (j0 + k) + 2]}, st);
          }
        }
      }
      run = agg_apply(tot, run);
      __syncthreads();
      for (int i = tid; i < 2 * nq; i += kThreads) {
        const int j = i >> 1, d = i & 1;
        carry[4 * (int64_t)(c0 + j) + 2 * dir + d] = cbuf[i];
      }
    }
  }
}

// Last CTA, line batches: each thread scans the tile maps of whole lines
// (a line holds a few tiles) into their carries; lines start empty.  The
// maps of a chunk of tiles are requested before the chain uses them.
template <class R>
__device__ void carry_scan_lines(const R* agg, R* carry, int lines, int C) {
  constexpr int kChunk = 4;
  for (int l = threadIdx.x; l < lines; l += kThreads) {
    const int64_t b0 = (int64_t)l * C;
    LS<R> st = ls_empty<R>();
    for (int c = 0; c < C; c += kChunk) {
      Agg<R> m[kChunk];
#pragma unroll
      for (int k = 0; k < kChunk; ++k) m[k] = (c + k < C) ? ld_map(agg + 6 * (b0 + c + k)) : agg_identity<R>();
#pragma unroll
      for (int k = 0; k < kChunk; ++k) {
        if (c + k < C) {
          carry[4 * (b0 + c + k) + 0] = st.m;
          carry[4 * (b0 + c + k) + 1] = st.s;
          st = agg_apply(m[k], st);
        }
      }
    }
    st = ls_empty<R>();
    for (int c = C; c > 0; c -= kChunk) {
      Agg<R> m[kChunk];
#pragma unroll
      for (int k = 0; k < kChunk; ++k)
        m[k] = (c - 1 - k >= 0) ? ld_map(agg + 6 * (b0 + c - 1 - k) + 3) : agg_identity<R>();
#pragma unroll
      for (int k = 0; k < kChunk; ++k) {
        if (c - 1 - k >= 0) {
          carry[4 * (b0 + c - 1 - k) + 2] = st.m;
          carry[4 * (b0 + c - 1 - k) + 3] = st.s;
          st = agg_apply(m[k], st);
        }
      }
    }
  }
}

// Last CTA: this thread's share of the float64 sum of the C per-tile partials
__device__ __forceinline__ double load_parts(const double* part, int C) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int t = threadIdx.x;
#pragma unroll 1
  for (; t + 3 * kThreads < C; t += 4 * kThreads) {
    s0 += __ldcg(part + t);
    s1 += __ldcg(part + t + kThreads);
    s2 += __ldcg(part + t + 2 * kThreads);
    s3 += __ldcg(part + t + 3 * kThreads);
  }
  for (; t < C; t += kThreads) s0 += __ldcg(part + t);
  return (s0 + s1) + (s2 + s3);
}

// Last CTA: sum over the block (all threads; every thread gets the total)
template <class R>
__device__ double block_sum(double s, TileSmem<R>& sm) {
  s = warp_sum(s);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = s;
  __syncthreads();
  double tot = 0.0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) tot += sm.red[w];
  return tot;
}

// Outputs at one O point (smem slot oi) from l2 = log2 S in its frame: the
// division of eq. iteration in the log domain (new absorbed potential), the
// log2 sums of a first 2D pass, products, and the marginal error term.
template <class R, int kFlags>
__device__ __forceinline__ void emit_o(const ApplyArgs<R>& a, TileSmem<R>& sm, int oi, R l2, int64_t ob,
                                       int o_start, R o_scale, R& err) {
  using T = Tr<R>;
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
    if (o_scale > R(0)) {
      err += fabs(o_scale * T::ex2(l2) - mo);
    } else {
      // S - 1 without the cancellation of ex2(l2) - 1 near l2 = 0
      const R x = l2 * R(0.69314718055994530942);
      const R sm1 = (fabs(x) < R(0.03)) ? x * (R(1) + x * (R(0.5) + x * (R(1.0 / 6) + x * R(1.0 / 24))))
                                        : T::ex2(l2) - R(1);
      err += mo * fabs(sm1);
    }
  }
}

// Last CTA of a launch with at most kSmallTail tiles on one line: warp 0
// scans the forward tile maps, warp 1 the backward ones, 32 tiles per round
// (one per lane, shuffle scans; the state leaving a round enters the next),
// warp 2 sums the error partials; every thread gets the error sum.  Short
// dependent chains and little code for the small problems whose launches
// this tail would otherwise dominate.
constexpr int kSmallTail = 128;

template <class R, int kFlags>
__device__ double finish_small(const ApplyArgs<R>& a, TileSmem<R>& sm, int units) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if ((kFlags & (F_NEXT | F_AGG_ONLY)) && warp < 2) {
    const bool bwd = warp == 1;
    LS<R> run = ls_empty<R>();
    const int rounds = (a.C + 31) >> 5;
#pragma unroll 1
    for (int r = 0; r < rounds; ++r) {
      const int t = bwd ? a.C - 1 - (32 * r + lane) : 32 * r + lane;   // this lane's tile
      Agg<R> f = t >= 0 && t < a.C ? ld_map(a.agg_out + 6 * t + (bwd ? 3 : 0)) : agg_identity<R>();
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const Agg<R> u = shfl_up_agg(f, o);
        if (lane >= o) f = agg_then(u, f);
      }
      Agg<R> fx = shfl_up_agg(f, 1);
      if (lane == 0) fx = agg_identity<R>();
      const LS<R> st = agg_apply(fx, run);
      if (t >= 0 && t < a.C) {
        a.carry_out[4 * t + (bwd ? 2 : 0)] = st.m;
        a.carry_out[4 * t + (bwd ? 3 : 1)] = st.s;
      }
      const Agg<R> tot = {__shfl_sync(0xffffffffu, f.D, 31), __shfl_sync(0xffffffffu, f.m, 31),
                          __shfl_sync(0xffffffffu, f.s, 31)};
      run = agg_apply(tot, run);
    }
  }
  if ((kFlags & F_ERR) && warp == 2) {
    double e = 0.0;
#pragma unroll 1
    for (int i = lane; i < units; i += 32) e += __ldcg(a.part + i);
    e = warp_sum(e);
    if (lane == 0) sm.red[0] = e;
  }
  __syncthreads();
  return (kFlags & F_ERR) ? sm.red[0] : 0.0;
}

// Last CTA of a launch with kSmallTail < C <= mid_tail<R>() tiles on one line
// (1025 float32, 683 float64):
// four warps per direction.  Warp q of a direction scans the q-th quarter of
// the tiles (in scan order: left to right forward, right to left backward)
// in rounds of 32 and keeps each tile's exclusive prefix map within its
// quarter in shared memory; the quarter totals then give each quarter its
// entry state, which the same warp pushes through its tiles' prefix maps.
template <class R>
constexpr int mid_tail() {   // tiles whose prefix maps (6 values) fit in the staging arrays
  return (int)((sizeof(TileSmem<R>::pot) + sizeof(TileSmem<R>::mass)) / (6 * sizeof(R)));
}

template <class R, int kFlags>
__device__ double finish_mid(const ApplyArgs<R>& a, TileSmem<R>& sm, int units) {
  constexpr int kMidTail = mid_tail<R>();
  R* pre = reinterpret_cast<R*>(sm.pot);   // [dir][tile][3]: prefix maps (pot and mass are adjacent)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int C = a.C;
  const bool bwd = warp >= 4;
  const int q = warp & 3;
  const int Q = (C + 3) >> 2;
  const int k0 = q * Q, k1 = min(k0 + Q, C);
  R* mine = pre + (bwd ? 3 * kMidTail : 0);
  Agg<R> run = agg_identity<R>();
  double e = 0.0;
  if (kFlags & (F_NEXT | F_AGG_ONLY)) {
#pragma unroll 1
    for (int kb = k0; kb < k1; kb += 32) {
      const int k = kb + lane;
      const int t = bwd ? C - 1 - k : k;
      Agg<R> f = k < k1 ? ld_map(a.agg_out + 6 * t + (bwd ? 3 : 0)) : agg_identity<R>();
#pragma unroll 1
      for (int o = 1; o < 32; o <<= 1) {
        const Agg<R> u = shfl_up_agg(f, o);
        if (lane >= o) f = agg_then(u, f);
      }
      Agg<R> fx = shfl_up_agg(f, 1);
      if (lane == 0) fx = agg_identity<R>();
      if (k < k1) {
        const Agg<R> p = agg_then(run, fx);
        mine[3 * k] = p.D;
        mine[3 * k + 1] = p.m;
        mine[3 * k + 2] = p.s;
      }
      const Agg<R> tot = {__shfl_sync(0xffffffffu, f.D, 31), __shfl_sync(0xffffffffu, f.m, 31),
                          __shfl_sync(0xffffffffu, f.s, 31)};
      run = agg_then(run, tot);
    }
    if (lane == 0) sm.wf[warp] = run;
  }
  if (kFlags & F_ERR) {
    // error partials: every thread sums a strided share (float64)
#pragma unroll 1
    for (int i = threadIdx.x; i < units; i += kThreads) e += __ldcg(a.part + i);
  }
  __syncthreads();
  if (kFlags & (F_NEXT | F_AGG_ONLY)) {
    LS<R> in = ls_empty<R>();
#pragma unroll 1
    for (int w = 0; w < q; ++w) in = agg_apply(sm.wf[(bwd ? 4 : 0) + w], in);
#pragma unroll 1
    for (int k = k0 + lane; k < k1; k += 32) {
      const int t = bwd ? C - 1 - k : k;
      const LS<R> st = agg_apply(Agg<R>{mine[3 * k], mine[3 * k + 1], mine[3 * k + 2]}, in);
      a.carry_out[4 * t + (bwd ? 2 : 0)] = st.m;
      a.carry_out[4 * t + (bwd ? 3 : 1)] = st.s;
    }
  }
  double errsum = 0.0;
  if (kFlags & F_ERR) errsum = block_sum<R>(e, sm);
  return errsum;
}

// The end of a launch, in the CTA that finishes last: carries of the next
// application, the float64 error sum, the loop control.  This code runs once
// per launch on one SM, mostly from a cold instruction cache: its loops stay
// rolled.
template <class R, int kFlags>
__device__ void finish_launch(const ApplyArgs<R>& a, TileSmem<R>& sm, int units) {
  double errsum = 0.0;
  if (a.lines == 1 && a.C <= kSmallTail) {
    errsum = finish_small<R, kFlags>(a, sm, units);
  } else if (a.lines == 1 && a.C <= mid_tail<R>()) {
    errsum = finish_mid<R, kFlags>(a, sm, units);
  } else {
    // the error partials are requested first so that their loads overlap the scan
    double ep = 0.0;
    if (kFlags & F_ERR) ep = load_parts(a.part, units);
    if (kFlags & (F_NEXT | F_AGG_ONLY)) {
      if (a.lines == 1) carry_scan<R>(a.agg_out, a.carry_out, a.C, sm);
      else carry_scan_lines<R>(a.agg_out, a.carry_out, a.lines, a.C);
    }
    if (kFlags & F_ERR) errsum = block_sum<R>(ep, sm);
  }
  if (threadIdx.x == 0) {
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

// One unit (line, tile) of a launch: steps 1-4 of the header comment.
template <class R, int kFlags, int E>
__device__ __forceinline__ bool apply_unit(const ApplyArgs<R>& a, TileSmem<R>& sm, int unit, bool first) {
  static_assert(E <= kElems, "the shared tile is sized for kElems points per thread");
  constexpr int kT = E * kThreads;   // merged points per tile
  constexpr bool kAggOnly = (kFlags & F_AGG_ONLY) != 0;
  constexpr bool kFrameW = (kFlags & F_FRAME_W) != 0;
  constexpr bool kWValid = (kFlags & F_WVALID) != 0;
  using T = Tr<R>;
  using Pot = typename T::Pot;
  constexpr bool kBatch = (kFlags & F_BATCH) != 0;
  // the launches of 1D plans: one line, unit strides, no offsets
  constexpr bool kUnit = (kFlags & (F_FRAME_W | F_WVALID | F_QOUT | F_BATCH)) == 0;
  // batches: unit strides, an offset per instance
  constexpr bool kStride1 = (kFlags & (F_FRAME_W | F_WVALID | F_QOUT)) == 0;
  const int tid = threadIdx.x;
  const int C = a.C;
  // geometry of the unit: its line (or instance), tile, sequence length, the
  // offsets of its O and W data and of its packed gaps and type bits
  int line, tile, x0, x1;
  int64_t L, ob, wb, pos0 = 0;
  R w_uniform = a.w_uniform, o_scale = a.o_scale;
  if constexpr (kBatch) {
    const int b = a.tinst[unit];
    const int tb = a.itile[b];
    line = b;
    tile = unit - tb;
    const int64_t xb = a.ioffx[b], yb = a.ioffy[b];
    L = (a.ioffx[b + 1] - xb) + (a.ioffy[b + 1] - yb);
    ob = a.o_is_x ? xb : yb;
    wb = a.o_is_x ? yb : xb;
    const int32_t* tx = a.tile_x0 + tb + b;
    x0 = tx[tile];
    x1 = tx[tile + 1];
    pos0 = (int64_t)tb * kT;
    if (a.iuni) {
      w_uniform = a.iuni[2 * b];
      o_scale = a.iuni[2 * b + 1];
    }
  } else {
    line = unit / C;
    tile = unit - line * C;
    L = a.L;
    ob = (int64_t)line * a.o_ls;
    wb = (int64_t)line * a.w_ls;
    x0 = a.tile_x0[tile];
    x1 = a.tile_x0[tile + 1];
  }
  const int64_t k0 = (int64_t)tile * kT;
  const int64_t kend = min(k0 + (int64_t)kT, L);
  const int y0 = (int)(k0 - x0), y1 = (int)(kend - x1);
  const int o_start = a.o_is_x ? x0 : y0;
  const int n_o = a.o_is_x ? (x1 - x0) : (y1 - y0);
  const int w_start = a.o_is_x ? y0 : x0;
  const int n_w = a.o_is_x ? (y1 - y0) : (x1 - x0);
  const int wofs = n_o + 1;   // smem index of the W point before the tile

  // this thread's points
  const int64_t seg = k0 + (int64_t)tid * E;
  const int64_t gseg = seg + pos0;   // position in the packed gap / type-bit arrays
  uint32_t vmask = 0;
  if (seg < L) {
    int64_t nv = L - seg;
    vmask = nv >= E ? ((1u << E) - 1u) : ((1u << nv) - 1u);
  }
  uint32_t bits = (seg < L) ? ((a.tbits[gseg >> 5] >> (gseg & 31)) & ((1u << E) - 1u)) : 0u;
  const uint32_t xmask = bits & vmask, ymask = (~bits) & vmask;
  const uint32_t omask = a.o_is_x ? xmask : ymask;
  const uint32_t wmask = a.o_is_x ? ymask : xmask;
  R g[E];
  load_gaps<R, E>(a.gap, gseg, g);

  // stage the tile's O and W data (plus the point before the tile) in shared
  // memory.  The O side is never written by the launch just before this one
  // (every launch writes only its own O side, and consecutive launches
  // alternate sides), so the first unit stages it before waiting for that
  // launch (programmatic dependent launch); the W side, the carries and the
  // loop control come after the wait.
  if (!kFrameW) {
    for (int i = tid; i < n_o + 1; i += kThreads) {
      const int64_t gi = kUnit      ? (int64_t)max(o_start - 1 + i, 0)
                         : kStride1 ? ob + max(o_start - 1 + i, 0)
                                    : ob + (int64_t)max(o_start - 1 + i, 0) * a.o_es;
      cp_async(&sm.pot[i], &a.pO[gi]);
      cp_async(&sm.mass[i], &a.mO[gi]);
    }
  }
  const int o_before = block_exclusive_sum<kThreads>(__popc(omask), sm.iscan);
  // threads past the end of the sequence own no points; keep their index in range
  const int w_before = min((int)(seg - k0) - o_before, n_w);
  if (first) {
    griddep_wait();
    if ((kFlags & F_CHECK_DONE) && *(volatile int32_t*)(a.ctrl + 1)) {
      cp_async_commit_wait();
      return false;
    }
    griddep_launch_dependents();
  }
  if (w_uniform <= R(0) || (kFlags & F_NEXT)) {
    for (int i = tid; i < n_w + 1; i += kThreads) {
      const int64_t gi = kUnit      ? (int64_t)max(w_start - 1 + i, 0)
                         : kStride1 ? wb + max(w_start - 1 + i, 0)
                                    : wb + (int64_t)max(w_start - 1 + i, 0) * a.w_es;
      cp_async(&sm.pot[wofs + i], &a.pW[gi]);
      if (!kWValid) cp_async(&sm.mass[wofs + i], &a.mW[gi]);
    }
  }
  cp_async_commit_wait();
  __syncthreads();

  if constexpr (kFrameW) {
    // frame of an O point: minus the potential of the last W point before it
    // (of the line's first W point when there is none); the O point before the
    // tile gets the frame its own tile gave it
    const bool uni = w_uniform > R(0);
    int oi = o_before, wl = w_before;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if ((omask >> e) & 1u) {
        ++oi;
        sm.pot[oi] = uni ? T::zero() : T::neg(sm.pot[wofs + wl]);
      }
      if ((wmask >> e) & 1u) ++wl;
    }
    if (tid == 0) sm.pot[0] = uni ? T::zero() : T::neg(a.pW[wb + (int64_t)a.fw[tile] * a.w_es]);
    __syncthreads();
  }

  R D[E], PB[E], L1[E], L2[E], mt[E], MF, MB;
  Agg<R> mapF, mapB;
  seg_terms<R, kWValid, E>(omask, wmask, g, sm.pot, o_before, sm.pot + wofs, sm.mass + wofs, w_before + 1,
                        w_uniform, D, PB, L1, L2, mt);
  const bool fast = seg_maps<R, E>(D, PB, L1, L2, mt, mapF, mapB, MF, MB);

  if constexpr (kAggOnly) {
    put_map(sm.tf, tid, mapF);
    put_map(sm.tb, tid, mapB);
    __syncthreads();
    if (tid < 64) rake_reduce<R>(sm, a.agg_out + 6 * (int64_t)unit);
    return true;
  }

  // entry states of the thread's points: forward (from the left) and
  // backward (from the right, in the frame of the thread's last point)
  LS<R> ef, eb;
  {
    LS<R> cf = ls_empty<R>(), cb = ls_empty<R>();
    if (a.carry_in) {
      const R* c = a.carry_in + 4 * (int64_t)unit;
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
  // with entry_b' = the backward entry state carried to the segment start;
  // each lam goes straight to its O point's outputs
  const R ebm = eb.m + PB[E - 1];
  int oi = o_before;   // smem index of the O point before the current one
  R err = R(0);
  if (fast) {
    // backward terms strictly after e, in place
    R acc = R(0);
#pragma unroll
    for (int e = E - 1; e >= 0; --e) {
      const R t = L2[e];
      L2[e] = acc;
      acc += t;
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
    for (int e = 0; e < E; ++e) {
      pf += L1[e];           // forward terms up to e
      if ((omask >> e) & 1u) {
        const R sf = fma(cF1, pf, cF0), sb = fma(cB1, L2[e], cB0);
        const R a1 = (sf > R(0)) ? LF + D[e] : T::kNegBig;
        const R a2 = (sb > R(0)) ? LB - PB[e] : T::kNegBig;
        const R M = fmax(a1, a2);
        emit_o<R, kFlags>(a, sm, ++oi, M + T::lg2(fma(sf, T::ex2(a1 - M), sb * T::ex2(a2 - M))), ob,
                          o_start, o_scale, err);
      }
    }
  } else {
    // levels spread over more than 60 bits: running-max log-sums
    R lam[E];
    R fm[E], fs[E];
    R m = ef.m, sv = ef.s;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (mt[e] > R(0)) ls_add_fast(m, sv, L1[e], mt[e]);
      fm[e] = m;
      fs[e] = sv;
    }
    m = ebm;
    sv = eb.s;
#pragma unroll
    for (int e = E - 1; e >= 0; --e) {
      LS<R> s2 = ls_add(fm[e] + D[e], fs[e], m - PB[e], sv);
      lam[e] = s2.m + T::lg2(s2.s);
      if (mt[e] > R(0)) ls_add_fast(m, sv, L2[e], mt[e]);
    }
#pragma unroll
    for (int e = 0; e < E; ++e)
      if ((omask >> e) & 1u) emit_o<R, kFlags>(a, sm, ++oi, lam[e], ob, o_start, o_scale, err);
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
    a.part[unit] = tot;
  }
  if constexpr ((kFlags & F_OUT_POT) != 0) {
    if constexpr (kUnit) {
      for (int i = tid; i < n_o; i += kThreads) a.pO_out[o_start + i] = sm.pot[1 + i];
    } else if constexpr (kStride1) {
      for (int i = tid; i < n_o; i += kThreads) a.pO_out[ob + o_start + i] = sm.pot[1 + i];
    } else {
      for (int i = tid; i < n_o; i += kThreads) a.pO_out[ob + (int64_t)(o_start + i) * a.o_es] = sm.pot[1 + i];
    }
  }
  if constexpr ((kFlags & F_QOUT) != 0) {
    const int64_t qb = (int64_t)line * a.q_ls;
    for (int i = tid; i < n_o; i += kThreads) a.q_out[qb + (int64_t)(o_start + i) * a.q_es] = T::neg(sm.pot[1 + i]);
  }
  if (kFlags & F_NEXT) {
    // next application: O' = current W (frames = current W potentials),
    // W' = current O (new potentials, same masses); same gaps (reloaded: they
    // are not kept in registers through the outputs)
    load_gaps<R, E>(a.gap, gseg, g);
    seg_terms<R, false, E>(wmask, omask, g, sm.pot + wofs, w_before, sm.pot, sm.mass, o_before + 1, R(0), D,
                 PB, L1, L2, mt);
    (void)seg_maps<R, E>(D, PB, L1, L2, mt, mapF, mapB, MF, MB);
    put_map(sm.tf, tid, mapF);
    put_map(sm.tb, tid, mapB);
    __syncthreads();
    if (tid < 64) rake_reduce<R>(sm, a.agg_out + 6 * (int64_t)unit);
  }
  return true;
}

#ifndef FINOM_MINB
#define FINOM_MINB 4
#endif
// Persistent CTAs: as many as fit on the device; CTA b handles the units
// b, b + G, b + 2G, ... (G = grid size; a counter shared by all CTAs costs
// more in contention than it gains in balance).  The last CTA to finish
// (ticket ctrl[0]) scans the new tile maps into carries, reduces the error
// and updates the loop control.
template <class R, int kFlags, int E = kElems>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? FINOM_MINB : 1) k_apply(ApplyArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem<R>& sm = *reinterpret_cast<TileSmem<R>*>(smem_raw);
  const int tid = threadIdx.x;
  if constexpr ((kFlags & F_BATCH) != 0) {
    // batches: the units are the tiles of the still active instances
    griddep_wait();
    if ((kFlags & F_CHECK_DONE) && *(volatile int32_t*)(a.ctrl + 1)) return;
    griddep_launch_dependents();
    const int units = *(volatile const int32_t*)a.acount;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
      apply_unit<R, kFlags, E>(a, sm, a.alist[u], false);
      __syncthreads();
    }
    return;
  }
  const int units = a.lines * a.C;
  for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
    if (!apply_unit<R, kFlags, E>(a, sm, unit, unit == (int)blockIdx.x)) return;   // the loop is done
    __syncthreads();
  }
  griddep_wait();   // (a no-op after the first unit's wait)
  if (last_cta<R>(a.ctrl, (int)gridDim.x, sm)) finish_launch<R, kFlags>(a, sm, units);
}

}  // namespace finom
