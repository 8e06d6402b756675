// Batches of independent 1D instances in one launch per half step.
//
// Thousands of Sinkhorn solves of uneven sizes (each its own mesh pair, eps
// and masses) run as one sequence of launches of the half-step kernel
// (half.cuh, H_BATCH): the instances' merged sequences are packed one after
// another, each starting on a tile boundary, so that a tile belongs to one
// instance and every kernel unit (a tile of the active list) finds its
// instance in a table.  Every point carries its levels beta+- = b +- Z with
// Z = z / (eps_b ln 2) in its own instance's eps.  After each half step,
// k_batch_end gives every instance a warp that scans its tile aggregates into
// the carries of the next application, sums its marginal error, counts its
// iterations and retires it when it has converged (its tiles leave the
// active list).  The loop is captured in a CUDA graph and runs until the
// last instance has retired.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "finom_internal.h"
#include "half.cuh"

namespace finom {

template <class R>
finom_status half_launch(const HalfArgs<R>&, int, int, cudaStream_t);
template <class R>
void log_mass(const double*, int64_t, void*, cudaStream_t);

namespace {

constexpr double kLn2 = 0.69314718055994530942;

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// instance of element i: the largest b with off[b] <= i
__device__ __forceinline__ int find_inst(const int64_t* off, int B, int64_t i) {
  int lo = 0, hi = B;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// entries of sorted a[0..n) that are <= v (strict: < v)
__device__ __forceinline__ int64_t bcount(const double* a, int64_t n, double v, bool strict) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (strict ? (a[mid] < v) : (a[mid] <= v)) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void k_bcheck(const double* a, const int64_t* off, int B, int64_t n, int* bad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = find_inst(off, B, i);
  const double v = a[i];
  bool ok = isfinite(v);
  if (i + 1 < off[b + 1]) ok = ok && v <= a[i + 1];
  if (!ok) atomicOr(bad, 1);
}

// merged position of each point inside its instance (ties: y before x), and
// the scatter of coordinates and types into the packed merged arrays
__global__ void k_bpos(const double* a, int64_t n, const int64_t* offa, const double* o, const int64_t* offo,
                       const int32_t* itile, int B, int64_t tile, int strict, int64_t* pos, double* z,
                       uint8_t* type, uint8_t t) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = find_inst(offa, B, i);
  const double v = a[i];
  const int64_t loc = (i - offa[b]) + bcount(o + offo[b], offo[b + 1] - offo[b], v, strict != 0);
  pos[i] = loc;
  const int64_t k = (int64_t)itile[b] * tile + loc;
  z[k] = v;
  type[k] = t;
}

// gaps in bits (each instance's eps) and packed type bits; one thread per
// packed position (the packed length is a whole number of tiles)
__global__ void k_bgaps(const double* z, const uint8_t* type, const int32_t* tinst, const int32_t* itile,
                        const int64_t* offx, const int64_t* offy, const double* ieps, int64_t tile,
                        int64_t total, double* gap64, uint32_t* bits) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool live = k < total;
  int ty = 0;
  double gv = 0.0;
  if (live) {
    const int b = tinst[k / tile];
    const int64_t loc = k - (int64_t)itile[b] * tile;
    const int64_t Lb = (offx[b + 1] - offx[b]) + (offy[b + 1] - offy[b]);
    if (loc < Lb) {
      ty = type[k];
      if (loc > 0) gv = (z[k] - z[k - 1]) / (ieps[b] * kLn2);
    }
  }
  const unsigned w = __ballot_sync(0xffffffffu, ty != 0);
  if (!live) return;
  if ((threadIdx.x & 31) == 0) bits[k >> 5] = w;
  gap64[k] = gv;
}

// tile_x0 of every instance: C_b + 1 entries from itile[b] + b, the number of
// the instance's x points before each of its tile boundaries (tiles of `tile`
// points; itile holds the instances' first tiles in that tiling)
__global__ void k_btiles(const int64_t* posx, const int64_t* offx, const int32_t* itile, int B, int64_t tile,
                         int64_t n, int32_t* tx) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  int lo = 0, hi = B;   // instance: the largest b with itile[b] + b <= e
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if ((int64_t)itile[mid] + mid <= e) lo = mid; else hi = mid;
  }
  const int b = lo;
  const int64_t t = e - ((int64_t)itile[b] + b);
  const int64_t bound = t * tile;
  const int64_t* p = posx + offx[b];
  int64_t a = 0, c = offx[b + 1] - offx[b];
  while (a < c) {
    const int64_t mid = (a + c) >> 1;
    if (p[mid] < bound) a = mid + 1; else c = mid;
  }
  tx[e] = (int32_t)a;
}

// per-instance mass normalisation (one CTA per instance): m = u / sum(u) in the
// plan precision and in float64; a non-finite, negative or all-zero instance
// sets *bad
template <class Mass>
__global__ void k_bmass(const double* u, const int64_t* off, Mass* m, double* m64, int* bad) {
  __shared__ double sh[256];
  const int b = blockIdx.x;
  const int64_t i0 = off[b], i1 = off[b + 1];
  double s = 0.0;
  bool ok = true;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const double v = u[i];
    ok = ok && isfinite(v) && v >= 0.0;
    s += v;
  }
  if (!ok) atomicOr(bad, 1);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double tot = sh[0];
  if (threadIdx.x == 0 && !(tot > 0.0 && isfinite(tot))) atomicOr(bad, 1);
  if (!(tot > 0.0)) return;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const double v = u[i] / tot;
    m64[i] = v;
    m[i] = (Mass)v;
  }
}

__device__ __forceinline__ void bput(float4* p, double bp, double bm) {
  const float ph = (float)bp, mh = (float)bm;
  *p = make_float4(ph, (float)(bp - (double)ph), mh, (float)(bm - (double)mh));
}
__device__ __forceinline__ void bput(double2* p, double bp, double bm) { *p = make_double2(bp, bm); }
__device__ __forceinline__ double blevel(float4 v) { return 0.5 * (((double)v.x + (double)v.y) + ((double)v.z + (double)v.w)); }
__device__ __forceinline__ double blevel(double2 v) { return 0.5 * (v.x + v.y); }

// start levels of every point: b = log2(1 / n_b) (phi = 1/N, psi = 1/M of
// its instance, Algorithm 1), Z = z / (eps_b ln 2)
template <class Beta>
__global__ void k_bbeta_start(const double* z, const int64_t* off, int B, const double* ieps, int64_t n,
                              Beta* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = find_inst(off, B, i);
  const double lb = -log2((double)(off[b + 1] - off[b]));
  const double Z = z[i] / (ieps[b] * kLn2);
  bput(out + i, lb + Z, lb - Z);
}

// potentials of the state each instance stopped in (the buffer of its
// iteration count, shifted by its resumes): f = eps ln2 b (-inf where m = 0)
// and the smooth potential P = b - log2 m (0 where m = 0) into p64
template <class Beta>
__global__ void k_bexport(const Beta* pa, const Beta* pb, const double* m64, const int64_t* off, int B,
                          const int32_t* ictl, const double* ieps, int64_t n, double* f, double* p64) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = find_inst(off, B, i);
  const int32_t it = ictl[b] ? ictl[2 * B + b] : ictl[B + b];
  const int32_t q = (it + ictl[4 * B + b]) & 1;   // the buffer of iteration it's state
  if (it == 0) {
    // stopped at the first loop head: the start phi = 1/n (Algorithm 1)
    p64[i] = 0.0;
    f[i] = ieps[b] * log(1.0 / (double)(off[b + 1] - off[b]));
    return;
  }
  const double lv = blevel((q ? pb : pa)[i]);
  const double w = m64[i];
  p64[i] = (w > 0.0) ? lv - log2(w) : 0.0;
  f[i] = (w > 0.0) ? ieps[b] * kLn2 * lv : -INFINITY;
}

// 1/n of each point's instance (the start weights)
__global__ void k_buniform(const int64_t* off, int B, int64_t n, double* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = find_inst(off, B, i);
  out[i] = 1.0 / (double)(off[b + 1] - off[b]);
}

// dst[i] = src[i] for the points of the instances flagged in swap
template <class T>
__global__ void k_bswap(T* dst, const T* src, const int64_t* off, int B, const int32_t* swap, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (swap[find_inst(off, B, i)]) dst[i] = src[i];
}

// per instance sum over its points of m f (m > 0), one CTA per instance
__global__ void k_bdot(const double* m, const double* f, const int64_t* off, double* out) {
  __shared__ double sh[256];
  const int b = blockIdx.x;
  double s = 0.0;
  for (int64_t i = off[b] + threadIdx.x; i < off[b + 1]; i += blockDim.x)
    if (m[i] > 0.0) s += m[i] * f[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[b] += sh[0];
}

template <class R>
struct BatchEndArgs {
  const int32_t* itile;
  int B;
  const R* agg;       // 2 kSt per tile: tile aggregates of the next application (forward | backward)
  R* carry;           // 2 kSt per tile
  const double* part; // per tile: error partials
  int32_t* ictl;      // 6 x B: done | completed iterations | iterations at exit | converged | parity flip |
                      //        iteration budget (0: maxit)
  double* ierr;       // per instance: error of its last check
  const double* itol;
  int64_t maxit;
  int32_t* ctrl;      // [1] every instance retired, [2] active instances, [6] an instance retired
                      //     since the last compaction
  int maps, err, iter_end;
};

// retire instance b (lane 0): the last active instance ends the loop
__device__ __forceinline__ void retire(int32_t* ctrl) {
  ctrl[6] = 1;
  if (atomicSub(ctrl + 2, 1) == 1) ctrl[1] = 1;
}

// carries of one direction of one instance (a warp): the log-sum of the
// aggregates of the tiles before (dir 0) or after (dir 1) each tile, 32
// tiles per step of a running state
template <class R, int dir>
__device__ __forceinline__ void bend_carries(const BatchEndArgs<R>& a, int t0, int nt, int lane) {
  using H = HT<R>;
  constexpr int kS = H::kSt;
  St<R> run = st_empty<R>();
  for (int c = 0; c < nt; c += 32) {
    const int t = dir == 0 ? c + lane : nt - 1 - c - lane;
    const bool in = dir == 0 ? t < nt : t >= 0;
    St<R> inc = st_empty<R>();
    if (in) H::get(a.agg + 2 * kS * (int64_t)(t0 + t) + dir * kS, inc.M, inc.s);
#pragma unroll 1
    for (int o = 1; o < 32; o <<= 1) {
      const St<R> u = st_shfl_up(inc, o);
      if (lane >= o) inc = st_comb(u, inc);
    }
    St<R> ex = st_shfl_up(inc, 1);
    if (lane == 0) ex = st_empty<R>();
    const St<R> st = st_comb(run, ex);
    if (in) H::put(a.carry + 2 * kS * (int64_t)(t0 + t) + dir * kS, st.M, st.s);
    run = st_comb(run, st_shfl_idx(inc, 31));
  }
}

// After a half step: one warp per instance.  Its tile aggregates become
// carries (forward and backward), its error partials its loop-head error
// (Algorithm 1 check), and its iteration count and retirement are updated.
template <class R>
__global__ void k_batch_end(BatchEndArgs<R> a) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= a.B) return;
  int32_t* done = a.ictl + b;
  if (*done) return;
  const int t0 = a.itile[b], nt = a.itile[b + 1] - t0;
  if (a.maps) {
    bend_carries<R, 0>(a, t0, nt, lane);
    bend_carries<R, 1>(a, t0, nt, lane);
  }
  if (a.err) {
    double e = 0.0;
    for (int t = lane; t < nt; t += 32) e += a.part[t0 + t];
    e = warp_sum(e);
    if (lane == 0) {
      a.ierr[b] = e;
      if (e <= a.itol[b]) {
        *done = 1;
        a.ictl[2 * a.B + b] = a.ictl[a.B + b];
        a.ictl[3 * a.B + b] = 1;
        retire(a.ctrl);
      }
    }
  }
  if (a.iter_end && lane == 0) {
    int32_t* it = a.ictl + a.B + b;
    *it += 1;
    const int32_t cap = a.ictl[5 * a.B + b];
    if ((int64_t)*it >= a.maxit || (cap > 0 && *it >= cap)) {
      *done = 1;
      a.ictl[2 * a.B + b] = *it;
      retire(a.ctrl);
    }
  }
}

// The tiles of the active instances, in instance order, and their number
// (one CTA of 1024 threads: each takes a run of instances, a block scan
// places the runs).  Only when an instance retired since the last
// compaction (*dirty); most half steps retire none and return at once.
__global__ void __launch_bounds__(1024) k_batch_compact(const int32_t* itile, const int32_t* idone, int B,
                                                        int32_t* alist, int32_t* acount, int32_t* dirty) {
  __shared__ int32_t sh[1024];
  const int tid = threadIdx.x;
  if (*(volatile int32_t*)dirty == 0) return;
  const int per = (B + 1023) / 1024;
  const int b0 = min(B, tid * per), b1 = min(B, b0 + per);
  int32_t n = 0;
  for (int b = b0; b < b1; ++b)
    if (!idone[b]) n += itile[b + 1] - itile[b];
  sh[tid] = n;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {   // inclusive scan (Hillis-Steele)
    const int32_t v = tid >= o ? sh[tid - o] : 0;
    __syncthreads();
    sh[tid] += v;
    __syncthreads();
  }
  int32_t at = sh[tid] - n;
  for (int b = b0; b < b1; ++b)
    if (!idone[b])
      for (int32_t t = itile[b]; t < itile[b + 1]; ++t) alist[at++] = t;
  if (tid == 1023) {
    *acount = sh[1023];
    *dirty = 0;   // every thread read the flag before the first barrier
  }
}

template <class R>
finom_status ensure_state_batch(finom_plan_s* p) {
  SolveState& st = p->st;
  if (st.ready) return FINOM_OK;
  const int64_t N = p->N, M = p->M, T = p->C, B = p->B;
  const size_t bs = sizeof(typename HT<R>::Beta), ls = sizeof(typename HT<R>::Lv);
  const size_t per_tile = 2 * HT<R>::kSt;
  for (int q = 0; q < 2; ++q) {
    FINOM_CUDA(cudaMalloc(&st.px[q], bs * N));
    FINOM_CUDA(cudaMalloc(&st.py[q], bs * M));
  }
  FINOM_CUDA(cudaMalloc(&st.qom, ls * N));   // log2 masses of x
  FINOM_CUDA(cudaMalloc(&st.qwm, ls * M));   // log2 masses of y
  FINOM_CUDA(cudaMalloc(&st.mu64, sizeof(double) * N));
  FINOM_CUDA(cudaMalloc(&st.nu64, sizeof(double) * M));
  FINOM_CUDA(cudaMalloc(&st.tx, sizeof(double) * std::max<int64_t>(N, 512)));
  FINOM_CUDA(cudaMalloc(&st.ty, sizeof(double) * std::max<int64_t>(M, 512)));
  FINOM_CUDA(cudaMalloc(&st.aggs, sizeof(R) * per_tile * T));
  FINOM_CUDA(cudaMalloc(&st.carries, sizeof(R) * per_tile * T));
  FINOM_CUDA(cudaMalloc(&st.part, sizeof(double) * T));
  FINOM_CUDA(cudaMalloc(&st.scal, sizeof(double) * std::max<int64_t>(520, 2 * B)));
  FINOM_CUDA(cudaMalloc(&st.ctrl, sizeof(int32_t) * 8));
  FINOM_CUDA(cudaMalloc(&st.bad, sizeof(int)));
  FINOM_CUDA(cudaMalloc(&st.ictl, sizeof(int32_t) * 6 * B));
  FINOM_CUDA(cudaMalloc(&st.ierr, sizeof(double) * B));
  FINOM_CUDA(cudaMalloc(&st.itol, sizeof(double) * B));
  FINOM_CUDA(cudaMalloc(&st.alist, sizeof(int32_t) * T));
  FINOM_CUDA(cudaMemset(st.ctrl, 0, sizeof(int32_t) * 8));
  FINOM_CUDA(cudaMemset(st.part, 0, sizeof(double) * T));
  FINOM_CUDA(cudaStreamCreateWithFlags(&st.stream, cudaStreamNonBlocking));
  st.ready = true;
  return FINOM_OK;
}

// the half step of parity q (psi: o_is_x = false, levels py[q] -> py[1-q]
// against phi px[q]; phi: px[q] -> px[1-q] against psi py[1-q]), or with
// mode the aggregate / check launch of that application
template <class R>
HalfArgs<R> batch_args(finom_plan_s* p, bool o_is_x, int q) {
  using Beta = typename HT<R>::Beta;
  using Lv = typename HT<R>::Lv;
  SolveState& st = p->st;
  HalfArgs<R> a{};
  a.tbits = p->tbits;
  a.tile_x0 = p->tile_x0;
  a.L = p->L;
  a.C = (int)p->C;   // grid sizing: all tiles of all instances
  a.o_is_x = o_is_x ? 1 : 0;
  a.tinst = p->tinst;
  a.itile = p->itile;
  a.ioffx = p->ioffx;
  a.ioffy = p->ioffy;
  a.alist = st.alist;
  a.acount = st.ctrl + 3;
  a.agg_out = (R*)st.aggs;
  a.carry_in = (const R*)st.carries;
  a.part = st.part;
  a.scal = st.scal;
  a.ctrl = st.ctrl;
  if (!o_is_x) {   // psi <- v / (K^T phi)
    a.bO = (const Beta*)st.py[q];
    a.bO_out = (Beta*)st.py[1 - q];
    a.bW = (const Beta*)st.px[q];
    a.lmO = (const Lv*)st.qwm;
    a.mO = st.nu64;
  } else {         // phi <- u / (K psi)
    a.bO = (const Beta*)st.px[q];
    a.bO_out = (Beta*)st.px[1 - q];
    a.bW = (const Beta*)st.py[1 - q];
    a.lmO = (const Lv*)st.qom;
  }
  return a;
}

template <class R>
finom_status launch_half(finom_plan_s* p, bool o_is_x, int q, int mode, cudaStream_t s) {
  return half_launch<R>(batch_args<R>(p, o_is_x, q), mode, p->elems, s);
}

template <class R>
finom_status launch_end(finom_plan_s* p, int maps, int err, int iter_end, cudaStream_t s) {
  SolveState& st = p->st;
  BatchEndArgs<R> e{};
  e.itile = p->itile;
  e.B = (int)p->B;
  e.agg = (const R*)st.aggs;
  e.carry = (R*)st.carries;
  e.part = st.part;
  e.ictl = st.ictl;
  e.ierr = st.ierr;
  e.itol = st.itol;
  e.maxit = st.maxit;
  e.ctrl = st.ctrl;
  e.maps = maps;
  e.err = err;
  e.iter_end = iter_end;
  k_batch_end<R><<<nblk(p->B, 8), 256, 0, s>>>(e);
  k_batch_compact<<<1, 1024, 0, s>>>(p->itile, st.ictl, (int)p->B, st.alist, st.ctrl + 3, st.ctrl + 6);
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return cuda_fail(ce, "k_batch_end launch");
  return FINOM_OK;
}

template <class R>
finom_status batch_iteration(finom_plan_s* p, int q, cudaStream_t s) {
  finom_status rc = launch_half<R>(p, false, q, kBatchY, s);
  if (rc == FINOM_OK) rc = launch_end<R>(p, 1, 1, 0, s);
  if (rc == FINOM_OK) rc = launch_half<R>(p, true, q, kBatchX, s);
  if (rc == FINOM_OK) rc = launch_end<R>(p, 1, 0, 1, s);
  return rc;
}

template <class R>
finom_status build_body_batch(finom_plan_s* p) {
  SolveState& st = p->st;
  if (st.body) {
    cudaGraphExecDestroy(st.body);
    st.body = nullptr;
  }
  cudaGraph_t g = nullptr;
  FINOM_CUDA(cudaStreamBeginCapture(st.stream, cudaStreamCaptureModeThreadLocal));
  finom_status rc = batch_iteration<R>(p, 1, st.stream);
  if (rc == FINOM_OK) rc = batch_iteration<R>(p, 0, st.stream);
  cudaError_t e = cudaStreamEndCapture(st.stream, &g);
  if (rc != FINOM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&st.body, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return FINOM_OK;
}

// Launch graph bodies (two iterations each) until every instance retired;
// the first body starts at parity 1 (iteration 0 was launched before).
bool stopped(const finom_plan_s* p) { return p->stop && p->stop->load(std::memory_order_relaxed) != 0; }

template <class R>
finom_status run_loop(finom_plan_s* p, int64_t maxit, cudaStream_t s) {
  SolveState& st = p->st;
  int64_t launched = 1, bodies = 1;
  for (;;) {
    int32_t h[8];
    FINOM_CUDA(cudaMemcpyAsync(h, st.ctrl, sizeof(h), cudaMemcpyDeviceToHost, s));
    FINOM_CUDA(cudaStreamSynchronize(s));
    if (h[1] || launched > maxit + 2 || stopped(p)) break;
    for (int64_t k = 0; k < bodies; ++k) FINOM_CUDA(cudaGraphLaunch(st.body, s));
    launched += 2 * bodies;
    bodies = std::min<int64_t>(bodies * 2, 64);
  }
  return FINOM_OK;
}

// Potentials of each instance's stop state into f, g; per instance the
// float64 W1 and marginal error (cost kernel on a view of the instance), the
// dual and the iteration count into res; err64 (optional) the float64 errors.
template <class R>
finom_status evaluate(finom_plan_s* p, double tol, int64_t maxit, double* f, double* g, finom_result* res,
                      cudaStream_t s, double* err64_out, const std::vector<char>* only = nullptr) {
  using Beta = typename HT<R>::Beta;
  SolveState& st = p->st;
  const int64_t B = p->B, N = p->N, M = p->M;
  std::vector<int32_t> ictl(4 * B);
  std::vector<double> ierr(B);
  FINOM_CUDA(cudaMemcpyAsync(ictl.data(), st.ictl, sizeof(int32_t) * 4 * B, cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaMemcpyAsync(ierr.data(), st.ierr, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
  k_bexport<Beta><<<nblk(N, 256), 256, 0, s>>>((const Beta*)st.px[0], (const Beta*)st.px[1], st.mu64, p->ioffx,
                                                 (int)B, st.ictl, p->ieps, N, f, st.tx);
  k_bexport<Beta><<<nblk(M, 256), 256, 0, s>>>((const Beta*)st.py[0], (const Beta*)st.py[1], st.nu64, p->ioffy,
                                                 (int)B, st.ictl, p->ieps, M, g, st.ty);
  double* dual = st.scal;   // 2 x B: sum u f | sum v g per instance
  FINOM_CUDA(cudaMemsetAsync(dual, 0, sizeof(double) * 2 * B, s));
  k_bdot<<<(unsigned)B, 256, 0, s>>>(st.mu64, f, p->ioffx, dual);
  k_bdot<<<(unsigned)B, 256, 0, s>>>(st.nu64, g, p->ioffy, dual + B);
  FINOM_CUDA(cudaGetLastError());
  std::vector<double> hd(2 * B);
  FINOM_CUDA(cudaMemcpyAsync(hd.data(), dual, sizeof(double) * 2 * B, cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  auto stop_iter = [&](int64_t b) { return ictl[b] ? ictl[2 * B + b] : ictl[B + b]; };
  // instances that stopped at their first loop head keep the start weights
  bool any0 = false;
  for (int64_t b = 0; b < B; ++b) any0 = any0 || stop_iter(b) == 0;
  double* uni0 = nullptr;
  if (any0) {
    FINOM_CUDA(cudaMallocAsync(&uni0, sizeof(double) * (N + M), s));
    k_buniform<<<nblk(N, 256), 256, 0, s>>>(p->ioffx, (int)B, N, uni0);
    k_buniform<<<nblk(M, 256), 256, 0, s>>>(p->ioffy, (int)B, M, uni0 + N);
  }
  finom_status rc = FINOM_OK;
  for (int64_t b = 0; b < B && rc == FINOM_OK; ++b) {
    if (only && !(*only)[b]) continue;   // unchanged since the last evaluation
    // a view of instance b for the float64 cost kernel (it owns nothing)
    finom_plan_s view;
    const int64_t t0 = p->hitile[b], nt = p->hitile[b + 1] - t0;
    view.N = p->hoffx[b + 1] - p->hoffx[b];
    view.M = p->hoffy[b + 1] - p->hoffy[b];
    view.L = view.N + view.M;
    (void)nt;
    // the float64 cost kernel works in 2048-point tiles from the instance's
    // start: its own tile table, the packed arrays padded at the end
    view.C = p->hitilec[b + 1] - p->hitilec[b];
    view.eps = p->heps[b];
    view.tbits = p->tbits + t0 * (p->btile / 32);
    view.gap64 = p->gap64 + t0 * p->btile;
    view.tile_x0 = p->tile_x0c + p->hitilec[b] + b;
    const int32_t its = stop_iter(b);
    const bool start = its == 0;
    const double* mx = start ? uni0 + p->hoffx[b] : st.mu64 + p->hoffx[b];
    const double* my = start ? uni0 + N + p->hoffy[b] : st.nu64 + p->hoffy[b];
    double err64 = 0.0, w1 = 0.0;
    rc = cost64(&view, st.tx + p->hoffx[b], st.ty + p->hoffy[b], mx, my, &err64, &w1, s);
    if (start) err64 = ierr[b];   // the loop's own check of the start
    finom_result& r = res[b];
    r.w1 = w1;
    r.marginal_err = err64;
    r.marginal_err_loop = ierr[b];
    r.dual = hd[b] + hd[B + b];
    r.iters = maxit == 0 ? 0 : its;
    r.converged = (err64 <= tol || (ictl[3 * B + b] && sizeof(R) == sizeof(double))) ? 1 : 0;
    r.status = FINOM_OK;
    if (err64_out) err64_out[b] = err64;
  }
  if (uni0) cudaFreeAsync(uni0, s);
  return rc;
}

// Start of a batch solve on stream s: masses, start state, iteration 0
// (maxit = 0: only the first loop-head check).
template <class R>
finom_status begin_batch(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                         cudaStream_t s) {
  using Beta = typename HT<R>::Beta;
  finom_status rc = ensure_state_batch<R>(p);
  if (rc != FINOM_OK) return rc;
  SolveState& st = p->st;
  const int64_t B = p->B, N = p->N, M = p->M;
  // masses, per instance, and their log2
  FINOM_CUDA(cudaMemsetAsync(st.bad, 0, sizeof(int), s));
  k_bmass<double><<<(unsigned)B, 256, 0, s>>>(u, p->ioffx, st.mu64, st.mu64, st.bad);
  k_bmass<double><<<(unsigned)B, 256, 0, s>>>(v, p->ioffy, st.nu64, st.nu64, st.bad);
  int hbad = 0;
  FINOM_CUDA(cudaMemcpyAsync(&hbad, st.bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  if (hbad) {
    set_error("finom_solve_batch: every instance's masses must be finite, >= 0, with a positive sum");
    return FINOM_EINVAL;
  }
  log_mass<R>(st.mu64, N, st.qom, s);
  log_mass<R>(st.nu64, M, st.qwm, s);
  // start: phi = 1/N_b, psi = 1/M_b
  k_bbeta_start<Beta><<<nblk(N, 256), 256, 0, s>>>(p->x, p->ioffx, (int)B, p->ieps, N, (Beta*)st.px[0]);
  k_bbeta_start<Beta><<<nblk(M, 256), 256, 0, s>>>(p->y, p->ioffy, (int)B, p->ieps, M, (Beta*)st.py[0]);
  fill_d(st.itol, B, tol, s);
  FINOM_CUDA(cudaMemsetAsync(st.ictl, 0, sizeof(int32_t) * 6 * B, s));
  FINOM_CUDA(cudaMemsetAsync(st.ierr, 0, sizeof(double) * B, s));
  int32_t c0[8] = {0, 0, (int32_t)B, 0, 0, 0, 1, 0};
  FINOM_CUDA(cudaMemcpyAsync(st.ctrl, c0, sizeof(c0), cudaMemcpyHostToDevice, s));
  st.tol = tol;
  st.maxit = maxit;
  k_batch_compact<<<1, 1024, 0, s>>>(p->itile, st.ictl, (int)B, st.alist, st.ctrl + 3, st.ctrl + 6);
  // iteration 0: aggregates of the first K^T phi, then its half step with
  // the check at the first loop head, then the phi half step
  rc = launch_half<R>(p, false, 0, kBatchAgg, s);
  if (rc == FINOM_OK) rc = launch_end<R>(p, 1, 0, 0, s);
  if (rc != FINOM_OK) return rc;
  st.active = true;
  st.launched = 0;
  if (maxit == 0) {
    rc = launch_half<R>(p, false, 0, kBatchCheck, s);
    if (rc == FINOM_OK) rc = launch_end<R>(p, 0, 1, 0, s);
    return rc;
  }
  rc = launch_half<R>(p, false, 0, kBatchY, s);
  if (rc == FINOM_OK) rc = launch_end<R>(p, 1, 1, 0, s);
  if (rc == FINOM_OK) rc = launch_half<R>(p, true, 0, kBatchX, s);
  if (rc == FINOM_OK) rc = launch_end<R>(p, 1, 0, 1, s);
  st.launched = 1;
  return rc;
}

template <class R>
finom_status solve_batch_impl(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                              double* f, double* g, finom_result* res, cudaStream_t us) {
  using Beta = typename HT<R>::Beta;
  FINOM_CUDA(cudaStreamSynchronize(us));
  finom_status rc = ensure_state_batch<R>(p);
  if (rc != FINOM_OK) return rc;
  SolveState& st = p->st;
  cudaStream_t s = st.stream;
  const int64_t B = p->B, N = p->N, M = p->M;
  rc = begin_batch<R>(p, u, v, tol, maxit, s);
  if (rc != FINOM_OK) return rc;
  if (maxit == 0) {
    rc = evaluate<R>(p, tol, maxit, f, g, res, s, nullptr);
    st.active = false;
    return rc;
  }
  rc = build_body_batch<R>(p);
  if (rc != FINOM_OK) return rc;
  std::vector<double> err64(B), prev64(B, INFINITY);
  std::vector<int32_t> ictl(6 * B);
  std::vector<char> changed(B, 1), final_(B, 0);
  for (int attempt = 0;; ++attempt) {
    rc = run_loop<R>(p, maxit, s);
    if (rc != FINOM_OK) return rc;
    rc = evaluate<R>(p, tol, maxit, f, g, res, s, err64.data(), &changed);
    if (rc != FINOM_OK) return rc;
    if (sizeof(R) == sizeof(double) || attempt >= 6 || stopped(p)) break;
    // float64 verification: an instance whose float32 check passed but whose
    // float64 error is above tol resumes from its stop state (the skipped phi
    // half step of its stop iteration) with a tighter loop tolerance.  Their
    // states are first moved to parity 0, so one sequence of launches serves
    // them all.
    FINOM_CUDA(cudaMemcpyAsync(ictl.data(), st.ictl, sizeof(int32_t) * 6 * B, cudaMemcpyDeviceToHost, s));
    std::vector<double> itol(B), ierr(B);
    FINOM_CUDA(cudaMemcpyAsync(itol.data(), st.itol, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
    FINOM_CUDA(cudaMemcpyAsync(ierr.data(), st.ierr, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
    FINOM_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> swap(B, 0);
    int32_t n_resume = 0;
    for (int64_t b = 0; b < B; ++b) {
      changed[b] = 0;
      const int32_t l = ictl[2 * B + b];
      if (!ictl[3 * B + b] || l == 0 || err64[b] <= tol || final_[b]) continue;
      // a resume that did not lower the float64 error met the float32 floor
      // of this instance
      if (err64[b] >= prev64[b]) {
        final_[b] = 1;
        continue;
      }
      prev64[b] = err64[b];
      const double fr = std::max(0.1, std::min(0.8, 0.8 * tol / err64[b]));
      itol[b] = std::max(ierr[b] * fr, 0.0);
      ictl[b] = 0;              // active again
      ictl[B + b] = l;          // completed iterations at the stop
      ictl[3 * B + b] = 0;
      // its stop state sits in buffer (l + flip) & 1; moved to 0, iteration
      // l + 1 then runs at parity 1, i.e. flip = l & 1 from now on
      swap[b] = (l + ictl[4 * B + b]) & 1;
      ictl[4 * B + b] = l & 1;
      // a resume gets a budget of iterations (a float32 floor above the
      // tightened tolerance would otherwise run it to maxit)
      ictl[5 * B + b] = (int32_t)std::min<int64_t>(maxit, (int64_t)l + std::max<int64_t>(1000, l / 2));
      changed[b] = 1;
      ++n_resume;
    }
    if (n_resume == 0) break;
    int32_t* dswap = nullptr;
    FINOM_CUDA(cudaMallocAsync(&dswap, sizeof(int32_t) * B, s));
    FINOM_CUDA(cudaMemcpyAsync(dswap, swap.data(), sizeof(int32_t) * B, cudaMemcpyHostToDevice, s));
    FINOM_CUDA(cudaMemcpyAsync(st.ictl, ictl.data(), sizeof(int32_t) * 6 * B, cudaMemcpyHostToDevice, s));
    FINOM_CUDA(cudaMemcpyAsync(st.itol, itol.data(), sizeof(double) * B, cudaMemcpyHostToDevice, s));
    k_bswap<Beta><<<nblk(N, 256), 256, 0, s>>>((Beta*)st.px[0], (const Beta*)st.px[1], p->ioffx, (int)B, dswap, N);
    k_bswap<Beta><<<nblk(M, 256), 256, 0, s>>>((Beta*)st.py[1], (const Beta*)st.py[0], p->ioffy, (int)B, dswap, M);
    cudaFreeAsync(dswap, s);
    int32_t c1[8] = {0, 0, n_resume, 0, 0, 0, 1, 0};
    FINOM_CUDA(cudaMemcpyAsync(st.ctrl, c1, sizeof(c1), cudaMemcpyHostToDevice, s));
    k_batch_compact<<<1, 1024, 0, s>>>(p->itile, st.ictl, (int)B, st.alist, st.ctrl + 3, st.ctrl + 6);
    // the phi half step of the stop iterations, at parity 0
    rc = launch_half<R>(p, true, 0, kBatchX, s);
    if (rc == FINOM_OK) rc = launch_end<R>(p, 1, 0, 1, s);
    if (rc != FINOM_OK) return rc;
  }
  st.tol = tol;
  st.active = false;
  if (sizeof(R) == sizeof(double) || stopped(p)) return FINOM_OK;
  // instances whose float32 state cannot reach tol in float64 (a float32
  // floor above tol: coarse gaps in bits) are finished in float64, warm
  // started from their float32 potentials
  for (int64_t b = 0; b < B; ++b) {
    if (err64[b] <= tol || res[b].iters >= maxit) continue;
    const int64_t xo = p->hoffx[b], yo = p->hoffy[b];
    const int64_t nb = p->hoffx[b + 1] - xo, mb = p->hoffy[b + 1] - yo;
    finom_plan_t p64 = nullptr;
    rc = finom_plan(p->x + xo, nb, p->y + yo, mb, p->heps[b], FINOM_F64, s, &p64);
    if (rc != FINOM_OK) return rc;
    finom_result r64;
    rc = finom_solve(p64, st.mu64 + xo, st.nu64 + yo, tol, maxit - res[b].iters, f + xo, g + yo, 1, &r64, s);
    finom_plan_destroy(p64);
    if (rc != FINOM_OK) return rc;
    r64.iters += res[b].iters;
    r64.marginal_err_loop = res[b].marginal_err_loop;
    res[b] = r64;
  }
  return FINOM_OK;
}

}  // namespace

finom_status plan_batch_build(finom_plan_s* p, const double* x, const int64_t* offx, const double* y,
                              const int64_t* offy, int64_t B, const double* eps, cudaStream_t s) {
  p->B = B;
  p->hoffx.assign(offx, offx + B + 1);
  p->hoffy.assign(offy, offy + B + 1);
  p->heps.assign(eps, eps + B);
  const int64_t tile = p->btile;
  p->hitile.assign(B + 1, 0);
  p->hitilec.assign(B + 1, 0);
  std::vector<int32_t> tinst;
  for (int64_t b = 0; b < B; ++b) {
    const int64_t Lb = (offx[b + 1] - offx[b]) + (offy[b + 1] - offy[b]);
    const int64_t Cb = (Lb + tile - 1) / tile;
    p->hitile[b + 1] = (int32_t)(p->hitile[b] + Cb);
    p->hitilec[b + 1] = (int32_t)(p->hitilec[b] + (Lb + kTile - 1) / kTile);
    for (int64_t t = 0; t < Cb; ++t) tinst.push_back((int32_t)b);
  }
  const int64_t T = p->hitile[B], Tc = p->hitilec[B], N = offx[B], M = offy[B];
  p->N = N;
  p->M = M;
  p->C = T;
  p->L = T * tile;
  const int64_t total = T * tile;
  // packed arrays: whole tiles, plus one 2048-point tile of padding so that the
  // cost kernel's 2048-point tiles of the last instance stay inside them
  const int64_t alloc = total + kTile;
  FINOM_CUDA(cudaMalloc(&p->x, sizeof(double) * N));
  FINOM_CUDA(cudaMalloc(&p->y, sizeof(double) * M));
  FINOM_CUDA(cudaMemcpyAsync(p->x, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  FINOM_CUDA(cudaMemcpyAsync(p->y, y, sizeof(double) * M, cudaMemcpyDeviceToDevice, s));
  FINOM_CUDA(cudaMalloc(&p->ioffx, sizeof(int64_t) * (B + 1)));
  FINOM_CUDA(cudaMalloc(&p->ioffy, sizeof(int64_t) * (B + 1)));
  FINOM_CUDA(cudaMalloc(&p->itile, sizeof(int32_t) * (B + 1)));
  FINOM_CUDA(cudaMalloc(&p->tinst, sizeof(int32_t) * T));
  FINOM_CUDA(cudaMalloc(&p->ieps, sizeof(double) * B));
  FINOM_CUDA(cudaMemcpyAsync(p->ioffx, offx, sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice, s));
  FINOM_CUDA(cudaMemcpyAsync(p->ioffy, offy, sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice, s));
  FINOM_CUDA(cudaMemcpyAsync(p->itile, p->hitile.data(), sizeof(int32_t) * (B + 1), cudaMemcpyHostToDevice, s));
  FINOM_CUDA(cudaMemcpyAsync(p->tinst, tinst.data(), sizeof(int32_t) * T, cudaMemcpyHostToDevice, s));
  FINOM_CUDA(cudaMemcpyAsync(p->ieps, eps, sizeof(double) * B, cudaMemcpyHostToDevice, s));

  int* bad = nullptr;
  FINOM_CUDA(cudaMalloc(&bad, sizeof(int)));
  FINOM_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  k_bcheck<<<nblk(N, 256), 256, 0, s>>>(p->x, p->ioffx, (int)B, N, bad);
  k_bcheck<<<nblk(M, 256), 256, 0, s>>>(p->y, p->ioffy, (int)B, M, bad);
  int hbad = 0;
  FINOM_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  cudaFree(bad);
  if (hbad) {
    set_error("finom_plan_batch: every instance's x and y must be finite and sorted non-decreasing");
    return FINOM_EINVAL;
  }
  FINOM_CUDA(cudaMalloc(&p->tbits, sizeof(uint32_t) * (alloc / 32)));
  FINOM_CUDA(cudaMemsetAsync(p->tbits, 0, sizeof(uint32_t) * (alloc / 32), s));
  FINOM_CUDA(cudaMalloc(&p->gap64, sizeof(double) * alloc));
  FINOM_CUDA(cudaMemsetAsync(p->gap64, 0, sizeof(double) * alloc, s));
  FINOM_CUDA(cudaMalloc(&p->tile_x0, sizeof(int32_t) * (T + B)));
  FINOM_CUDA(cudaMalloc(&p->tile_x0c, sizeof(int32_t) * (Tc + B)));
  int32_t* itilec = nullptr;
  FINOM_CUDA(cudaMalloc(&itilec, sizeof(int32_t) * (B + 1)));
  FINOM_CUDA(cudaMemcpyAsync(itilec, p->hitilec.data(), sizeof(int32_t) * (B + 1), cudaMemcpyHostToDevice, s));
  int64_t *posx = nullptr, *posy = nullptr;
  double* z = nullptr;
  uint8_t* type = nullptr;
  FINOM_CUDA(cudaMalloc(&posx, sizeof(int64_t) * N));
  FINOM_CUDA(cudaMalloc(&posy, sizeof(int64_t) * M));
  FINOM_CUDA(cudaMalloc(&z, sizeof(double) * total));
  FINOM_CUDA(cudaMalloc(&type, total));
  FINOM_CUDA(cudaMemsetAsync(type, 0, total, s));
  FINOM_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * total, s));
  k_bpos<<<nblk(N, 256), 256, 0, s>>>(p->x, N, p->ioffx, p->y, p->ioffy, p->itile, (int)B, tile, 0, posx, z,
                                       type, 1);
  k_bpos<<<nblk(M, 256), 256, 0, s>>>(p->y, M, p->ioffy, p->x, p->ioffx, p->itile, (int)B, tile, 1, posy, z,
                                       type, 0);
  k_bgaps<<<nblk(total, 256), 256, 0, s>>>(z, type, p->tinst, p->itile, p->ioffx, p->ioffy, p->ieps, tile, total,
                                            p->gap64, p->tbits);
  k_btiles<<<nblk(T + B, 256), 256, 0, s>>>(posx, p->ioffx, p->itile, (int)B, tile, T + B, p->tile_x0);
  k_btiles<<<nblk(Tc + B, 256), 256, 0, s>>>(posx, p->ioffx, itilec, (int)B, kTile, Tc + B, p->tile_x0c);
  FINOM_CUDA(cudaGetLastError());
  FINOM_CUDA(cudaStreamSynchronize(s));
  cudaFree(itilec);
  cudaFree(posx);
  cudaFree(posy);
  cudaFree(z);
  cudaFree(type);
  return FINOM_OK;
}

void plan_batch_free(finom_plan_s* p) {
  cudaFree(p->tile_x0c);
  p->tile_x0c = nullptr;
  cudaFree(p->ioffx);
  cudaFree(p->ioffy);
  cudaFree(p->itile);
  cudaFree(p->tinst);
  cudaFree(p->ieps);
  p->ioffx = p->ioffy = nullptr;
  p->itile = p->tinst = nullptr;
  p->ieps = nullptr;
}

finom_status solve_batch(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                         double* f, double* g, finom_result* res, cudaStream_t s) {
  return p->prec == FINOM_F32_LOG ? solve_batch_impl<float>(p, u, v, tol, maxit, f, g, res, s)
                                  : solve_batch_impl<double>(p, u, v, tol, maxit, f, g, res, s);
}

finom_status solve_batch_begin(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                               cudaStream_t s) {
  return p->prec == FINOM_F32_LOG ? begin_batch<float>(p, u, v, tol, maxit, s)
                                  : begin_batch<double>(p, u, v, tol, maxit, s);
}

finom_status solve_batch_step(finom_plan_s* p, int64_t iters, cudaStream_t s) {
  SolveState& st = p->st;
  for (int64_t k = 0; k < iters; ++k) {
    const int q = (int)(st.launched & 1);
    finom_status rc = p->prec == FINOM_F32_LOG ? batch_iteration<float>(p, q, s) : batch_iteration<double>(p, q, s);
    if (rc != FINOM_OK) return rc;
    ++st.launched;
  }
  return FINOM_OK;
}

finom_status solve_batch_end(finom_plan_s* p, double* f, double* g, finom_result* res, cudaStream_t s) {
  SolveState& st = p->st;
  finom_status rc = p->prec == FINOM_F32_LOG ? evaluate<float>(p, st.tol, st.maxit, f, g, res, s, nullptr)
                                             : evaluate<double>(p, st.tol, st.maxit, f, g, res, s, nullptr);
  st.active = false;
  return rc;
}

}  // namespace finom
