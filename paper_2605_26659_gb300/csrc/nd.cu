// d-dimensional FINOM on tensor-product grids (Sec. 3, the closing remark on
// higher dimensions: with a separable L1 cost K = K_d (x) ... (x) K_1, and a
// product with K is d batches of 1D products, one axis after the other).
//
// Grids: mu on the nodes x^1 (x) ... (x) x^d, nu on y^1 (x) ... (x) y^d, both
// with n_1 x ... x n_d points stored axis 0 fastest (the paper's vec() for
// d = 2).  Axis plan k merges x^k (the x side) with y^k (the y side).  An
// application of K to a grid of log-weights runs one axis pass per axis of
// the half-step kernel (half.cuh, H_LINES): every line of the grid along
// axis k is one 1D product with axis plan k.  Passes before the last write
// log2 of the partial product (a level pair per grid point) for the next
// pass; the last pass divides (Sinkhorn's eq. iteration in log form) at the
// output grid and, for K^T phi, adds the marginal error of the loop head.
// The float64 check of the marginal error and W1 = <C, Gamma> run the same
// passes in float64; <C_k, Gamma> replaces axis k's pass by its cost-weighted
// form, from the lower and upper block sums of plain and of
// distance-weighted levels (sum (z_o - z_m) w_m = (z_o - z0) sum w_m -
// sum (z_m - z0) w_m on the lower side, the mirror on the upper side).
//
// Layouts.  Every pass reads and writes whole contiguous lines: layout L_k
// stores a grid with axis k fastest, then k+1, ..., d-1, 0, ..., k-1.  nu's
// grid lives in L_0 (the caller's order), mu's in L_{d-1}.  K psi runs axes
// 0, 1, ..., d-1 and turns its partial product from L_k into L_{k+1} between
// passes (a transpose of an n_k x G/n_k matrix); K^T phi runs axes d-1, ...,
// 0 and turns L_k into L_{k-1}.  The last pass of either meets the output
// grid in its own layout, so no grid is ever read or written with a stride.
// mu's grids change layout only at the ABI (masses and warm starts in, the
// potentials out).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>

#include "finom_internal.h"
#include "half.cuh"

namespace finom {

template <class R>
finom_status half_launch(const HalfArgs<R>&, int, int, cudaStream_t);

namespace {

constexpr double kLn2 = 0.69314718055994530942;

template <class R>
using LvT = typename HT<R>::Lv;

inline unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

__device__ __forceinline__ void put_lv(float2* p, double v) {
  const float h = (float)v;
  *p = make_float2(h, (float)(v - (double)h));
}
__device__ __forceinline__ void put_lv(double* p, double v) { *p = v; }
__device__ __forceinline__ double get_lv(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ double get_lv(double v) { return v; }

// positions in bits of n axis nodes (level pairs and float64), and log2 of
// their distance to z0 (float64; -inf at z0)
template <class Lv>
__global__ void k_axis_tables(const double* x, int64_t n, double scale, double z0, Lv* z, double* z64,
                              double* lz) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i] * scale;
  put_lv(z + i, v);
  z64[i] = v;
  const double d = v - z0 * scale;
  lz[i] = d > 0.0 ? log2(d) : -INFINITY;
}

// grid of log-weights: b = f * fscale (f given, -inf: none) or fill
template <class Lv>
__global__ void k_grid_set(Lv* g, int64_t n, const double* f, double fscale, double fill, double none) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double b = fill;
  if (f) b = (f[i] > -INFINITY) ? f[i] * fscale : none;
  put_lv(g + i, b);
}

// log-weights of linear values (b = log2 v, v <= 0: none)
template <class Lv>
__global__ void k_grid_lin(Lv* g, int64_t n, const double* v, double none) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  put_lv(g + i, v[i] > 0.0 ? log2(v[i]) : none);
}

// log2 of normalised masses (none for zero)
template <class Lv>
__global__ void k_grid_lmass(const double* m, int64_t n, Lv* lm, double none) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  put_lv(lm + i, m[i] > 0.0 ? log2(m[i]) : none);
}

// a grid of level pairs in float64 (none -> -inf)
template <class Lv>
__global__ void k_grid_to64(const Lv* g, int64_t n, double none, double* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double b = get_lv(g[i]);
  out[i] = b > 0.5 * none ? b : -INFINITY;
}

// potential f = eps ln 2 * b (-inf without mass)
__global__ void k_f_of(const double* b, const double* m, int64_t n, double eps_ln2, double* f) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  f[i] = (m[i] > 0.0 && b[i] > -INFINITY) ? eps_ln2 * b[i] : -INFINITY;
}

// product outputs from the last pass's log2 sums q: ln (K w) + a / eps, or K w
template <class Lv>
__global__ void k_prod_out(const Lv* q, int64_t n, const double* a, double inv_eps, int lin, double none,
                           double* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double l2 = get_lv(q[i]);
  const bool empty = !(l2 > 0.5 * none);
  if (lin) out[i] = empty ? 0.0 : exp2(l2);
  else out[i] = empty ? -INFINITY : kLn2 * l2 + (a ? a[i] * inv_eps : 0.0);
}

// cost-weighted axis pass from the block sums of plain (fb0) and
// distance-weighted (fb1) levels (log2; lower sums at [0, G), upper at
// [G, 2G)): sum_m |z_o - z_m| w_m K_om as log2 in q
__global__ void k_moment(const double* fb0, const double* fb1, int64_t G, const double* z64, double z0s,
                         int64_t inner, int64_t nk, double* q) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= G) return;
  const int64_t o = (i / inner) % nk;
  const double D = z64[o] - z0s;   // distance of the output node to z0 (bits, >= 0)
  const double lD = D > 0.0 ? log2(D) : -INFINITY;
  // lower: D P0 - P1; upper: Q1 - D Q0
  const double t[4] = {lD + fb0[i], fb1[i], fb1[G + i], lD + fb0[G + i]};
  double M = -INFINITY;
  for (int k = 0; k < 4; ++k) M = fmax(M, t[k]);
  if (!(M > -INFINITY)) {
    q[i] = -INFINITY;
    return;
  }
  const double v = (exp2(t[0] - M) - exp2(t[1] - M)) + (exp2(t[2] - M) - exp2(t[3] - M));
  q[i] = v > 0.0 ? M + log2(v) : -INFINITY;
}

// sums over a grid in float64, one partial per block: mode 0:
// |2^{b + q} - m| (marginal error), mode 1: 2^{b + q} (mass of the plan)
__global__ void k_grid_sum(const double* b, const double* q, const double* m, int64_t n, int mode,
                           double* part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double l = b[i] + q[i];
    const double w = (l > -INFINITY) ? exp2(l) : 0.0;
    acc += mode == 0 ? fabs(w - m[i]) : w;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_parts(const double* part, int n, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s;
  }
}

// dst = the transpose of src: src holds an R x C matrix with its rows index
// fastest (entry (r, c) at r + R c), dst holds it at c + C r.  32 x 32 tiles
// staged in shared memory (coalesced on both sides), grid-stride over tiles.
template <class T>
__global__ void __launch_bounds__(256) k_rot(const T* __restrict__ src, int64_t R, int64_t C, T* __restrict__ dst) {
  __shared__ T t[32][33];
  const int64_t tr = (R + 31) / 32, tiles = tr * ((C + 31) / 32);
  for (int64_t b = blockIdx.x; b < tiles; b += gridDim.x) {
    const int64_t r0 = (b % tr) * 32, c0 = (b / tr) * 32;
#pragma unroll
    for (int k = threadIdx.y; k < 32; k += 8) {
      const int64_t r = r0 + threadIdx.x, c = c0 + k;
      if (r < R && c < C) t[k][threadIdx.x] = src[r + R * c];
    }
    __syncthreads();
#pragma unroll
    for (int k = threadIdx.y; k < 32; k += 8) {
      const int64_t c = c0 + threadIdx.x, r = r0 + k;
      if (r < R && c < C) dst[c + C * r] = t[threadIdx.x][k];
    }
    __syncthreads();
  }
}

int64_t nd_lines(const finom_plan_s* p, int k) { return p->nd_G / p->nd_n[k]; }

// A grid from layout L_k to L_{k+1} (fwd) or L_{k-1} (!fwd), src -> dst.
template <class T>
void nd_rot(const finom_plan_s* p, int k, bool fwd, const T* src, T* dst, cudaStream_t s) {
  const int d = p->dim, G = (int)p->nd_G;
  if (d == 1) {   // one layout only
    cudaMemcpyAsync(dst, src, sizeof(T) * G, cudaMemcpyDeviceToDevice, s);
    return;
  }
  // L_k -> L_{k+1}: axis k (fastest) becomes the slowest; L_k -> L_{k-1}:
  // the slowest axis, k-1, becomes the fastest
  const int64_t R = fwd ? p->nd_n[k] : p->nd_G / p->nd_n[(k + d - 1) % d];
  const int64_t C = p->nd_G / R;
  const int64_t tiles = ((R + 31) / 32) * ((C + 31) / 32);
  k_rot<T><<<(unsigned)std::min<int64_t>(tiles, 4096), dim3(32, 8), 0, s>>>(src, R, C, dst);
}

// largest (lines x tiles) over the axis passes
int64_t nd_units(const finom_plan_s* p) {
  int64_t u = 1;
  for (int k = 0; k < p->dim; ++k) u = std::max(u, nd_lines(p, k) * p->nd_ax[k]->Ce);
  return u;
}

// Solve state: px / py: mu / nu log-weights (level pairs, ping-pong); qom /
// qwm: their log2 masses; q2: two grids of partial products; mu64 / nu64:
// float64 masses; tx, ty: float64 grids; aggs / carries / part per unit.
template <class R>
finom_status ensure_state_nd(finom_plan_s* p) {
  SolveState& st = p->st;
  if (st.ready) return FINOM_OK;
  const int64_t G = p->nd_G, U = nd_units(p);
  const size_t lv = sizeof(LvT<R>);
  for (int q = 0; q < 2; ++q) {
    FINOM_CUDA(cudaMalloc(&st.px[q], lv * G));
    FINOM_CUDA(cudaMalloc(&st.py[q], lv * G));
  }
  FINOM_CUDA(cudaMalloc(&st.qom, lv * G));
  FINOM_CUDA(cudaMalloc(&st.qwm, lv * G));
  FINOM_CUDA(cudaMalloc(&st.q2, lv * 2 * G));
  FINOM_CUDA(cudaMalloc(&st.mu64, sizeof(double) * G));
  FINOM_CUDA(cudaMalloc(&st.nu64, sizeof(double) * G));
  FINOM_CUDA(cudaMalloc(&st.tx, sizeof(double) * std::max<int64_t>(G, 512)));
  FINOM_CUDA(cudaMalloc(&st.ty, sizeof(double) * std::max<int64_t>(G, 512)));
  FINOM_CUDA(cudaMalloc(&st.aggs, sizeof(R) * 2 * HT<R>::kSt * U));
  FINOM_CUDA(cudaMalloc(&st.carries, sizeof(R) * 2 * HT<R>::kSt * U));
  FINOM_CUDA(cudaMalloc(&st.part, sizeof(double) * U));
  FINOM_CUDA(cudaMalloc(&st.scal, sizeof(double) * 520));
  FINOM_CUDA(cudaMalloc(&st.ctrl, sizeof(int32_t) * 8));
  FINOM_CUDA(cudaMalloc(&st.bad, sizeof(int)));
  FINOM_CUDA(cudaMemset(st.ctrl, 0, sizeof(int32_t) * 8));
  FINOM_CUDA(cudaMemset(st.scal, 0, sizeof(double) * 520));
  FINOM_CUDA(cudaStreamCreateWithFlags(&st.stream, cudaStreamNonBlocking));
  st.ready = true;
  return FINOM_OK;
}

// float64 workspace of the checks: grids b_mu, b_nu, two partial products,
// the block sums of two passes (2 grids each), aggregates / carries / parts
double* w64(finom_plan_s* p) {
  if (!p->nd_w64) {
    const int64_t G = p->nd_G, U = nd_units(p);
    if (cudaMalloc(&p->nd_w64, sizeof(double) * (8 * G + 9 * U + 512)) != cudaSuccess) p->nd_w64 = nullptr;
  }
  return p->nd_w64;
}

// One axis pass along axis k.  W: log-weights on the grid (gW; positions of
// the W side's nodes); O: grid frames gO (or frames 0 for QOUT / FB passes).
// Lines of two tiles form their carries inside the pass (each tile from the
// other's W points); lines of more tiles get them from an aggregate launch.
template <class R>
finom_status nd_pass(finom_plan_s* p, int k, int o_is_x, const LvT<R>* gW, int mode, const LvT<R>* gO,
                     LvT<R>* gO_out, const LvT<R>* lmO, LvT<R>* q_out, double* out, const double* zlogW,
                     R* aggs, R* carries, double* part, cudaStream_t s, double tol, int64_t maxit) {
  finom_plan_s* ax = p->nd_ax[k];
  HalfArgs<R> a{};
  a.tbits = ax->tbits;
  a.tile_x0 = ax->tile_x0e;
  a.L = ax->L;
  a.C = (int)ax->Ce;
  a.o_is_x = o_is_x;
  a.lines = (int)nd_lines(p, k);
  a.inner = 1;   // the grid is in layout L_k: lines along axis k are contiguous
  a.nk = p->nd_n[k];
  a.gW = gW;
  a.gO = gO;
  a.gO_out = gO_out;
  a.lmO = lmO;
  a.mO = (lmO && !o_is_x) ? p->st.nu64 : nullptr;   // nu's masses (layout L_0) for the error term
  a.q_out = q_out;
  a.out = out;
  a.grid = p->nd_G;
  const bool f64 = sizeof(R) == sizeof(double);
  a.zW = (const LvT<R>*)(o_is_x ? (f64 ? (void*)p->nd_zy64[k] : p->nd_zy[k]) : (f64 ? (void*)p->nd_zx64[k] : p->nd_zx[k]));
  a.zO = (const LvT<R>*)(o_is_x ? (f64 ? (void*)p->nd_zx64[k] : p->nd_zx[k]) : (f64 ? (void*)p->nd_zy64[k] : p->nd_zy[k]));
  a.zlogW = (const LvT<R>*)zlogW;
  a.agg_out = aggs;
  a.carry_out = carries;
  a.part = part;
  a.scal = p->st.scal;
  a.ctrl = p->st.ctrl;
  a.tol = tol;
  a.maxit = maxit;
  a.carry_in = nullptr;
  a.pair = a.C == 2 ? 1 : 0;   // two tiles per line: carries formed inside the pass
  if (a.C > 2) {
    finom_status rc = half_launch<R>(a, zlogW ? kLineAggZ : kLineAgg, ax->elems, s);
    if (rc != FINOM_OK) return rc;
    a.carry_in = carries;
  }
  return half_launch<R>(a, mode, ax->elems, s);
}

// One application of Algorithm 1 on the grids (o_is_x = 0: psi <- nu / K^T
// phi with the loop-head check; 1: phi <- mu / K psi).  K psi: W = nu in L_0,
// axes 0 .. d-1, output mu in L_{d-1}; K^T phi: W = mu in L_{d-1}, axes d-1
// .. 0, output nu in L_0.  The source grid is read from src, the output
// grid's frames from dst_in, its new log-weights go to dst_out.
template <class R>
finom_status nd_application(finom_plan_s* p, int o_is_x, const LvT<R>* src, const LvT<R>* dst_in,
                            LvT<R>* dst_out, bool check_only, cudaStream_t s) {
  SolveState& st = p->st;
  const int d = p->dim;
  LvT<R>* Qa = (LvT<R>*)st.q2;
  LvT<R>* Qb = Qa + p->nd_G;
  const LvT<R>* lm = (const LvT<R>*)(o_is_x ? st.qom : st.qwm);
  const LvT<R>* w = src;
  for (int j = 0; j < d; ++j) {
    const int k = o_is_x ? j : d - 1 - j;
    finom_status rc;
    if (j + 1 < d) {
      rc = nd_pass<R>(p, k, o_is_x, w, kLineQ, nullptr, nullptr, nullptr, Qa, nullptr, nullptr, (R*)st.aggs,
                      (R*)st.carries, st.part, s, st.tol, st.maxit);
      if (rc != FINOM_OK) return rc;
      nd_rot(p, k, o_is_x != 0, Qa, Qb, s);
      w = Qb;
      continue;
    } else {
      const int mode = check_only ? kLineCheck : (o_is_x ? kLineX : kLineY);
      rc = nd_pass<R>(p, k, o_is_x, w, mode, dst_in, dst_out, lm, nullptr, nullptr, nullptr, (R*)st.aggs,
                      (R*)st.carries, st.part, s, st.tol, st.maxit);
    }
    if (rc != FINOM_OK) return rc;
  }
  return FINOM_OK;
}

// iteration with parity q: psi from py[q] to py[1-q] against phi px[q], then
// phi from px[q] to px[1-q] against the new psi
template <class R>
finom_status nd_iteration(finom_plan_s* p, int q, cudaStream_t s) {
  SolveState& st = p->st;
  finom_status rc = nd_application<R>(p, 0, (const LvT<R>*)st.px[q], (const LvT<R>*)st.py[q],
                                      (LvT<R>*)st.py[1 - q], false, s);
  if (rc != FINOM_OK) return rc;
  return nd_application<R>(p, 1, (const LvT<R>*)st.py[1 - q], (const LvT<R>*)st.px[q], (LvT<R>*)st.px[1 - q],
                           false, s);
}

template <class R>
finom_status nd_build_body(finom_plan_s* p, int pairs, cudaGraphExec_t* out) {
  SolveState& st = p->st;
  if (*out) {
    cudaGraphExecDestroy(*out);
    *out = nullptr;
  }
  cudaGraph_t g = nullptr;
  FINOM_CUDA(cudaStreamBeginCapture(st.stream, cudaStreamCaptureModeThreadLocal));
  finom_status rc = FINOM_OK;
  for (int k = 0; k < pairs && rc == FINOM_OK; ++k) {
    rc = nd_iteration<R>(p, 1, st.stream);
    if (rc == FINOM_OK) rc = nd_iteration<R>(p, 0, st.stream);
  }
  cudaError_t e = cudaStreamEndCapture(st.stream, &g);
  if (rc != FINOM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return FINOM_OK;
}

template <class R>
finom_status nd_begin(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                      const double* f0, const double* g0, cudaStream_t s) {
  finom_status rc = ensure_state_nd<R>(p);
  if (rc != FINOM_OK) return rc;
  SolveState& st = p->st;
  const int64_t G = p->nd_G;
  // masses: nu's in L_0; mu's normalised in L_0, then turned into L_{d-1}
  double* red = st.scal + 256;   // partial sums of the normalisation
  rc = normalise_masses(u, G, st.tx, red, st.bad, nullptr, s);
  if (rc != FINOM_OK) return rc;
  nd_rot(p, 0, false, (const double*)st.tx, st.mu64, s);
  rc = normalise_masses(v, G, st.nu64, red, st.bad, nullptr, s);
  if (rc != FINOM_OK) return rc;
  const double none = (double)HT<R>::kNone;
  k_grid_lmass<<<nb(G), 256, 0, s>>>(st.mu64, G, (LvT<R>*)st.qom, none);
  k_grid_lmass<<<nb(G), 256, 0, s>>>(st.nu64, G, (LvT<R>*)st.qwm, none);
  const double scale = 1.0 / (p->eps * kLn2);
  st.warm = (f0 != nullptr && g0 != nullptr);
  const double start = std::log2(1.0 / (double)G);   // Algorithm 2: Phi = Psi = 1/(NM)
  LvT<R>* tmp = (LvT<R>*)st.q2;
  k_grid_set<<<nb(G), 256, 0, s>>>(tmp, G, st.warm ? f0 : nullptr, scale, start, none);
  nd_rot(p, 0, false, (const LvT<R>*)tmp, (LvT<R>*)st.px[0], s);
  k_grid_set<<<nb(G), 256, 0, s>>>((LvT<R>*)st.py[0], G, st.warm ? g0 : nullptr, scale, start, none);
  FINOM_CUDA(cudaGetLastError());
  FINOM_CUDA(cudaMemsetAsync(st.ctrl, 0, sizeof(int32_t) * 8, s));
  FINOM_CUDA(cudaMemsetAsync(st.scal, 0, sizeof(double) * 8, s));
  st.tol = tol;
  st.maxit = maxit;
  st.launched = 0;
  st.active = true;
  if (maxit == 0) {   // only the loop-head check of l = 0
    return nd_application<R>(p, 0, (const LvT<R>*)st.px[0], (const LvT<R>*)st.py[0], (LvT<R>*)st.py[1], true, s);
  }
  rc = nd_iteration<R>(p, 0, s);
  if (rc != FINOM_OK) return rc;
  st.launched = 1;
  return FINOM_OK;
}

template <class R>
finom_status nd_step(finom_plan_s* p, int64_t iters, cudaStream_t s) {
  SolveState& st = p->st;
  for (int64_t k = 0; k < iters;) {
    if ((st.launched & 1) && iters - k >= kChunkIters) {
      if (!st.chunk || st.chunk_tol != st.tol || st.chunk_maxit != st.maxit) {
        finom_status rc = nd_build_body<R>(p, kChunkIters / 2, &st.chunk);
        if (rc != FINOM_OK) return rc;
        st.chunk_tol = st.tol;
        st.chunk_maxit = st.maxit;
      }
      FINOM_CUDA(cudaGraphLaunch(st.chunk, s));
      st.launched += kChunkIters;
      k += kChunkIters;
      continue;
    }
    finom_status rc = nd_iteration<R>(p, (int)(st.launched & 1), s);
    if (rc != FINOM_OK) return rc;
    ++st.launched;
    ++k;
  }
  return FINOM_OK;
}

finom_status nd_poll(finom_plan_s* p, cudaStream_t s, int32_t* done, int64_t* iters) {
  int32_t h[8];
  FINOM_CUDA(cudaMemcpyAsync(h, p->st.ctrl, sizeof(h), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  if (done) *done = h[1];
  if (iters) *iters = h[1] ? h[3] : h[2];
  return FINOM_OK;
}

// float64 check of given log-weight grids bx (mu, layout L_{d-1}) and by
// (nu, L_0), in bits, with the masses mu (L_{d-1}) and nu (L_0):
// the marginal error sum_j |psi_j (K^T phi)_j - nu_j| of Algorithm 1's loop
// head and W1 = <C, Gamma> = sum_k <C_k, Gamma> (C_k: the axis-k part of the
// separable cost), from axis passes of the float64 kernel.
finom_status nd_check64(finom_plan_s* p, const double* bx, const double* by, const double* mu,
                        const double* nu, double* err, double* w1, cudaStream_t s) {
  double* ws = w64(p);
  if (!ws) {
    set_error("d-dimensional check: out of device memory");
    return FINOM_ENOMEM;
  }
  const int64_t G = p->nd_G, U = nd_units(p);
  double *Qa = ws, *Qb = ws + G, *FB0 = ws + 2 * G, *FB1 = ws + 4 * G, *Qm = ws + 6 * G;
  // kernel partials per unit, then up to 256 block partials of the grid
  // sums, then the sums themselves
  double *aggs = ws + 8 * G, *carries = aggs + 4 * U, *part = carries + 4 * U, *red = part + U,
         *sums = red + 256;
  const int d = p->dim;
  const int blocks = (int)std::min<int64_t>(256, (G + 255) / 256);
  // marginal error: K^T phi on the nu grid (axes d-1 .. 0, from L_{d-1} to L_0)
  {
    const double* w = bx;
    for (int k = d - 1; k >= 0; --k) {
      finom_status rc = nd_pass<double>(p, k, 0, w, kLineQ, nullptr, nullptr, nullptr, Qa, nullptr, nullptr,
                                        aggs, carries, part, s, 0.0, 0);
      if (rc != FINOM_OK) return rc;
      w = Qa;
      if (k > 0) {
        nd_rot(p, k, false, (const double*)Qa, Qb, s);
        w = Qb;
      }
    }
    k_grid_sum<<<blocks, 256, 0, s>>>(by, w, nu, G, 0, red);
    k_sum_parts<<<1, 32, 0, s>>>(red, blocks, sums);
  }
  // <C_k, Gamma> for every axis k: K psi (axes 0 .. d-1, from L_0 to
  // L_{d-1}) with axis k cost-weighted, then sum_i phi_i (.)_i
  for (int k = 0; k < d; ++k) {
    const double* w = by;
    for (int j = 0; j < d; ++j) {
      finom_status rc;
      double* out = Qa;
      if (j == k) {
        rc = nd_pass<double>(p, j, 1, w, kLineFB, nullptr, nullptr, nullptr, nullptr, FB0, nullptr, aggs,
                             carries, part, s, 0.0, 0);
        if (rc == FINOM_OK)
          rc = nd_pass<double>(p, j, 1, w, kLineFBZ, nullptr, nullptr, nullptr, nullptr, FB1, p->nd_ly64[j],
                               aggs, carries, part, s, 0.0, 0);
        if (rc != FINOM_OK) return rc;
        // layout L_j: the node along axis j is the fastest index
        k_moment<<<nb(G), 256, 0, s>>>(FB0, FB1, G, p->nd_zx64[j], p->nd_z0s[j], 1, p->nd_n[j], Qm);
        out = Qm;
      } else {
        rc = nd_pass<double>(p, j, 1, w, kLineQ, nullptr, nullptr, nullptr, Qa, nullptr, nullptr, aggs, carries,
                             part, s, 0.0, 0);
        if (rc != FINOM_OK) return rc;
      }
      w = out;
      if (j + 1 < d) {
        nd_rot(p, j, true, (const double*)out, Qb, s);
        w = Qb;
      }
    }
    k_grid_sum<<<blocks, 256, 0, s>>>(bx, w, mu, G, 1, red);
    k_sum_parts<<<1, 32, 0, s>>>(red, blocks, sums + 1 + k);
  }
  FINOM_CUDA(cudaGetLastError());
  double h[1 + finom_plan_s::kMaxDim];
  FINOM_CUDA(cudaMemcpyAsync(h, sums, sizeof(double) * (1 + d), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  *err = h[0];
  double tot = 0.0;
  for (int k = 0; k < d; ++k) tot += h[1 + k];
  *w1 = p->eps * kLn2 * tot;
  return FINOM_OK;
}

template <class R>
finom_status nd_end(finom_plan_s* p, double* f, double* g, finom_result* res, cudaStream_t s) {
  SolveState& st = p->st;
  const int64_t G = p->nd_G;
  int32_t h[8];
  double loop_err = 0.0;
  FINOM_CUDA(cudaMemcpyAsync(h, st.ctrl, sizeof(h), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaMemcpyAsync(&loop_err, st.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  const bool done = h[1] != 0;
  int64_t iters = done ? h[3] : h[2];
  if (st.maxit == 0) iters = 0;
  const int q = (int)(iters & 1);
  const double none = (double)HT<R>::kNone;
  k_grid_to64<<<nb(G), 256, 0, s>>>((const LvT<R>*)st.px[q], G, none, st.tx);
  k_grid_to64<<<nb(G), 256, 0, s>>>((const LvT<R>*)st.py[q], G, none, st.ty);
  double err64 = 0.0, w1 = 0.0;
  finom_status rc = nd_check64(p, st.tx, st.ty, st.mu64, st.nu64, &err64, &w1, s);
  if (rc != FINOM_OK) return rc;
  const double eps_ln2 = p->eps * kLn2;
  double* d2 = st.scal + 16;
  if (iters == 0 && !st.warm) {
    // the start Phi = Psi = 1/(NM) at every point (Algorithm 2)
    fill_d(f, G, p->eps * std::log(1.0 / (double)G), s);
    fill_d(g, G, p->eps * std::log(1.0 / (double)G), s);
    dot_pos(st.mu64, f, G, d2, s);
  } else {
    // mu's potentials in L_{d-1}, then in the caller's order
    double* fd = (double*)st.q2;
    k_f_of<<<nb(G), 256, 0, s>>>(st.tx, st.mu64, G, eps_ln2, fd);
    dot_pos(st.mu64, fd, G, d2, s);
    nd_rot(p, p->dim - 1, true, (const double*)fd, f, s);
    k_f_of<<<nb(G), 256, 0, s>>>(st.ty, st.nu64, G, eps_ln2, g);
  }
  dot_pos(st.nu64, g, G, d2 + 1, s);
  double hd[2];
  FINOM_CUDA(cudaMemcpyAsync(hd, d2, sizeof(hd), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  if (res) {
    res->w1 = w1;
    res->marginal_err = err64;
    res->marginal_err_loop = loop_err;
    res->dual = hd[0] + hd[1];
    res->iters = iters;
    res->converged = (err64 <= st.tol) ? 1 : 0;
    res->status = FINOM_OK;
  }
  st.active = false;
  return FINOM_OK;
}

template <class R>
finom_status nd_blocking(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit, double* f,
                         double* g, int32_t warm, finom_result* res, cudaStream_t us) {
  FINOM_CUDA(cudaStreamSynchronize(us));
  finom_status rc = ensure_state_nd<R>(p);
  if (rc != FINOM_OK) return rc;
  SolveState& st = p->st;
  cudaStream_t s = st.stream;
  rc = nd_begin<R>(p, u, v, tol, maxit, warm ? f : nullptr, warm ? g : nullptr, s);
  if (rc != FINOM_OK) return rc;
  if (maxit > 0) {
    // loop until the device check stops it; a float32 stop is verified in
    // float64 and, if needed, resumed from its exact state with a tighter
    // loop tolerance (as for 1D plans)
    for (int attempt = 0;; ++attempt) {
      rc = nd_build_body<R>(p, 1, &st.body);
      if (rc != FINOM_OK) return rc;
      int64_t bodies = 1;
      for (;;) {
        int32_t done = 0;
        rc = nd_poll(p, s, &done, nullptr);
        if (rc != FINOM_OK) return rc;
        if (done) break;
        if (st.launched & 1) {
          for (int64_t b = 0; b < bodies; ++b) FINOM_CUDA(cudaGraphLaunch(st.body, s));
          st.launched += 2 * bodies;
        } else {
          rc = nd_step<R>(p, 1, s);
          if (rc != FINOM_OK) return rc;
        }
        bodies = std::min<int64_t>(bodies * 2, 64);
      }
      if (sizeof(R) == sizeof(double) || attempt >= 6) break;
      int32_t h[8];
      double loop_err = 0.0;
      FINOM_CUDA(cudaMemcpyAsync(h, st.ctrl, sizeof(h), cudaMemcpyDeviceToHost, s));
      FINOM_CUDA(cudaMemcpyAsync(&loop_err, st.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
      FINOM_CUDA(cudaStreamSynchronize(s));
      if (!h[4]) break;                      // stopped at maxit
      const int64_t l = h[3];
      if (l == 0 && !st.warm) break;
      const int q = (int)(l & 1);
      const int64_t G = p->nd_G;
      const double none = (double)HT<R>::kNone;
      k_grid_to64<<<nb(G), 256, 0, s>>>((const LvT<R>*)st.px[q], G, none, st.tx);
      k_grid_to64<<<nb(G), 256, 0, s>>>((const LvT<R>*)st.py[q], G, none, st.ty);
      double err64 = 0.0, w1 = 0.0;
      rc = nd_check64(p, st.tx, st.ty, st.mu64, st.nu64, &err64, &w1, s);
      if (rc != FINOM_OK) return rc;
      if (err64 <= tol) break;
      const double fct = std::max(0.1, std::min(0.97, 0.97 * tol / err64));
      st.tol = std::max(loop_err * fct, 0.0);
      int32_t zero[2] = {0, 0};
      FINOM_CUDA(cudaMemcpyAsync(st.ctrl + 1, &zero[0], sizeof(int32_t), cudaMemcpyHostToDevice, s));
      FINOM_CUDA(cudaMemcpyAsync(st.ctrl + 4, &zero[1], sizeof(int32_t), cudaMemcpyHostToDevice, s));
      rc = nd_application<R>(p, 1, (const LvT<R>*)st.py[1 - q], (const LvT<R>*)st.px[q], (LvT<R>*)st.px[1 - q],
                             false, s);
      if (rc != FINOM_OK) return rc;
      st.launched = l + 1;
    }
    st.tol = tol;
  }
  return nd_end<R>(p, f, g, res, s);
}

// K w (transpose: K^T w) on the grids, linear or log form (see finom_kv_log)
template <class R>
finom_status nd_product(finom_plan_s* p, bool transpose, bool logmode, const double* a, const double* b,
                        double* out, cudaStream_t s) {
  finom_status rc = ensure_state_nd<R>(p);
  if (rc != FINOM_OK) return rc;
  SolveState& st = p->st;
  st.active = false;
  const int64_t G = p->nd_G;
  const double none = (double)HT<R>::kNone;
  const double scale = 1.0 / (p->eps * kLn2);
  const double* ao = logmode ? (transpose ? b : a) : nullptr;
  const double* bw = logmode ? (transpose ? a : b) : b;
  LvT<R>* w0 = (LvT<R>*)st.py[0];   // scratch: the weights as log2 levels
  if (logmode) k_grid_set<<<nb(G), 256, 0, s>>>(w0, G, bw, scale, 0.0, none);
  else k_grid_lin<<<nb(G), 256, 0, s>>>(w0, G, bw, none);
  const int o_is_x = transpose ? 0 : 1;
  // axes 0 .. d-1, each pass from L_k, then into L_{k+1} (L_d = L_0)
  LvT<R>* Qa = (LvT<R>*)st.q2;
  LvT<R>* Qb = Qa + G;
  const LvT<R>* w = w0;
  for (int k = 0; k < p->dim; ++k) {
    rc = nd_pass<R>(p, k, o_is_x, w, kLineQ, nullptr, nullptr, nullptr, Qa, nullptr, nullptr, (R*)st.aggs,
                    (R*)st.carries, st.part, s, 0.0, 0);
    if (rc != FINOM_OK) return rc;
    w = Qa;
    if (p->dim > 1) {
      nd_rot(p, k, true, (const LvT<R>*)Qa, Qb, s);
      w = Qb;
    }
  }
  k_prod_out<<<nb(G), 256, 0, s>>>(w, G, ao, 1.0 / p->eps, logmode ? 0 : 1, none, out);
  FINOM_CUDA(cudaGetLastError());
  return FINOM_OK;
}

}  // namespace

finom_status plan_nd_build(finom_plan_s* p, int d, const int64_t* n, const double* const* xs,
                           const double* const* ys, cudaStream_t s) {
  p->nd = true;
  p->dim = d;
  int64_t G = 1;
  for (int k = 0; k < d; ++k) {
    p->nd_n[k] = n[k];
    G *= n[k];
  }
  p->nd_G = G;
  p->N = G;
  p->M = G;
  const double scale = 1.0 / (p->eps * kLn2);
  const bool f32 = p->prec == FINOM_F32_LOG;
  for (int k = 0; k < d; ++k) {
    finom_plan_s* ax = new (std::nothrow) finom_plan_s();
    if (!ax) return FINOM_ENOMEM;
    p->nd_ax[k] = ax;
    ax->N = n[k];
    ax->M = n[k];
    ax->eps = p->eps;
    ax->prec = p->prec;
    ax->device = p->device;
    finom_status rc = build_plan(ax, xs[k], ys[k], s);
    // the smallest tile that holds a whole line (lines give the parallelism;
    // a line in one tile needs no carries and no aggregate launch)
    int e = kElemsSmall;
    if (tile_points(e) < 2 * n[k]) {
      e = 1;
      while (e < kElems && tile_points(e) < 2 * n[k]) e *= 2;
    }
    if (rc == FINOM_OK) rc = build_tiles_e(ax, e, s);
    if (rc != FINOM_OK) return rc;
    // the axis minimum over both meshes (the sorted copies' first entries)
    double x0 = 0.0, y0 = 0.0;
    FINOM_CUDA(cudaMemcpyAsync(&x0, ax->x, sizeof(double), cudaMemcpyDeviceToHost, s));
    FINOM_CUDA(cudaMemcpyAsync(&y0, ax->y, sizeof(double), cudaMemcpyDeviceToHost, s));
    FINOM_CUDA(cudaStreamSynchronize(s));
    const double z0 = std::min(x0, y0);
    p->nd_z0s[k] = z0 * scale;
    const size_t lv = f32 ? sizeof(float2) : sizeof(double);
    FINOM_CUDA(cudaMalloc(&p->nd_zx[k], lv * n[k]));
    FINOM_CUDA(cudaMalloc(&p->nd_zy[k], lv * n[k]));
    FINOM_CUDA(cudaMalloc(&p->nd_zx64[k], sizeof(double) * n[k]));
    FINOM_CUDA(cudaMalloc(&p->nd_zy64[k], sizeof(double) * n[k]));
    FINOM_CUDA(cudaMalloc(&p->nd_lx64[k], sizeof(double) * n[k]));
    FINOM_CUDA(cudaMalloc(&p->nd_ly64[k], sizeof(double) * n[k]));
    if (f32) {
      k_axis_tables<<<nb(n[k]), 256, 0, s>>>(ax->x, n[k], scale, z0, (float2*)p->nd_zx[k], p->nd_zx64[k], p->nd_lx64[k]);
      k_axis_tables<<<nb(n[k]), 256, 0, s>>>(ax->y, n[k], scale, z0, (float2*)p->nd_zy[k], p->nd_zy64[k], p->nd_ly64[k]);
    } else {
      k_axis_tables<<<nb(n[k]), 256, 0, s>>>(ax->x, n[k], scale, z0, (double*)p->nd_zx[k], p->nd_zx64[k], p->nd_lx64[k]);
      k_axis_tables<<<nb(n[k]), 256, 0, s>>>(ax->y, n[k], scale, z0, (double*)p->nd_zy[k], p->nd_zy64[k], p->nd_ly64[k]);
    }
    FINOM_CUDA(cudaGetLastError());
  }
  FINOM_CUDA(cudaStreamSynchronize(s));
  return FINOM_OK;
}

void plan_nd_free(finom_plan_s* p) {
  for (int k = 0; k < finom_plan_s::kMaxDim; ++k) {
    if (p->nd_ax[k]) {
      free_plan(p->nd_ax[k]);
      delete p->nd_ax[k];
      p->nd_ax[k] = nullptr;
    }
    void* bufs[] = {p->nd_zx[k], p->nd_zy[k], p->nd_zx64[k], p->nd_zy64[k], p->nd_lx64[k], p->nd_ly64[k]};
    for (void* b : bufs) cudaFree(b);
  }
  cudaFree(p->nd_w64);
  p->nd_w64 = nullptr;
}

finom_status kv_nd(finom_plan_s* p, bool transpose_k, bool logmode, const double* a, const double* b,
                   double* out, cudaStream_t s) {
  return p->prec == FINOM_F32_LOG ? nd_product<float>(p, transpose_k, logmode, a, b, out, s)
                                  : nd_product<double>(p, transpose_k, logmode, a, b, out, s);
}

finom_status solve_nd(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                      double* f, double* g, int32_t warm, finom_result* res, cudaStream_t s) {
  return p->prec == FINOM_F32_LOG ? nd_blocking<float>(p, u, v, tol, maxit, f, g, warm, res, s)
                                  : nd_blocking<double>(p, u, v, tol, maxit, f, g, warm, res, s);
}

finom_status solve_nd_begin(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                            const double* f0, const double* g0, cudaStream_t s) {
  return p->prec == FINOM_F32_LOG ? nd_begin<float>(p, u, v, tol, maxit, f0, g0, s)
                                  : nd_begin<double>(p, u, v, tol, maxit, f0, g0, s);
}

finom_status solve_nd_step(finom_plan_s* p, int64_t iters, cudaStream_t s) {
  return p->prec == FINOM_F32_LOG ? nd_step<float>(p, iters, s) : nd_step<double>(p, iters, s);
}

finom_status solve_nd_end(finom_plan_s* p, double* f, double* g, finom_result* res, cudaStream_t s) {
  return p->prec == FINOM_F32_LOG ? nd_end<float>(p, f, g, res, s) : nd_end<double>(p, f, g, res, s);
}

// W1 and the marginal error of given potentials f (mu grid), g (nu grid)
// and masses u, v (normalised here), in float64
finom_status cost_nd(finom_plan_s* p, const double* u, const double* v, const double* f, const double* g,
                     double* w1, double* err, cudaStream_t s) {
  finom_status rc = p->prec == FINOM_F32_LOG ? ensure_state_nd<float>(p) : ensure_state_nd<double>(p);
  if (rc != FINOM_OK) return rc;
  SolveState& st = p->st;
  const int64_t G = p->nd_G;
  double* red = st.scal + 256;
  // mu's masses and log-weights into L_{d-1} (through ty), nu's in L_0
  rc = normalise_masses(u, G, st.ty, red, st.bad, nullptr, s);
  if (rc != FINOM_OK) return rc;
  nd_rot(p, 0, false, (const double*)st.ty, st.mu64, s);
  rc = normalise_masses(v, G, st.nu64, red, st.bad, nullptr, s);
  if (rc != FINOM_OK) return rc;
  const double scale = 1.0 / (p->eps * kLn2);
  k_grid_set<<<nb(G), 256, 0, s>>>(st.ty, G, f, scale, 0.0, -INFINITY);
  nd_rot(p, 0, false, (const double*)st.ty, st.tx, s);
  k_grid_set<<<nb(G), 256, 0, s>>>(st.ty, G, g, scale, 0.0, -INFINITY);
  st.active = false;
  return nd_check64(p, st.tx, st.ty, st.mu64, st.nu64, err, w1, s);
}

}  // namespace finom
