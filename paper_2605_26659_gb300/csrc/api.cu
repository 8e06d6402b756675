// C ABI of libfinom: argument checking, plan lifetime, kernel products and
// the Sinkhorn loop (Algorithm 1) driven from the host with CUDA graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>
#include <new>
#include <string>

#include "finom_internal.h"
#include "half.cuh"

namespace finom {

static thread_local std::string g_err;

void set_error(const std::string& m) { g_err = m; }

finom_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FINOM_ENOMEM : FINOM_ECUDA;
}

template <class R>
finom_status half_launch(const HalfArgs<R>&, int, int, cudaStream_t);
template <class R>
void beta_set(void*, const double*, int64_t, double, const double*, double, double, cudaStream_t);
template <class R>
void beta_lin(void*, const double*, int64_t, double, const double*, cudaStream_t);
template <class R>
void log_mass(const double*, int64_t, void*, cudaStream_t);
template <class R>
void f_from_beta(const void*, const double*, int64_t, double, double*, double*, cudaStream_t);

namespace {

constexpr double kLn2 = 0.69314718055994530942;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

template <class R>
constexpr size_t beta_size() { return sizeof(typename HT<R>::Beta); }
template <class R>
constexpr size_t level_size() { return sizeof(typename HT<R>::Lv); }

// Device state of the loop of a 1D plan: per point its two levels
// (beta+, beta-) of the half-step kernel (half.cuh), ping-pong; log2 masses;
// float64 masses; tile aggregates and carries (two log-sum states per tile).
template <class R>
finom_status ensure_state(finom_plan_s* p) {
  SolveState& st = p->st;
  if (st.ready) return FINOM_OK;
  const int64_t N = p->N, M = p->M, C = p->Ce, NM = std::max(N, M);
  const int64_t per_tile = 2 * HT<R>::kSt;
  for (int q = 0; q < 2; ++q) {
    FINOM_CUDA(cudaMalloc(&st.px[q], beta_size<R>() * N));
    FINOM_CUDA(cudaMalloc(&st.py[q], beta_size<R>() * M));
  }
  FINOM_CUDA(cudaMalloc(&st.qom, level_size<R>() * N));   // log2 masses of x
  FINOM_CUDA(cudaMalloc(&st.qwm, level_size<R>() * M));   // log2 masses of y
  FINOM_CUDA(cudaMalloc(&st.mu64, sizeof(double) * N));
  FINOM_CUDA(cudaMalloc(&st.nu64, sizeof(double) * M));
  // (also the scratch of normalise_masses: at least 257 entries)
  FINOM_CUDA(cudaMalloc(&st.tx, sizeof(double) * std::max<int64_t>(N, 512)));
  FINOM_CUDA(cudaMalloc(&st.ty, sizeof(double) * std::max<int64_t>(M, 512)));
  FINOM_CUDA(cudaMalloc(&st.aggs, sizeof(R) * per_tile * C));
  FINOM_CUDA(cudaMalloc(&st.carries, sizeof(R) * per_tile * C));
  FINOM_CUDA(cudaMalloc(&st.part, sizeof(double) * C));
  FINOM_CUDA(cudaMalloc(&st.scal, sizeof(double) * 520));
  FINOM_CUDA(cudaMalloc(&st.ctrl, sizeof(int32_t) * 8));
  FINOM_CUDA(cudaMalloc(&st.bad, sizeof(int)));
  FINOM_CUDA(cudaMalloc(&st.qo, beta_size<R>() * NM));
  FINOM_CUDA(cudaMalloc(&st.qw, beta_size<R>() * NM));
  FINOM_CUDA(cudaMemset(st.ctrl, 0, sizeof(int32_t) * 8));
  FINOM_CUDA(cudaMemset(st.scal, 0, sizeof(double) * 520));
  FINOM_CUDA(cudaMemset(st.carries, 0, sizeof(R) * per_tile * C));
  FINOM_CUDA(cudaStreamCreateWithFlags(&st.stream, cudaStreamNonBlocking));
  st.ready = true;
  return FINOM_OK;
}

void free_state(finom_plan_s* p) {
  SolveState& st = p->st;
  if (st.body) cudaGraphExecDestroy(st.body);
  if (st.chunk) cudaGraphExecDestroy(st.chunk);
  for (int q = 0; q < 2; ++q) {
    cudaFree(st.px[q]);
    cudaFree(st.py[q]);
  }
  void* bufs[] = {st.mu64, st.nu64, st.tx, st.ty, st.aggs, st.carries, st.part, st.scal, st.ctrl,
                  st.bad, st.qo, st.qom, st.qw, st.qwm, st.q2, st.ictl, st.ierr, st.itol, st.alist};
  for (void* b : bufs) cudaFree(b);
  if (st.stream) cudaStreamDestroy(st.stream);
  st = SolveState();
}

template <class R>
HalfArgs<R> base_args(finom_plan_s* p) {
  HalfArgs<R> a{};
  a.tbits = p->tbits;
  a.tile_x0 = p->tile_x0e;
  a.L = p->L;
  a.C = (int)p->Ce;
  a.agg_out = (R*)p->st.aggs;
  a.carry_in = (const R*)p->st.carries;
  a.carry_out = (R*)p->st.carries;
  a.part = p->st.part;
  a.scal = p->st.scal;
  a.ctrl = p->st.ctrl;
  return a;
}

template <class R>
finom_status launch_half(const HalfArgs<R>& a, int mode, finom_plan_s* p, cudaStream_t s) {
  return half_launch<R>(a, mode, p->elems, s);
}

// One kernel product: O frames qo, W levels qw; the tile aggregates of the
// W side first, then the product itself (outputs to out).
template <class R>
finom_status product(finom_plan_s* p, int o_is_x, double* out, int mode, cudaStream_t s) {
  using Beta = typename HT<R>::Beta;
  SolveState& st = p->st;
  st.active = false;   // a product overwrites the loop's scan scratch
  HalfArgs<R> a = base_args<R>(p);
  a.o_is_x = o_is_x;
  a.bO = (const Beta*)st.qo;
  a.bW = (const Beta*)st.qw;
  a.out = out;
  a.carry_in = nullptr;
  finom_status rc = launch_half<R>(a, kHalfAgg, p, s);
  if (rc != FINOM_OK) return rc;
  a.carry_in = (const R*)st.carries;
  return launch_half<R>(a, mode, p, s);
}

template <class R>
HalfArgs<R> half_args(finom_plan_s* p, bool o_is_x, int q) {
  using Beta = typename HT<R>::Beta;
  using Lv = typename HT<R>::Lv;
  SolveState& st = p->st;
  HalfArgs<R> a = base_args<R>(p);
  a.tol = st.tol;
  a.maxit = st.maxit;
  if (!o_is_x) {   // psi <- nu / (K^T phi): outputs on y, weights on x
    a.o_is_x = 0;
    a.bO = (const Beta*)st.py[q];
    a.lmO = (const Lv*)st.qwm;
    a.mO = st.nu64;
    a.bO_out = (Beta*)st.py[1 - q];
    a.bW = (const Beta*)st.px[q];
  } else {         // phi <- mu / (K psi): outputs on x, weights on y
    a.o_is_x = 1;
    a.bO = (const Beta*)st.px[q];
    a.lmO = (const Lv*)st.qom;
    a.bO_out = (Beta*)st.px[1 - q];
    a.bW = (const Beta*)st.py[1 - q];
  }
  return a;
}

// one Sinkhorn iteration with parity q (iteration l has q = l % 2)
template <class R>
finom_status launch_iteration(finom_plan_s* p, int q, cudaStream_t s) {
  finom_status rc = launch_half<R>(half_args<R>(p, false, q), kHalfY, p, s);
  if (rc != FINOM_OK) return rc;
  return launch_half<R>(half_args<R>(p, true, q), kHalfX, p, s);
}

// graph of 2 * pairs iterations starting at an odd iteration (q = 1, 0, 1, ...)
template <class R>
finom_status build_body(finom_plan_s* p, int pairs, cudaGraphExec_t* out) {
  SolveState& st = p->st;
  if (*out) {
    cudaGraphExecDestroy(*out);
    *out = nullptr;
  }
  cudaGraph_t g = nullptr;
  FINOM_CUDA(cudaStreamBeginCapture(st.stream, cudaStreamCaptureModeThreadLocal));
  finom_status rc = FINOM_OK;
  for (int k = 0; k < pairs && rc == FINOM_OK; ++k) {
    rc = launch_iteration<R>(p, 1, st.stream);
    if (rc == FINOM_OK) rc = launch_iteration<R>(p, 0, st.stream);
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
finom_status solve_begin(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                         const double* f0, const double* g0, cudaStream_t s) {
  finom_status rc = ensure_state<R>(p);
  if (rc != FINOM_OK) return rc;
  SolveState& st = p->st;
  const int64_t N = p->N, M = p->M;
  rc = normalise_masses(u, N, st.mu64, st.tx, st.bad, nullptr, s);
  if (rc != FINOM_OK) return rc;
  rc = normalise_masses(v, M, st.nu64, st.ty, st.bad, nullptr, s);
  if (rc != FINOM_OK) return rc;
  log_mass<R>(st.mu64, N, st.qom, s);
  log_mass<R>(st.nu64, M, st.qwm, s);
  const double scale = 1.0 / (p->eps * kLn2);
  st.warm = (f0 != nullptr && g0 != nullptr);
  if (st.warm) {
    beta_set<R>(st.px[0], p->x, N, scale, f0, scale, 0.0, s);
    beta_set<R>(st.py[0], p->y, M, scale, g0, scale, 0.0, s);
  } else {
    // the paper's start phi = 1/N, psi = 1/M at every point
    beta_set<R>(st.px[0], p->x, N, scale, nullptr, 0.0, std::log2(1.0 / (double)N), s);
    beta_set<R>(st.py[0], p->y, M, scale, nullptr, 0.0, std::log2(1.0 / (double)M), s);
  }
  FINOM_CUDA(cudaMemsetAsync(st.ctrl, 0, sizeof(int32_t) * 8, s));
  FINOM_CUDA(cudaMemsetAsync(st.scal, 0, sizeof(double) * 8, s));
  st.tol = sizeof(R) == sizeof(float) ? std::max(tol, kF32LoopFloor) : tol;
  st.tol_user = tol;
  st.maxit = maxit;
  st.launched = 0;
  st.active = true;
  // iteration 0: the tile aggregates of phi, then psi <- nu / K^T phi (its
  // loop-head check against the starting psi), then phi <- mu / K psi
  HalfArgs<R> a0 = half_args<R>(p, false, 0);
  HalfArgs<R> agg = a0;
  agg.carry_in = nullptr;
  rc = launch_half<R>(agg, kHalfAgg, p, s);
  if (rc != FINOM_OK) return rc;
  if (maxit == 0) return launch_half<R>(a0, kHalfCheck, p, s);   // only the loop-head check of l = 0
  rc = launch_half<R>(a0, kHalfY, p, s);
  if (rc != FINOM_OK) return rc;
  rc = launch_half<R>(half_args<R>(p, true, 0), kHalfX, p, s);
  if (rc != FINOM_OK) return rc;
  st.launched = 1;
  return FINOM_OK;
}

// Iterations of a stepwise solve: single launches up to an odd iteration,
// then graphs of kChunkIters iterations, then single launches for the rest.
template <class R>
finom_status solve_step(finom_plan_s* p, int64_t iters, cudaStream_t s) {
  SolveState& st = p->st;
  for (int64_t k = 0; k < iters;) {
    if ((st.launched & 1) && iters - k >= kChunkIters) {
      if (!st.chunk || st.chunk_tol != st.tol || st.chunk_maxit != st.maxit) {
        finom_status rc = build_body<R>(p, kChunkIters / 2, &st.chunk);
        if (rc != FINOM_OK) return rc;
        st.chunk_tol = st.tol;
        st.chunk_maxit = st.maxit;
      }
      FINOM_CUDA(cudaGraphLaunch(st.chunk, s));
      st.launched += kChunkIters;
      k += kChunkIters;
      continue;
    }
    finom_status rc = launch_iteration<R>(p, (int)(st.launched & 1), s);
    if (rc != FINOM_OK) return rc;
    ++st.launched;
    ++k;
  }
  return FINOM_OK;
}

finom_status solve_poll(finom_plan_s* p, cudaStream_t s, int32_t* done, int64_t* iters) {
  int32_t h[8];
  FINOM_CUDA(cudaMemcpyAsync(h, p->st.ctrl, sizeof(h), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  if (done) *done = h[1];
  if (iters) *iters = h[1] ? h[3] : h[2];
  return FINOM_OK;
}

template <class R>
finom_status solve_end(finom_plan_s* p, double* f, double* g, finom_result* res, cudaStream_t s) {
  SolveState& st = p->st;
  const int64_t N = p->N, M = p->M;
  int32_t h[8];
  double loop_err = 0.0;
  FINOM_CUDA(cudaMemcpyAsync(h, st.ctrl, sizeof(h), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaMemcpyAsync(&loop_err, st.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  const bool done = h[1] != 0;
  int64_t iters = done ? h[3] : h[2];
  int32_t converged = h[4];
  if (st.maxit == 0) iters = 0;
  const double eps_ln2 = p->eps * kLn2;
  double err64 = 0.0, w1 = 0.0;
  if (iters == 0 && !st.warm) {
    // the paper's start phi = 1/N, psi = 1/M; its marginal error is the one
    // the loop measured at the first loop head (plan precision)
    fill_d(f, N, p->eps * std::log(1.0 / (double)N), s);
    fill_d(g, M, p->eps * std::log(1.0 / (double)M), s);
    fill_d(st.tx, N, 0.0, s);
    fill_d(st.ty, M, 0.0, s);
    double* uu = nullptr;
    FINOM_CUDA(cudaMallocAsync(&uu, sizeof(double) * (N + M), s));
    fill_d(uu, N, 1.0 / (double)N, s);
    fill_d(uu + N, M, 1.0 / (double)M, s);
    finom_status rc = cost64(p, st.tx, st.ty, uu, uu + N, &err64, &w1, s);
    cudaFreeAsync(uu, s);
    if (rc != FINOM_OK) return rc;
    err64 = loop_err;
  } else {
    const int q = (int)(iters & 1);
    f_from_beta<R>(st.px[q], st.mu64, N, eps_ln2, f, st.tx, s);
    f_from_beta<R>(st.py[q], st.nu64, M, eps_ln2, g, st.ty, s);
    finom_status rc = cost64(p, st.tx, st.ty, st.mu64, st.nu64, &err64, &w1, s);
    if (rc != FINOM_OK) return rc;
  }
  double* d2 = st.scal + 16;
  dot_pos(st.mu64, f, N, d2, s);
  dot_pos(st.nu64, g, M, d2 + 1, s);
  double hd[2];
  FINOM_CUDA(cudaMemcpyAsync(hd, d2, sizeof(hd), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  if (res) {
    res->w1 = w1;
    res->marginal_err = err64;
    res->marginal_err_loop = loop_err;
    res->dual = hd[0] + hd[1];
    res->iters = iters;
    res->converged = (err64 <= st.tol_user || (converged && sizeof(R) == sizeof(double))) ? 1 : 0;
    res->status = FINOM_OK;
  }
  st.active = false;
  return FINOM_OK;
}

template <class R>
finom_status solve_blocking(finom_plan_s* p, const double* u, const double* v, double tol,
                            int64_t maxit, double* f, double* g, int32_t warm, finom_result* res,
                            cudaStream_t us) {
  FINOM_CUDA(cudaStreamSynchronize(us));   // inputs are produced on the caller's stream
  finom_status rc = ensure_state<R>(p);
  if (rc != FINOM_OK) return rc;
  SolveState& st = p->st;
  cudaStream_t s = st.stream;
  rc = solve_begin<R>(p, u, v, tol, maxit, warm ? f : nullptr, warm ? g : nullptr, s);
  if (rc != FINOM_OK) return rc;
  if (maxit > 0) {
    // Loop until the device-side check stops it.  When the check passed in
    // the plan's precision, verify the marginal error in float64; if that is
    // still above tol, tighten the loop tolerance and resume from the exact
    // state at the stop (the skipped phi half step of iteration l).
    for (int attempt = 0;; ++attempt) {
      rc = build_body<R>(p, 1, &st.body);
      if (rc != FINOM_OK) return rc;
      int64_t bodies = 1;
      for (;;) {
        int32_t done = 0;
        rc = solve_poll(p, s, &done, nullptr);
        if (rc != FINOM_OK) return rc;
        if (done) break;
        if (st.launched & 1) {
          for (int64_t b = 0; b < bodies; ++b) FINOM_CUDA(cudaGraphLaunch(st.body, s));
          st.launched += 2 * bodies;
        } else {
          rc = solve_step<R>(p, 1, s);
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
      if (l == 0 && !st.warm) break;         // the start already met tol
      double err64 = 0.0, w1 = 0.0;
      const int q = (int)(l & 1);
      const double eps_ln2 = p->eps * kLn2;
      // float64 smooth potentials into tx, ty (f, g receive the full ones)
      f_from_beta<R>(st.px[q], st.mu64, p->N, eps_ln2, f, st.tx, s);
      f_from_beta<R>(st.py[q], st.nu64, p->M, eps_ln2, g, st.ty, s);
      rc = cost64(p, st.tx, st.ty, st.mu64, st.nu64, &err64, &w1, s);
      if (rc != FINOM_OK) return rc;
      if (err64 <= tol) break;
      // resume: clear the stop, continue with the phi half step of iteration l
      // (not below the float32 floor: then the float64 finish below)
      const double fr = std::max(0.1, std::min(0.97, 0.97 * tol / err64));
      if (loop_err * fr < kF32LoopFloor) break;
      st.tol = loop_err * fr;
      int32_t zero[2] = {0, 0};
      FINOM_CUDA(cudaMemcpyAsync(st.ctrl + 1, &zero[0], sizeof(int32_t), cudaMemcpyHostToDevice, s));
      FINOM_CUDA(cudaMemcpyAsync(st.ctrl + 4, &zero[1], sizeof(int32_t), cudaMemcpyHostToDevice, s));
      rc = launch_half<R>(half_args<R>(p, true, q), kHalfX, p, s);
      if (rc != FINOM_OK) return rc;
      st.launched = l + 1;
    }
    st.tol = sizeof(R) == sizeof(float) ? std::max(tol, kF32LoopFloor) : tol;
  }
  finom_result r32{};
  rc = solve_end<R>(p, f, g, &r32, s);
  if (rc != FINOM_OK) return rc;
  // a float32 solve whose float64 error is still above tol (a float32 floor
  // above it) is finished in float64, warm-started from its potentials, on a
  // float64 plan of the same meshes; iters counts both parts
  if (sizeof(R) == sizeof(float) && !r32.converged && r32.iters < maxit) {
    finom_plan_t p64 = nullptr;
    rc = finom_plan(p->x, p->N, p->y, p->M, p->eps, FINOM_F64, s, &p64);
    if (rc != FINOM_OK) return rc;
    finom_result r64{};
    rc = finom_solve(p64, u, v, tol, maxit - r32.iters, f, g, 1, &r64, s);
    finom_plan_destroy(p64);
    if (rc != FINOM_OK) return rc;
    r64.iters += r32.iters;
    r64.marginal_err_loop = r32.marginal_err_loop;
    r32 = r64;
  }
  if (res) *res = r32;
  return FINOM_OK;
}

bool bad_plan(finom_plan_t p) {
  if (!p) {
    set_error("null plan");
    return true;
  }
  return false;
}

// the calls for one problem refuse batch plans
bool batch_plan(finom_plan_t p, const char* what) {
  if (p && p->B > 0) {
    set_error(std::string(what) + ": a batch plan takes finom_solve_batch");
    return true;
  }
  return false;
}

}  // namespace
}  // namespace finom

using namespace finom;

namespace {

// Standalone products: one pass of the half-step kernel with the O frames
// at 0 (levels +-Z), which yields ln (K w) at every O point directly in
// float64 (the levels are exact pairs; see half.cuh).  The O side's own
// absorption of a log product is added afterwards.
template <class R>
finom_status kv_impl(finom_plan_t p, bool transpose, bool logmode, const double* a, const double* b,
                     double* out, cudaStream_t s) {
  finom_status rc = ensure_state<R>(p);
  if (rc != FINOM_OK) return rc;
  SolveState& st = p->st;
  const int64_t N = p->N, M = p->M;
  const int64_t nO = transpose ? M : N, nW = transpose ? N : M;
  const double* posO = transpose ? p->y : p->x;
  const double* posW = transpose ? p->x : p->y;
  const double scale = 1.0 / (p->eps * kLn2);
  // log products: the O side's absorption (added at the end) and the W
  // side's absorption (the weights); linear products: the weights are b
  const double* ao = logmode ? (transpose ? b : a) : nullptr;
  const double* bw = logmode ? (transpose ? a : b) : b;
  if (logmode) beta_set<R>(st.qw, posW, nW, scale, bw, scale, 0.0, s);
  else beta_lin<R>(st.qw, posW, nW, scale, bw, s);
  beta_set<R>(st.qo, posO, nO, scale, nullptr, 0.0, 0.0, s);
  const int o_is_x = transpose ? 0 : 1;
  rc = product<R>(p, o_is_x, out, logmode ? kHalfLog : kHalfLin, s);
  if (rc != FINOM_OK) return rc;
  if (logmode) add_scaled(out, ao, 1.0 / p->eps, nO, s);
  FINOM_CUDA(cudaGetLastError());
  return FINOM_OK;
}

finom_status kv_dispatch(finom_plan_t p, bool transpose, bool logmode, const double* a,
                         const double* b, double* out, void* stream) {
  if (bad_plan(p)) return FINOM_EINVAL;
  if (batch_plan(p, "kernel product")) return FINOM_ENOTSUP;
  if (!out || (!logmode && !b) || (logmode && (!a || !b))) {
    set_error("kernel product: null argument");
    return FINOM_EINVAL;
  }
  DeviceGuard dg(p->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (p->nd) return kv_nd(p, transpose, logmode, a, b, out, s);
  return p->prec == FINOM_F32_LOG ? kv_impl<float>(p, transpose, logmode, a, b, out, s)
                                  : kv_impl<double>(p, transpose, logmode, a, b, out, s);
}

}  // namespace

extern "C" {

int finom_version(void) { return 200; }

const char* finom_last_error(void) { return g_err.c_str(); }

finom_status finom_plan(const double* x, int64_t N, const double* y, int64_t M, double eps,
                        finom_precision prec, void* stream, finom_plan_t* out) {
  if (!out) {
    set_error("finom_plan: out is NULL");
    return FINOM_EINVAL;
  }
  *out = nullptr;
  if (!x || !y || N < 1 || M < 1 || !(eps > 0.0) || !std::isfinite(eps) ||
      (prec != FINOM_F64 && prec != FINOM_F32_LOG)) {
    set_error("finom_plan: need x, y non-null, N, M >= 1, eps > 0 finite, known precision");
    return FINOM_EINVAL;
  }
  if (N + M > (int64_t)INT32_MAX - 2 * kTile) {
    set_error("finom_plan: N + M too large");
    return FINOM_EINVAL;
  }
  finom_plan_s* p = new (std::nothrow) finom_plan_s();
  if (!p) return FINOM_ENOMEM;
  p->N = N;
  p->M = M;
  p->eps = eps;
  p->prec = prec;
  cudaGetDevice(&p->device);
  finom_status rc = build_plan(p, x, y, (cudaStream_t)stream);
  if (rc == FINOM_OK) rc = build_tiles_e(p, tune_pick(prec, N + M), (cudaStream_t)stream);
  if (rc != FINOM_OK) {
    free_plan(p);
    delete p;
    return rc;
  }
  *out = p;
  return FINOM_OK;
}

finom_status finom_plan_2d(const double* x1, const double* x2, int64_t N, const double* y1,
                           const double* y2, int64_t M, double eps, finom_precision prec,
                           void* stream, finom_plan_t* out) {
  if (!out) {
    set_error("finom_plan_2d: out is NULL");
    return FINOM_EINVAL;
  }
  *out = nullptr;
  if (!x1 || !x2 || !y1 || !y2 || N < 1 || M < 1 || !(eps > 0.0) || !std::isfinite(eps) ||
      (prec != FINOM_F64 && prec != FINOM_F32_LOG)) {
    set_error("finom_plan_2d: need x1, x2, y1, y2 non-null, N, M >= 1, eps > 0 finite, known precision");
    return FINOM_EINVAL;
  }
  if (N > (int64_t)INT32_MAX / 4 || M > (int64_t)INT32_MAX / 4 || N * M > ((int64_t)1 << 31)) {
    set_error("finom_plan_2d: grid too large (N*M <= 2^31 points per grid)");
    return FINOM_EINVAL;
  }
  // the d = 2 case of a d-dimensional plan: axis 0 merges x1 with x2, axis 1
  // y1 with y2; grid points (k, i) at k + N i are axis 0 fastest
  const int64_t n[2] = {N, M};
  const double* xs[2] = {x1, y1};
  const double* ys[2] = {x2, y2};
  return finom_plan_nd(2, n, xs, ys, eps, prec, stream, out);
}

finom_status finom_plan_nd(int32_t d, const int64_t* n, const double* const* xs, const double* const* ys,
                           double eps, finom_precision prec, void* stream, finom_plan_t* out) {
  if (!out) {
    set_error("finom_plan_nd: out is NULL");
    return FINOM_EINVAL;
  }
  *out = nullptr;
  if (d < 1 || d > finom_plan_s::kMaxDim || !n || !xs || !ys || !(eps > 0.0) || !std::isfinite(eps) ||
      (prec != FINOM_F64 && prec != FINOM_F32_LOG)) {
    set_error("finom_plan_nd: need 1 <= d <= 8, n, xs, ys non-null, eps > 0 finite, known precision");
    return FINOM_EINVAL;
  }
  int64_t G = 1;
  for (int k = 0; k < d; ++k) {
    if (n[k] < 1 || !xs[k] || !ys[k] || 2 * n[k] > (int64_t)INT32_MAX / 2) {
      set_error("finom_plan_nd: every axis needs n[k] >= 1 and non-null node arrays");
      return FINOM_EINVAL;
    }
    G *= n[k];
    if (G > (int64_t)INT32_MAX) {
      set_error("finom_plan_nd: the grid must have fewer than 2^31 points");
      return FINOM_EINVAL;
    }
  }
  finom_plan_s* p = new (std::nothrow) finom_plan_s();
  if (!p) return FINOM_ENOMEM;
  p->eps = eps;
  p->prec = prec;
  cudaGetDevice(&p->device);
  finom_status rc = plan_nd_build(p, d, n, xs, ys, (cudaStream_t)stream);
  if (rc != FINOM_OK) {
    plan_nd_free(p);
    delete p;
    return rc;
  }
  *out = p;
  return FINOM_OK;
}

finom_status finom_plan_axes(finom_plan_t plan, int32_t* d, int64_t* n) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (!plan->nd) {
    set_error("finom_plan_axes: not a plan of finom_plan_nd");
    return FINOM_ENOTSUP;
  }
  if (d) *d = plan->dim;
  if (n)
    for (int k = 0; k < plan->dim; ++k) n[k] = plan->nd_n[k];
  return FINOM_OK;
}

finom_status finom_plan_destroy(finom_plan_t plan) {
  if (!plan) return FINOM_OK;
  DeviceGuard dg(plan->device);
  cudaDeviceSynchronize();
  free_state(plan);
  free_plan(plan);
  plan_nd_free(plan);
  plan_batch_free(plan);
  delete plan;
  return FINOM_OK;
}

finom_status finom_plan_batch(const double* x, const int64_t* offx, const double* y, const int64_t* offy,
                              int64_t B, const double* eps, finom_precision prec, void* stream,
                              finom_plan_t* out) {
  return finom_plan_batch_elems(x, offx, y, offy, B, eps, prec, 0, stream, out);
}

finom_status finom_plan_batch_elems(const double* x, const int64_t* offx, const double* y, const int64_t* offy,
                                    int64_t B, const double* eps, finom_precision prec, int32_t elems,
                                    void* stream, finom_plan_t* out) {
  if (!out) {
    set_error("finom_plan_batch: out is NULL");
    return FINOM_EINVAL;
  }
  *out = nullptr;
  if (elems == 0) elems = tune_pick_batch(prec);
  if (!tile_kind_ok(elems)) {
    set_error("finom_plan_batch: tile kind must be 1, 2, 4 or 8 points per thread, or -1 (64-point tiles)");
    return FINOM_EINVAL;
  }
  if (!x || !y || !offx || !offy || !eps || B < 1 || B > (int64_t)1 << 24 ||
      (prec != FINOM_F64 && prec != FINOM_F32_LOG)) {
    set_error("finom_plan_batch: need x, y, offx, offy, eps non-null, 1 <= B <= 2^24, known precision");
    return FINOM_EINVAL;
  }
  if (offx[0] != 0 || offy[0] != 0) {
    set_error("finom_plan_batch: offx[0] and offy[0] must be 0");
    return FINOM_EINVAL;
  }
  int64_t tiles = 0;
  for (int64_t b = 0; b < B; ++b) {
    const int64_t n = offx[b + 1] - offx[b], m = offy[b + 1] - offy[b];
    if (n < 1 || m < 1 || !(eps[b] > 0.0) || !std::isfinite(eps[b])) {
      set_error("finom_plan_batch: instance " + std::to_string((long long)b) +
                " needs at least one x and one y point and eps > 0 finite");
      return FINOM_EINVAL;
    }
    tiles += (n + m + kTile - 1) / kTile;
  }
  if (tiles * kTile > (int64_t)INT32_MAX || offx[B] > (int64_t)INT32_MAX || offy[B] > (int64_t)INT32_MAX) {
    set_error("finom_plan_batch: batch too large");
    return FINOM_EINVAL;
  }
  finom_plan_s* p = new (std::nothrow) finom_plan_s();
  if (!p) return FINOM_ENOMEM;
  p->btile = tile_points(elems);
  p->elems = elems;
  p->eps = eps[0];
  p->prec = prec;
  cudaGetDevice(&p->device);
  finom_status rc = plan_batch_build(p, x, offx, y, offy, B, eps, (cudaStream_t)stream);
  if (rc != FINOM_OK) {
    free_plan(p);
    plan_batch_free(p);
    delete p;
    return rc;
  }
  *out = p;
  return FINOM_OK;
}

finom_status finom_plan_set_elems(finom_plan_t plan, int32_t elems, void* stream) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (plan->dim != 1 || plan->nd || plan->B > 0) {
    set_error("finom_plan_set_elems: only 1D single-problem plans choose their tile size");
    return FINOM_ENOTSUP;
  }
  if (elems == plan->elems) return FINOM_OK;
  DeviceGuard dg(plan->device);
  FINOM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  free_state(plan);   // the scan scratch is sized by the tile count
  return build_tiles_e(plan, elems, (cudaStream_t)stream);
}

finom_status finom_plan_elems(finom_plan_t plan, int32_t* elems, int64_t* tiles) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (elems) *elems = plan->elems;
  if (tiles) *tiles = plan->Ce;
  return FINOM_OK;
}

finom_status finom_plan_instances(finom_plan_t plan, int64_t* B) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (B) *B = plan->B;
  return FINOM_OK;
}

finom_status finom_solve_batch_begin(finom_plan_t plan, const double* u, const double* v, double tol,
                                     int64_t maxit, void* stream) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (plan->B == 0 || !u || !v || !(tol >= 0.0) || maxit < 0) {
    set_error("finom_solve_batch_begin: need a batch plan, u, v non-null, tol >= 0, maxit >= 0");
    return FINOM_EINVAL;
  }
  DeviceGuard dg(plan->device);
  return solve_batch_begin(plan, u, v, tol, maxit, (cudaStream_t)stream);
}

finom_status finom_solve_batch_step(finom_plan_t plan, int64_t iterations, void* stream) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (plan->B == 0 || !plan->st.active || iterations < 0) {
    set_error("finom_solve_batch_step: no batch solve in progress (finom_solve_batch_begin first)");
    return FINOM_EINVAL;
  }
  DeviceGuard dg(plan->device);
  return solve_batch_step(plan, iterations, (cudaStream_t)stream);
}

finom_status finom_solve_batch_end(finom_plan_t plan, double* f, double* g, finom_result* res, void* stream) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (plan->B == 0 || !plan->st.active || !f || !g || !res) {
    set_error("finom_solve_batch_end: no batch solve in progress or null output");
    return FINOM_EINVAL;
  }
  DeviceGuard dg(plan->device);
  return solve_batch_end(plan, f, g, res, (cudaStream_t)stream);
}

finom_status finom_solve_batch(finom_plan_t plan, const double* u, const double* v, double tol,
                               int64_t maxit, double* f, double* g, finom_result* res, void* stream) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (plan->B == 0) {
    set_error("finom_solve_batch: not a batch plan");
    return FINOM_EINVAL;
  }
  if (!u || !v || !f || !g || !res || !(tol >= 0.0) || maxit < 0) {
    set_error("finom_solve_batch: need u, v, f, g, res non-null, tol >= 0, maxit >= 0");
    return FINOM_EINVAL;
  }
  DeviceGuard dg(plan->device);
  finom_status rc = solve_batch(plan, u, v, tol, maxit, f, g, res, (cudaStream_t)stream);
  if (rc != FINOM_OK)
    for (int64_t b = 0; b < plan->B; ++b) res[b].status = rc;
  return rc;
}

finom_status finom_plan_shape(finom_plan_t plan, int32_t* dim, int64_t* N, int64_t* M) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (dim) *dim = plan->dim;
  if (plan->nd) {
    if (N) *N = plan->nd_n[0];
    if (M) *M = plan->nd_G / plan->nd_n[0];
    return FINOM_OK;
  }
  if (N) *N = plan->N;
  if (M) *M = plan->M;
  return FINOM_OK;
}

finom_status finom_plan_info(finom_plan_t plan, int64_t* N, int64_t* M, double* eps,
                             int32_t* precision) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (N) *N = plan->N;
  if (M) *M = plan->M;
  if (eps) *eps = plan->eps;
  if (precision) *precision = (int32_t)plan->prec;
  return FINOM_OK;
}

finom_status finom_dividing_index(finom_plan_t plan, int32_t* zeta, int32_t* zetaT, void* stream) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (batch_plan(plan, "finom_dividing_index")) return FINOM_ENOTSUP;
  if (plan->dim != 1 || plan->nd) {
    set_error("finom_dividing_index: a grid plan has one dividing index per axis; use 1D plans of the axes");
    return FINOM_ENOTSUP;
  }
  DeviceGuard dg(plan->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (zeta) FINOM_CUDA(cudaMemcpyAsync(zeta, plan->zeta, sizeof(int32_t) * plan->N, cudaMemcpyDeviceToDevice, s));
  if (zetaT) FINOM_CUDA(cudaMemcpyAsync(zetaT, plan->zetaT, sizeof(int32_t) * plan->M, cudaMemcpyDeviceToDevice, s));
  return FINOM_OK;
}


finom_status finom_kv(finom_plan_t plan, const double* v, double* out, void* stream) {
  return kv_dispatch(plan, false, false, nullptr, v, out, stream);
}

finom_status finom_ktu(finom_plan_t plan, const double* u, double* out, void* stream) {
  return kv_dispatch(plan, true, false, nullptr, u, out, stream);
}

finom_status finom_kv_log(finom_plan_t plan, const double* a, const double* b, double* out,
                          void* stream) {
  return kv_dispatch(plan, false, true, a, b, out, stream);
}

finom_status finom_ktu_log(finom_plan_t plan, const double* a, const double* b, double* out,
                           void* stream) {
  return kv_dispatch(plan, true, true, a, b, out, stream);
}

finom_status finom_solve(finom_plan_t plan, const double* u, const double* v, double tol,
                         int64_t maxit, double* f, double* g, int32_t warm, finom_result* res,
                         void* stream) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (batch_plan(plan, "finom_solve")) return FINOM_ENOTSUP;
  if (!u || !v || !f || !g || !(tol >= 0.0) || maxit < 0) {
    set_error("finom_solve: need u, v, f, g non-null, tol >= 0, maxit >= 0");
    return FINOM_EINVAL;
  }
  DeviceGuard dg(plan->device);
  if (plan->nd) {
    finom_status rc = solve_nd(plan, u, v, tol, maxit, f, g, warm, res, (cudaStream_t)stream);
    if (res && rc != FINOM_OK) res->status = rc;
    return rc;
  }
  finom_status rc = plan->prec == FINOM_F32_LOG
                        ? solve_blocking<float>(plan, u, v, tol, maxit, f, g, warm, res, (cudaStream_t)stream)
                        : solve_blocking<double>(plan, u, v, tol, maxit, f, g, warm, res, (cudaStream_t)stream);
  if (res && rc != FINOM_OK) res->status = rc;
  return rc;
}

finom_status finom_solve_trace(finom_plan_t plan, const double* u, const double* v, int64_t maxit, int64_t every,
                               double* err, double* ms, int64_t* n, void* stream) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (batch_plan(plan, "finom_solve_trace")) return FINOM_ENOTSUP;
  if (!u || !v || !err || !ms || !n || maxit < 1 || every < 1) {
    set_error("finom_solve_trace: need u, v, err, ms, n non-null, maxit >= 1, every >= 1");
    return FINOM_EINVAL;
  }
  *n = 0;
  DeviceGuard dg(plan->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t K = (maxit + every - 1) / every;
  double* dtrace = nullptr;
  FINOM_CUDA(cudaMallocAsync(&dtrace, sizeof(double) * K, s));
  std::vector<cudaEvent_t> ev(K + 1, nullptr);
  finom_status rc = FINOM_OK;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "cudaEventCreate");
  // the loop without a stopping tolerance: the loop-head error of every
  // iteration is the one the kernels leave in the plan's control block
  if (rc == FINOM_OK) rc = finom_solve_begin(plan, u, v, 0.0, maxit, nullptr, nullptr, stream);
  if (rc == FINOM_OK) cudaEventRecord(ev[0], s);
  int64_t k = 0, done = 1;   // iterations launched (begin launched iteration 0)
  for (; rc == FINOM_OK && k < K; ++k) {
    const int64_t chunk = std::min(every, maxit - done);
    if (chunk > 0) rc = finom_solve_step(plan, chunk, stream);
    done += std::max<int64_t>(chunk, 0);
    if (rc != FINOM_OK) break;
    if (cudaMemcpyAsync(dtrace + k, plan->st.scal, sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      rc = cuda_fail(cudaGetLastError(), "trace copy");
    cudaEventRecord(ev[k + 1], s);
  }
  if (rc == FINOM_OK) {
    std::vector<double> h(k);
    if (k > 0 && cudaMemcpyAsync(h.data(), dtrace, sizeof(double) * k, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      rc = cuda_fail(cudaGetLastError(), "trace read");
    if (rc == FINOM_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "trace sync");
    for (int64_t i = 0; rc == FINOM_OK && i < k; ++i) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[0], ev[i + 1]);
      err[i] = h[i];
      ms[i] = t;
    }
    *n = k;
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  cudaFreeAsync(dtrace, s);
  plan->st.active = false;
  return rc;
}

finom_status finom_solve_eps_scaling(finom_plan_t plan, const double* u, const double* v, double tol,
                                     int64_t maxit, double eps0, double factor, double tol_stage, double* f,
                                     double* g, finom_result* res, void* stream) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (batch_plan(plan, "finom_solve_eps_scaling")) return FINOM_ENOTSUP;
  if (!u || !v || !f || !g || !res || !(tol >= 0.0) || maxit < 0 || !(eps0 > plan->eps) || !std::isfinite(eps0) ||
      !(factor > 0.0 && factor < 1.0) || !(tol_stage >= tol)) {
    set_error("finom_solve_eps_scaling: need u, v, f, g, res non-null, tol >= 0, maxit >= 0, eps0 > eps finite, "
              "0 < factor < 1, tol_stage >= tol");
    return FINOM_EINVAL;
  }
  DeviceGuard dg(plan->device);
  int64_t done = 0;
  int32_t warm = 0;
  for (double e = eps0; e > plan->eps * (1.0 + 1e-12) && done < maxit; e *= factor) {
    // the same meshes at the larger eps: a plan of its own, warm-started from
    // the potentials of the previous stage
    finom_plan_t q = nullptr;
    finom_status rc;
    if (plan->nd) {
      const double* xs[finom_plan_s::kMaxDim];
      const double* ys[finom_plan_s::kMaxDim];
      for (int k = 0; k < plan->dim; ++k) {
        xs[k] = plan->nd_ax[k]->x;
        ys[k] = plan->nd_ax[k]->y;
      }
      rc = finom_plan_nd(plan->dim, plan->nd_n, xs, ys, e, plan->prec, stream, &q);
    } else {
      rc = finom_plan(plan->x, plan->N, plan->y, plan->M, e, plan->prec, stream, &q);
    }
    finom_result r{};
    if (rc == FINOM_OK) rc = finom_solve(q, u, v, tol_stage, maxit - done, f, g, warm, &r, stream);
    finom_plan_destroy(q);
    if (rc != FINOM_OK) {
      res->status = rc;
      return rc;
    }
    done += r.iters;
    warm = 1;
  }
  finom_status rc = finom_solve(plan, u, v, tol, maxit - done, f, g, warm, res, stream);
  res->iters += done;
  return rc;
}

finom_status finom_solve_begin(finom_plan_t plan, const double* u, const double* v, double tol,
                               int64_t maxit, const double* f0, const double* g0, void* stream) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (batch_plan(plan, "finom_solve_begin")) return FINOM_ENOTSUP;
  if (!u || !v || !(tol >= 0.0) || maxit < 0) {
    set_error("finom_solve_begin: need u, v non-null, tol >= 0, maxit >= 0");
    return FINOM_EINVAL;
  }
  DeviceGuard dg(plan->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (plan->nd) return solve_nd_begin(plan, u, v, tol, maxit, f0, g0, s);
  return plan->prec == FINOM_F32_LOG ? solve_begin<float>(plan, u, v, tol, maxit, f0, g0, s)
                                     : solve_begin<double>(plan, u, v, tol, maxit, f0, g0, s);
}

finom_status finom_solve_step(finom_plan_t plan, int64_t iterations, void* stream) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (batch_plan(plan, "finom_solve_step")) return FINOM_ENOTSUP;
  if (!plan->st.active || iterations < 0) {
    set_error("finom_solve_step: no solve in progress (finom_solve_begin first) or negative count");
    return FINOM_EINVAL;
  }
  DeviceGuard dg(plan->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (plan->nd) return solve_nd_step(plan, iterations, s);
  return plan->prec == FINOM_F32_LOG ? solve_step<float>(plan, iterations, s)
                                     : solve_step<double>(plan, iterations, s);
}

finom_status finom_solve_poll(finom_plan_t plan, int32_t* done, int64_t* iters, void* stream) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (plan->B > 0) {   // batches: done = every instance retired, iters = iterations launched
    if (!plan->st.ready) {
      set_error("finom_solve_poll: no solve state");
      return FINOM_EINVAL;
    }
    DeviceGuard dg(plan->device);
    int32_t h[8];
    FINOM_CUDA(cudaMemcpyAsync(h, plan->st.ctrl, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    FINOM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (done) *done = h[1];
    if (iters) *iters = plan->st.launched;
    return FINOM_OK;
  }
  if (!plan->st.ready) {
    set_error("finom_solve_poll: no solve state");
    return FINOM_EINVAL;
  }
  DeviceGuard dg(plan->device);
  return solve_poll(plan, (cudaStream_t)stream, done, iters);
}

finom_status finom_solve_end(finom_plan_t plan, double* f, double* g, finom_result* res,
                             void* stream) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (batch_plan(plan, "finom_solve_end")) return FINOM_ENOTSUP;
  if (!plan->st.active || !f || !g) {
    set_error("finom_solve_end: no solve in progress or null output");
    return FINOM_EINVAL;
  }
  DeviceGuard dg(plan->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (plan->nd) return solve_nd_end(plan, f, g, res, s);
  return plan->prec == FINOM_F32_LOG ? solve_end<float>(plan, f, g, res, s)
                                     : solve_end<double>(plan, f, g, res, s);
}

finom_status finom_cost(finom_plan_t plan, const double* u, const double* v, const double* f,
                        const double* g, double* w1, double* err, void* stream) {
  if (bad_plan(plan)) return FINOM_EINVAL;
  if (batch_plan(plan, "finom_cost")) return FINOM_ENOTSUP;
  if (!u || !v || !f || !g || !w1 || !err) {
    set_error("finom_cost: null argument");
    return FINOM_EINVAL;
  }
  DeviceGuard dg(plan->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (plan->nd) return cost_nd(plan, u, v, f, g, w1, err, s);
  finom_status rc = plan->prec == FINOM_F32_LOG ? ensure_state<float>(plan) : ensure_state<double>(plan);
  if (rc != FINOM_OK) return rc;
  SolveState& st = plan->st;
  const double scale = 1.0 / (plan->eps * kLn2);
  // masses as given (not renormalised) and smooth potentials P = f/(eps ln2) - log2 u
  FINOM_CUDA(cudaMemcpyAsync(st.mu64, u, sizeof(double) * plan->N, cudaMemcpyDeviceToDevice, s));
  FINOM_CUDA(cudaMemcpyAsync(st.nu64, v, sizeof(double) * plan->M, cudaMemcpyDeviceToDevice, s));
  pot_from_f(f, st.mu64, plan->N, scale, st.tx, s);
  pot_from_f(g, st.nu64, plan->M, scale, st.ty, s);
  st.active = false;
  return cost64(plan, st.tx, st.ty, st.mu64, st.nu64, err, w1, s);
}

}  // extern "C"
