// 2D FINOM (Sec. 3, Algorithm 2) with the log-domain stabilisation of
// Appendix A, on two tensor-product grids
//     grid 1: (x1_k, y1_i), k < N, i < M      grid 2: (x2_l, y2_j), l < N, j < M
// with cost |x1_k - x2_l| + |y1_i - y2_j|, so that K = K_y (x) K_x
// (eq. 2d-kron).  Each product K' psi (eq. K'bpsi) is two batches of 1D
// stabilised products on the axis plans (x1 vs x2, y1 vs y2):
//   K' psi    : columns j of grid 2 along x (first pass, log2 Q),
//               then rows k of grid 1 along y (second pass, division);
//   K'^T phi  : rows k of grid 1 along y (first pass), then columns j of
//               grid 2 along x (second pass, division and the marginal error).
// The first pass has no output-side absorption (a_x = 0 in Appendix A); its
// float32 frames are taken from the weight side instead, and it writes log2 Q
// as a float-float pair.  Grid-1 data live row-major (i + M k), grid-2 data
// column-major (l + N j), so that every pass reads and writes whole lines;
// only the intermediate Q is written across lines.  The C ABI takes and
// returns column-major grids (vec() of the paper).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "apply.cuh"
#include "finom_internal.h"

namespace finom {

template <class R>
finom_status launch_apply(const ApplyArgs<R>& a, bool agg_only, cudaStream_t s);
template <class R>
void conv_weights_log(const double*, int64_t, double, void*, void*, cudaStream_t);
template <class R>
void conv_weights_lin(const double*, int64_t, void*, void*, cudaStream_t);
template <class R>
void fill_pot(void*, int64_t, double, cudaStream_t);
template <class R>
void conv_pot_from_f(const double*, const double*, int64_t, double, void*, cudaStream_t);
template <class R>
void conv_f_from_pot(const void*, const double*, int64_t, double, double*, double*, cudaStream_t);
template <class R>
finom_status normalise_masses(const double*, int64_t, void*, double*, double*, int*, double*,
                              cudaStream_t);
template <class R>
void frame_from_log(const double*, int64_t, void*, cudaStream_t);
template <class T>
void transpose(const T* src, int64_t rows, int64_t cols, T* dst, cudaStream_t s);
void fill_d(double*, int64_t, double, cudaStream_t);
void combine_passes(const double*, const double*, double, int64_t, int, double*, cudaStream_t);
void dot_pos(const double*, const double*, int64_t, double*, cudaStream_t);

namespace {

constexpr double kLn2 = 0.69314718055994530942;

template <class R>
using PotT = typename Tr<R>::Pot;
template <class R>
using MassT = typename Tr<R>::Mass;

int64_t gN(const finom_plan_s* p) { return p->ax->N; }
int64_t gM(const finom_plan_s* p) { return p->ay->N; }

// tiles of all lines of the largest pass
int64_t max_tiles(const finom_plan_s* p) {
  return std::max(p->ax->C * gM(p), p->ay->C * gN(p));
}

template <class R>
finom_status ensure_state2d(finom_plan_s* p) {
  SolveState& st = p->st;
  if (st.ready) return FINOM_OK;
  const int64_t NM = gN(p) * gM(p), T = max_tiles(p);
  const size_t ps = sizeof(PotT<R>), ms = sizeof(MassT<R>);
  for (int q = 0; q < 2; ++q) {
    FINOM_CUDA(cudaMalloc(&st.px[q], ps * NM));
    FINOM_CUDA(cudaMalloc(&st.py[q], ps * NM));
  }
  FINOM_CUDA(cudaMalloc(&st.mu, ms * NM));
  FINOM_CUDA(cudaMalloc(&st.nu, ms * NM));
  FINOM_CUDA(cudaMalloc(&st.mu64, sizeof(double) * NM));
  FINOM_CUDA(cudaMalloc(&st.nu64, sizeof(double) * NM));
  FINOM_CUDA(cudaMalloc(&st.tx, sizeof(double) * std::max<int64_t>(NM, 512)));
  FINOM_CUDA(cudaMalloc(&st.ty, sizeof(double) * std::max<int64_t>(NM, 512)));
  FINOM_CUDA(cudaMalloc(&st.t2, sizeof(double) * NM));
  FINOM_CUDA(cudaMalloc(&st.z, sizeof(double) * 2 * NM));
  FINOM_CUDA(cudaMalloc(&st.aggs, sizeof(R) * 6 * T));
  FINOM_CUDA(cudaMalloc(&st.carries, sizeof(R) * 4 * T));
  FINOM_CUDA(cudaMalloc(&st.part, sizeof(double) * T));
  FINOM_CUDA(cudaMalloc(&st.scal, sizeof(double) * 520));
  FINOM_CUDA(cudaMalloc(&st.ctrl, sizeof(int32_t) * 8));
  FINOM_CUDA(cudaMalloc(&st.bad, sizeof(int)));
  FINOM_CUDA(cudaMalloc(&st.qo, ps * NM));
  FINOM_CUDA(cudaMalloc(&st.qom, ms * NM));
  FINOM_CUDA(cudaMalloc(&st.qw, ps * NM));
  FINOM_CUDA(cudaMalloc(&st.qwm, ms * NM));
  FINOM_CUDA(cudaMalloc(&st.q2, ps * NM));
  FINOM_CUDA(cudaMemset(st.ctrl, 0, sizeof(int32_t) * 8));
  FINOM_CUDA(cudaMemset(st.scal, 0, sizeof(double) * 520));
  FINOM_CUDA(cudaMemset(st.part, 0, sizeof(double) * T));
  FINOM_CUDA(cudaStreamCreateWithFlags(&st.stream, cudaStreamNonBlocking));
  st.ready = true;
  return FINOM_OK;
}

// arguments of one line batch along axis plan ax (lines x tiles CTAs)
template <class R>
ApplyArgs<R> line_args(finom_plan_s* p, finom_plan_s* axp, int64_t lines, int o_is_x) {
  SolveState& st = p->st;
  ApplyArgs<R> a{};
  a.tbits = axp->tbits;
  a.gap = (const R*)axp->gap;
  a.tile_x0 = axp->tile_x0;
  a.L = axp->L;
  a.C = (int)axp->C;
  a.lines = (int)lines;
  a.o_is_x = o_is_x;
  a.fw = axp->fw[o_is_x];
  a.o_es = 1;
  a.w_es = 1;
  a.agg_out = (R*)st.aggs;
  a.carry_out = (R*)st.carries;
  a.carry_in = nullptr;
  a.part = st.part;
  a.scal = st.scal;
  a.ctrl = st.ctrl;
  a.tol = st.tol;
  a.maxit = st.maxit;
  return a;
}

// one pass; lines longer than a tile get their carries from a map pass first
template <class R>
finom_status run_pass(ApplyArgs<R> a, cudaStream_t s) {
  if (a.C > 1) {
    finom_status rc = launch_apply<R>(a, true, s);
    if (rc != FINOM_OK) return rc;
    a.carry_in = a.carry_out;
  }
  return launch_apply<R>(a, false, s);
}

// K'^T phi, first pass: rows k of grid 1 along y (W = y1 with phi, O = y2),
// log2 Q'(k, j) written along the line (k M + j): contiguous stores; the
// second pass reads it across lines
template <class R>
ApplyArgs<R> pass_t1(finom_plan_s* p, int q) {
  SolveState& st = p->st;
  const int64_t N = gN(p), M = gM(p);
  ApplyArgs<R> a = line_args<R>(p, p->ay, N, 0);
  a.pW = (const PotT<R>*)st.px[q];
  a.mW = (const MassT<R>*)st.mu;
  a.w_ls = M;
  a.q_out = (PotT<R>*)st.q2;
  a.q_ls = M;
  a.q_es = 1;
  a.flags = kMode2Inner;
  return a;
}

// K'^T phi, second pass: columns j of grid 2 along x (O = x2 with psi, W = x1
// with Q'): psi <- v / (K^T phi) and the marginal error of the loop head
template <class R>
ApplyArgs<R> pass_t2(finom_plan_s* p, int q) {
  SolveState& st = p->st;
  const int64_t N = gN(p), M = gM(p);
  ApplyArgs<R> a = line_args<R>(p, p->ax, M, 0);
  a.pO = (const PotT<R>*)st.py[q];
  a.mO = (const MassT<R>*)st.nu;
  a.o_ls = N;
  a.pO_out = (PotT<R>*)st.py[1 - q];
  a.pW = (const PotT<R>*)st.q2;
  a.w_ls = 1;
  a.w_es = M;
  a.flags = kMode2HalfB;
  return a;
}

// K' psi, first pass: columns j of grid 2 along x (W = x2 with psi, O = x1),
// log2 Q(k, j) written along the line (j N + k)
template <class R>
ApplyArgs<R> pass_a1(finom_plan_s* p, int q) {
  SolveState& st = p->st;
  const int64_t N = gN(p), M = gM(p);
  ApplyArgs<R> a = line_args<R>(p, p->ax, M, 1);
  a.pW = (const PotT<R>*)st.py[1 - q];
  a.mW = (const MassT<R>*)st.nu;
  a.w_ls = N;
  a.q_out = (PotT<R>*)st.q2;
  a.q_ls = N;
  a.q_es = 1;
  a.flags = kMode2Inner;
  return a;
}

// K' psi, second pass: rows k of grid 1 along y (O = y1 with phi, W = y2 with
// Q): phi <- u / (K psi); ends the iteration
template <class R>
ApplyArgs<R> pass_a2(finom_plan_s* p, int q) {
  SolveState& st = p->st;
  const int64_t N = gN(p), M = gM(p);
  ApplyArgs<R> a = line_args<R>(p, p->ay, N, 1);
  a.pO = (const PotT<R>*)st.px[q];
  a.mO = (const MassT<R>*)st.mu;
  a.o_ls = M;
  a.pO_out = (PotT<R>*)st.px[1 - q];
  a.pW = (const PotT<R>*)st.q2;
  a.w_ls = 1;
  a.w_es = N;
  a.flags = kMode2HalfA;
  return a;
}

template <class R>
finom_status half_phi(finom_plan_s* p, int q, cudaStream_t s) {
  finom_status rc = run_pass<R>(pass_a1<R>(p, q), s);
  if (rc != FINOM_OK) return rc;
  return run_pass<R>(pass_a2<R>(p, q), s);
}

template <class R>
finom_status iteration2d(finom_plan_s* p, int q, cudaStream_t s) {
  finom_status rc = run_pass<R>(pass_t1<R>(p, q), s);
  if (rc != FINOM_OK) return rc;
  rc = run_pass<R>(pass_t2<R>(p, q), s);
  if (rc != FINOM_OK) return rc;
  return half_phi<R>(p, q, s);
}

// graph of 2 * pairs iterations starting at an odd iteration (q = 1, 0, 1, ...)
template <class R>
finom_status build_body2d(finom_plan_s* p, int pairs, cudaGraphExec_t* out) {
  SolveState& st = p->st;
  if (*out) {
    cudaGraphExecDestroy(*out);
    *out = nullptr;
  }
  cudaGraph_t g = nullptr;
  FINOM_CUDA(cudaStreamBeginCapture(st.stream, cudaStreamCaptureModeThreadLocal));
  finom_status rc = FINOM_OK;
  for (int k = 0; k < pairs && rc == FINOM_OK; ++k) {
    rc = iteration2d<R>(p, 1, st.stream);
    if (rc == FINOM_OK) rc = iteration2d<R>(p, 0, st.stream);
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
finom_status begin2d(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                     const double* f0, const double* g0, cudaStream_t s) {
  finom_status rc = ensure_state2d<R>(p);
  if (rc != FINOM_OK) return rc;
  SolveState& st = p->st;
  const int64_t N = gN(p), M = gM(p), NM = N * M;
  // grid 1 masses: normalised column-major, then row-major copies
  rc = normalise_masses<R>(u, NM, st.qom, st.t2, st.tx, st.bad, nullptr, s);
  if (rc != FINOM_OK) return rc;
  transpose<MassT<R>>((const MassT<R>*)st.qom, N, M, (MassT<R>*)st.mu, s);
  transpose<double>(st.t2, N, M, st.mu64, s);
  rc = normalise_masses<R>(v, NM, st.nu, st.nu64, st.ty, st.bad, nullptr, s);
  if (rc != FINOM_OK) return rc;
  const double scale = 1.0 / (p->eps * kLn2);
  st.warm = (f0 != nullptr && g0 != nullptr);
  if (st.warm) {
    transpose<double>(f0, N, M, st.tx, s);
    conv_pot_from_f<R>(st.tx, st.mu64, NM, scale, st.px[0], s);
    conv_pot_from_f<R>(g0, st.nu64, NM, scale, st.py[0], s);
  } else {
    fill_pot<R>(st.px[0], NM, 0.0, s);
    fill_pot<R>(st.py[0], NM, 0.0, s);
  }
  FINOM_CUDA(cudaMemsetAsync(st.ctrl, 0, sizeof(int32_t) * 8, s));
  FINOM_CUDA(cudaMemsetAsync(st.scal, 0, sizeof(double) * 8, s));
  st.tol = tol;
  st.maxit = maxit;
  st.launched = 0;
  st.active = true;
  // iteration 0: the first K^T phi uses Phi = 1/(NM) (Algorithm 2) and
  // checks against Psi = 1/(NM)
  ApplyArgs<R> t1 = pass_t1<R>(p, 0);
  ApplyArgs<R> t2 = pass_t2<R>(p, 0);
  if (!st.warm) {
    t1.w_uniform = (R)(1.0 / (double)NM);
    t2.o_scale = (R)(1.0 / (double)NM);
  }
  rc = run_pass<R>(t1, s);
  if (rc != FINOM_OK) return rc;
  if (maxit == 0) {   // only the loop-head check of l = 0
    t2.flags = kMode2Check;
    return run_pass<R>(t2, s);
  }
  rc = run_pass<R>(t2, s);
  if (rc != FINOM_OK) return rc;
  rc = half_phi<R>(p, 0, s);
  if (rc != FINOM_OK) return rc;
  st.launched = 1;
  return FINOM_OK;
}

template <class R>
finom_status step2d(finom_plan_s* p, int64_t iters, cudaStream_t s) {
  SolveState& st = p->st;
  for (int64_t k = 0; k < iters;) {
    if ((st.launched & 1) && iters - k >= kChunkIters) {   // graphs of kChunkIters iterations
      if (!st.chunk || st.chunk_tol != st.tol || st.chunk_maxit != st.maxit) {
        finom_status rc = build_body2d<R>(p, kChunkIters / 2, &st.chunk);
        if (rc != FINOM_OK) return rc;
        st.chunk_tol = st.tol;
        st.chunk_maxit = st.maxit;
      }
      FINOM_CUDA(cudaGraphLaunch(st.chunk, s));
      st.launched += kChunkIters;
      k += kChunkIters;
      continue;
    }
    finom_status rc = iteration2d<R>(p, (int)(st.launched & 1), s);
    if (rc != FINOM_OK) return rc;
    ++st.launched;
    ++k;
  }
  return FINOM_OK;
}

finom_status poll(finom_plan_s* p, cudaStream_t s, int32_t* done, int64_t* iters, double* loop_err) {
  int32_t h[8];
  FINOM_CUDA(cudaMemcpyAsync(h, p->st.ctrl, sizeof(h), cudaMemcpyDeviceToHost, s));
  if (loop_err) FINOM_CUDA(cudaMemcpyAsync(loop_err, p->st.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  if (done) *done = h[1];
  if (iters) *iters = h[1] ? h[3] : h[2];
  return FINOM_OK;
}

// f (column-major, cost units) and the float64 smooth potentials of the
// state with parity q: tx = grid 1 (row-major), ty = grid 2 (column-major)
template <class R>
void export_potentials(finom_plan_s* p, int q, double* f, double* g, double* dual2, cudaStream_t s) {
  SolveState& st = p->st;
  const int64_t N = gN(p), M = gM(p), NM = N * M;
  const double eps_ln2 = p->eps * kLn2;
  conv_f_from_pot<R>(st.px[q], st.mu64, NM, eps_ln2, st.t2, st.tx, s);
  if (dual2) dot_pos(st.mu64, st.t2, NM, dual2, s);
  transpose<double>(st.t2, M, N, f, s);
  conv_f_from_pot<R>(st.py[q], st.nu64, NM, eps_ln2, g, st.ty, s);
  if (dual2) dot_pos(st.nu64, g, NM, dual2 + 1, s);
}

template <class R>
finom_status end2d(finom_plan_s* p, double* f, double* g, finom_result* res, cudaStream_t s) {
  SolveState& st = p->st;
  const int64_t N = gN(p), M = gM(p), NM = N * M;
  int32_t h[8];
  double loop_err = 0.0;
  FINOM_CUDA(cudaMemcpyAsync(h, st.ctrl, sizeof(h), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaMemcpyAsync(&loop_err, st.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  const bool done = h[1] != 0;
  int64_t iters = done ? h[3] : h[2];
  const int32_t converged = h[4];
  if (st.maxit == 0) iters = 0;
  double err64 = 0.0, w1 = 0.0;
  double* d2 = st.scal + 16;
  if (iters == 0 && !st.warm) {
    // Phi = Psi = 1/(NM): potentials eps log(1/(NM)); the error is the one
    // the loop measured at the first loop head
    const double f0 = p->eps * std::log(1.0 / (double)NM);
    fill_d(f, NM, f0, s);
    fill_d(g, NM, f0, s);
    fill_d(st.tx, NM, 0.0, s);
    fill_d(st.ty, NM, 0.0, s);
    double* uu = nullptr;
    FINOM_CUDA(cudaMallocAsync(&uu, sizeof(double) * NM, s));
    fill_d(uu, NM, 1.0 / (double)NM, s);
    finom_status rc = cost64_2d(p, st.tx, st.ty, uu, uu, &err64, &w1, s);
    cudaFreeAsync(uu, s);
    if (rc != FINOM_OK) return rc;
    err64 = loop_err;
    transpose<double>(st.mu64, M, N, st.t2, s);
    dot_pos(st.t2, f, NM, d2, s);
    dot_pos(st.nu64, g, NM, d2 + 1, s);
  } else {
    export_potentials<R>(p, (int)(iters & 1), f, g, d2, s);
    finom_status rc = cost64_2d(p, st.tx, st.ty, st.mu64, st.nu64, &err64, &w1, s);
    if (rc != FINOM_OK) return rc;
  }
  double hd[2];
  FINOM_CUDA(cudaMemcpyAsync(hd, d2, sizeof(hd), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  if (res) {
    res->w1 = w1;
    res->marginal_err = err64;
    res->marginal_err_loop = loop_err;
    res->dual = hd[0] + hd[1];
    res->iters = iters;
    res->converged = (err64 <= st.tol || (converged && sizeof(R) == sizeof(double))) ? 1 : 0;
    res->status = FINOM_OK;
  }
  st.active = false;
  return FINOM_OK;
}

template <class R>
finom_status blocking2d(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                        double* f, double* g, int32_t warm, finom_result* res, cudaStream_t us) {
  FINOM_CUDA(cudaStreamSynchronize(us));
  finom_status rc = ensure_state2d<R>(p);
  if (rc != FINOM_OK) return rc;
  SolveState& st = p->st;
  cudaStream_t s = st.stream;
  rc = begin2d<R>(p, u, v, tol, maxit, warm ? f : nullptr, warm ? g : nullptr, s);
  if (rc != FINOM_OK) return rc;
  if (maxit > 0) {
    // as in 1D: loop until the device-side check stops it; verify a float32
    // stop in float64 and resume with a tighter loop tolerance if needed
    for (int attempt = 0;; ++attempt) {
      rc = build_body2d<R>(p, 1, &st.body);
      if (rc != FINOM_OK) return rc;
      int64_t bodies = 1;
      for (;;) {
        int32_t done = 0;
        rc = poll(p, s, &done, nullptr, nullptr);
        if (rc != FINOM_OK) return rc;
        if (done) break;
        if (st.launched & 1) {
          for (int64_t b = 0; b < bodies; ++b) FINOM_CUDA(cudaGraphLaunch(st.body, s));
          st.launched += 2 * bodies;
        } else {
          rc = step2d<R>(p, 1, s);
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
      export_potentials<R>(p, q, f, g, nullptr, s);
      rc = cost64_2d(p, st.tx, st.ty, st.mu64, st.nu64, &err64, &w1, s);
      if (rc != FINOM_OK) return rc;
      if (err64 <= tol) break;
      const double fr = std::max(0.1, std::min(0.8, 0.8 * tol / err64));
      st.tol = std::max(loop_err * fr, 0.0);
      int32_t zero[2] = {0, 0};
      FINOM_CUDA(cudaMemcpyAsync(st.ctrl + 1, &zero[0], sizeof(int32_t), cudaMemcpyHostToDevice, s));
      FINOM_CUDA(cudaMemcpyAsync(st.ctrl + 4, &zero[1], sizeof(int32_t), cudaMemcpyHostToDevice, s));
      rc = half_phi<R>(p, q, s);
      if (rc != FINOM_OK) return rc;
      st.launched = l + 1;
    }
    st.tol = tol;
  }
  return end2d<R>(p, f, g, res, s);
}

// Standalone 2D products.  The first pass (Q, frames from the weights) runs
// once; the second runs twice, first with frame 0, then with the frame
// -log2 S0, and the passes are combined in float64 (as for 1D plans).
// All arrays column-major.
template <class R>
finom_status kv2d_impl(finom_plan_s* p, bool transpose_k, bool logmode, const double* a,
                       const double* b, double* out, cudaStream_t s) {
  finom_status rc = ensure_state2d<R>(p);
  if (rc != FINOM_OK) return rc;
  SolveState& st = p->st;
  st.active = false;
  const int64_t N = gN(p), M = gM(p), NM = N * M;
  const double scale = 1.0 / (p->eps * kLn2);
  const double* ao = logmode ? (transpose_k ? b : a) : nullptr;
  const double* bw = logmode ? (transpose_k ? a : b) : b;
  if (logmode) conv_weights_log<R>(bw, NM, scale, st.qw, st.qwm, s);
  else conv_weights_lin<R>(bw, NM, st.qw, st.qwm, s);
  ApplyArgs<R> p1, p2;
  if (!transpose_k) {
    // K v: columns j of grid 2 along x, then rows k of grid 1 along y
    p1 = line_args<R>(p, p->ax, M, 1);
    p1.pW = (const PotT<R>*)st.qw;
    p1.mW = (const MassT<R>*)st.qwm;
    p1.w_ls = N;
    p1.q_out = (PotT<R>*)st.q2;
    p1.q_ls = N;   // Q(k, j) at k + N j
    p1.q_es = 1;
    p2 = line_args<R>(p, p->ay, N, 1);
    p2.o_ls = 1;   // grid 1 row k: k + N i
    p2.o_es = N;
    p2.w_ls = 1;   // Q row k: k + N j
    p2.w_es = N;
  } else {
    // K^T u: rows k of grid 1 along y, then columns j of grid 2 along x
    p1 = line_args<R>(p, p->ay, N, 0);
    p1.pW = (const PotT<R>*)st.qw;
    p1.mW = (const MassT<R>*)st.qwm;
    p1.w_ls = 1;   // grid 1 row k: k + N i
    p1.w_es = N;
    p1.q_out = (PotT<R>*)st.q2;
    p1.q_ls = 1;   // Q'(k, j) at k + N j
    p1.q_es = N;
    p2 = line_args<R>(p, p->ax, M, 0);
    p2.o_ls = N;   // grid 2 column j
    p2.o_es = 1;
    p2.w_ls = N;   // Q' column j
    p2.w_es = 1;
  }
  p1.flags = kMode2InnerP;
  rc = run_pass<R>(p1, s);
  if (rc != FINOM_OK) return rc;
  p2.pO = (const PotT<R>*)st.qo;
  p2.mO = (const MassT<R>*)st.qom;
  p2.pW = (const PotT<R>*)st.q2;
  double* t0 = st.tx;
  fill_pot<R>(st.qo, NM, 0.0, s);
  p2.out = t0;
  p2.flags = kMode2Log;
  rc = run_pass<R>(p2, s);
  if (rc != FINOM_OK) return rc;
  frame_from_log<R>(t0, NM, st.qo, s);
  p2.out = out;
  p2.flags = logmode ? kMode2Log : kMode2Lin;
  rc = run_pass<R>(p2, s);
  if (rc != FINOM_OK) return rc;
  combine_passes(t0, ao, 1.0 / p->eps, NM, logmode ? 0 : 1, out, s);
  FINOM_CUDA(cudaGetLastError());
  return FINOM_OK;
}

}  // namespace

finom_status plan2d_build(finom_plan_s* p, const double* x1, const double* x2, int64_t N,
                          const double* y1, const double* y2, int64_t M, cudaStream_t s) {
  p->dim = 2;
  p->N = N * M;
  p->M = N * M;
  p->L = 0;
  p->C = 0;
  p->ax = new (std::nothrow) finom_plan_s();
  p->ay = new (std::nothrow) finom_plan_s();
  if (!p->ax || !p->ay) return FINOM_ENOMEM;
  for (finom_plan_s* a : {p->ax, p->ay}) {
    a->eps = p->eps;
    a->prec = p->prec;
    a->device = p->device;
  }
  p->ax->N = N;
  p->ax->M = N;
  p->ay->N = M;
  p->ay->M = M;
  finom_status rc = build_plan(p->ax, x1, x2, s);
  if (rc != FINOM_OK) return rc;
  return build_plan(p->ay, y1, y2, s);
}

void plan2d_free(finom_plan_s* p) {
  for (finom_plan_s** a : {&p->ax, &p->ay}) {
    if (*a) {
      free_plan(*a);
      delete *a;
      *a = nullptr;
    }
  }
}

finom_status kv2d(finom_plan_s* p, bool transpose_k, bool logmode, const double* a, const double* b,
                  double* out, cudaStream_t s) {
  return p->prec == FINOM_F32_LOG ? kv2d_impl<float>(p, transpose_k, logmode, a, b, out, s)
                                  : kv2d_impl<double>(p, transpose_k, logmode, a, b, out, s);
}

finom_status solve2d(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                     double* f, double* g, int32_t warm, finom_result* res, cudaStream_t s) {
  return p->prec == FINOM_F32_LOG ? blocking2d<float>(p, u, v, tol, maxit, f, g, warm, res, s)
                                  : blocking2d<double>(p, u, v, tol, maxit, f, g, warm, res, s);
}

finom_status solve2d_begin(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                           const double* f0, const double* g0, cudaStream_t s) {
  return p->prec == FINOM_F32_LOG ? begin2d<float>(p, u, v, tol, maxit, f0, g0, s)
                                  : begin2d<double>(p, u, v, tol, maxit, f0, g0, s);
}

finom_status solve2d_step(finom_plan_s* p, int64_t iters, cudaStream_t s) {
  return p->prec == FINOM_F32_LOG ? step2d<float>(p, iters, s) : step2d<double>(p, iters, s);
}

finom_status solve2d_end(finom_plan_s* p, double* f, double* g, finom_result* res, cudaStream_t s) {
  return p->prec == FINOM_F32_LOG ? end2d<float>(p, f, g, res, s) : end2d<double>(p, f, g, res, s);
}

// W1 and marginal error of given column-major potentials and masses (float64)
finom_status cost2d(finom_plan_s* p, const double* u, const double* v, const double* f,
                    const double* g, double* w1, double* err, cudaStream_t s) {
  finom_status rc = p->prec == FINOM_F32_LOG ? ensure_state2d<float>(p) : ensure_state2d<double>(p);
  if (rc != FINOM_OK) return rc;
  SolveState& st = p->st;
  st.active = false;
  const int64_t N = gN(p), M = gM(p), NM = N * M;
  const double scale = 1.0 / (p->eps * kLn2);
  transpose<double>(u, N, M, st.mu64, s);
  FINOM_CUDA(cudaMemcpyAsync(st.nu64, v, sizeof(double) * NM, cudaMemcpyDeviceToDevice, s));
  transpose<double>(f, N, M, st.tx, s);
  conv_pot_from_f<double>(st.tx, st.mu64, NM, scale, st.t2, s);
  conv_pot_from_f<double>(g, st.nu64, NM, scale, st.ty, s);
  return cost64_2d(p, st.t2, st.ty, st.mu64, st.nu64, err, w1, s);
}

}  // namespace finom
