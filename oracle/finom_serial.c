/*
 * Serial FINOM in plain C, float64 (test infrastructure).
 *
 * TEST INFRASTRUCTURE ONLY: compiled by oracle/serial_c.py and called from
 * tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
 * legs.  It shares no code with the CUDA library.
 *
 * The same steps as oracle/finom_serial.py, for inputs too large for Python
 * loops:
 *   - dividing index (Definition, Sec. 2.2): zeta(i) = #{j : y_j <= x_i};
 *   - the p/q recurrences (eqs. p and q by dynamic programming, Sec. 2.3) for
 *     the kernel with column absorption b (Remark log-domain-stabilization),
 *     evaluated in log arithmetic:
 *       p_1 = LSE_{j < zeta(1)} (b_j - (x_1 - y_j)) / eps
 *       p_{i+1} = logaddexp(p_i - (x_{i+1} - x_i)/eps, LSE of the block-edge
 *                 entries (b_j - (x_{i+1} - y_j))/eps, zeta(i) <= j < zeta(i+1))
 *     and the mirror-image backward recurrence for q;
 *   - Algorithm 1 (psi first, then phi) with absorption after every half step;
 *   - <C, Gamma> with the cost-weighted lower block: since
 *       (x_{i+1} - y_j) k_{i+1,j} = r_i (x_i - y_j) k_ij + (x_{i+1} - x_i) r_i k_ij,
 *     the cost-weighted sums obey c_{i+1} = r_i (c_i + (x_{i+1} - x_i) p_i)
 *     + block-edge terms, next to the p recurrence (and the mirror image for
 *     the upper block);
 *   - the 2D products of Appendix A (eq. K'bpsi): the 1D stabilised product
 *     applied to every column along x, then to every row along y; Algorithm 2
 *     with absorption after every half step; the 2D <C, Gamma> from the
 *     separable cost, C_x o K_x (x) K_y + K_x (x) C_y o K_y.
 * Build: gcc -O2 -fPIC -shared (no fast-math: IEEE semantics are kept).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static double lae(double a, double b) {
  if (a == -INFINITY) return b;
  if (b == -INFINITY) return a;
  double m = a > b ? a : b;
  return m + log1p(exp(-fabs(a - b)));
}

void finom_ref_dividing_index(const double* x, int64_t N, const double* y, int64_t M, int64_t* zeta) {
  int64_t j = 0;
  for (int64_t i = 0; i < N; ++i) {
    while (j < M && y[j] <= x[i]) ++j;
    zeta[i] = j;
  }
}

/*
 * out_i = log sum_j exp((b_j - |x_i - y_j|)/eps) for i < N (rows x, columns y).
 * b_j may be -inf.  Optional lp, lq receive log p, log q.  Optional
 * cost (N) receives log sum_j |x_i - y_j| exp((b_j - |x_i - y_j|)/eps).
 */
void finom_ref_log_apply(const double* x, int64_t N, const double* y, int64_t M, double eps,
                         const double* b, double* out, double* lp, double* lq, double* cost) {
  int64_t* zeta = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  double* P = (double*)malloc(sizeof(double) * (size_t)N);
  double* Q = (double*)malloc(sizeof(double) * (size_t)N);
  double* PC = (double*)malloc(sizeof(double) * (size_t)N);
  double* QC = (double*)malloc(sizeof(double) * (size_t)N);
  finom_ref_dividing_index(x, N, y, M, zeta);
  /* forward: lower block */
  double p = -INFINITY, pc = -INFINITY;
  int64_t j0 = 0;
  for (int64_t i = 0; i < N; ++i) {
    if (i > 0) {
      double dx = x[i] - x[i - 1];
      double lr = -dx / eps;
      /* c_{i} = r (c_{i-1} + dx p_{i-1}) */
      double t = (dx > 0.0 && p != -INFINITY) ? log(dx) + p : -INFINITY;
      pc = lae(pc, t);
      if (pc != -INFINITY) pc += lr;
      if (p != -INFINITY) p += lr;
    }
    for (int64_t j = j0; j < zeta[i]; ++j) {
      double d = x[i] - y[j];
      double e = (b[j] - d) / eps;
      p = lae(p, e);
      if (d > 0.0) pc = lae(pc, log(d) + e);
    }
    j0 = zeta[i];
    P[i] = p;
    PC[i] = pc;
  }
  /* backward: upper block */
  double q = -INFINITY, qc = -INFINITY;
  int64_t j1 = M;
  for (int64_t i = N - 1; i >= 0; --i) {
    if (i < N - 1) {
      double dx = x[i + 1] - x[i];
      double lr = -dx / eps;
      double t = (dx > 0.0 && q != -INFINITY) ? log(dx) + q : -INFINITY;
      qc = lae(qc, t);
      if (qc != -INFINITY) qc += lr;
      if (q != -INFINITY) q += lr;
    }
    for (int64_t j = j1 - 1; j >= zeta[i]; --j) {
      double d = y[j] - x[i];
      double e = (b[j] - d) / eps;
      q = lae(q, e);
      if (d > 0.0) qc = lae(qc, log(d) + e);
    }
    j1 = zeta[i];
    Q[i] = q;
    QC[i] = qc;
  }
  for (int64_t i = 0; i < N; ++i) {
    out[i] = lae(P[i], Q[i]);
    if (lp) lp[i] = P[i];
    if (lq) lq[i] = Q[i];
    if (cost) cost[i] = lae(PC[i], QC[i]);
  }
  free(zeta); free(P); free(Q); free(PC); free(QC);
}

/* compensated (Neumaier) accumulation */
typedef struct { double s, c; } nsum;
static void nadd(nsum* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v; else a->c += (v - t) + a->s;
  a->s = t;
}

/* || diag(psi) K^T phi - v ||_1 for f = eps log phi, g = eps log psi */
double finom_ref_marginal_error(const double* x, int64_t N, const double* y, int64_t M, double eps,
                                const double* f, const double* g, const double* v) {
  double* q = (double*)malloc(sizeof(double) * (size_t)M);
  finom_ref_log_apply(y, M, x, N, eps, f, q, NULL, NULL, NULL);
  nsum acc = {0.0, 0.0};
  for (int64_t j = 0; j < M; ++j) nadd(&acc, fabs(exp(g[j] / eps + q[j]) - v[j]));
  free(q);
  return acc.s + acc.c;
}

/* <C, Gamma>, Gamma_ij = exp((f_i + g_j - |x_i - y_j|)/eps) */
double finom_ref_cost(const double* x, int64_t N, const double* y, int64_t M, double eps,
                      const double* f, const double* g) {
  double* out = (double*)malloc(sizeof(double) * (size_t)N);
  double* c = (double*)malloc(sizeof(double) * (size_t)N);
  finom_ref_log_apply(x, N, y, M, eps, g, out, NULL, NULL, c);
  nsum acc = {0.0, 0.0};
  for (int64_t i = 0; i < N; ++i)
    if (f[i] != -INFINITY && c[i] != -INFINITY) nadd(&acc, exp(f[i] / eps + c[i]));
  free(out); free(c);
  return acc.s + acc.c;
}

/*
 * Algorithm 1 with absorption after every half step.  f, g (cost units) are
 * outputs; if warm != 0 they are also the starting potentials, else the start
 * is phi = 1/N, psi = 1/M.  Returns the completed iterations; *err receives
 * the marginal error at the loop exit.  u, v must sum to 1.
 */
int64_t finom_ref_sinkhorn(const double* x, int64_t N, const double* y, int64_t M, const double* u,
                           const double* v, double eps, double tol, int64_t maxit, int warm,
                           double* f, double* g, double* err) {
  double* q = (double*)malloc(sizeof(double) * (size_t)(N > M ? N : M));
  if (!warm) {
    for (int64_t i = 0; i < N; ++i) f[i] = eps * log(1.0 / (double)N);
    for (int64_t j = 0; j < M; ++j) g[j] = eps * log(1.0 / (double)M);
  }
  int64_t it = 0;
  double e = 0.0;
  for (;;) {
    /* log (K^T phi)_j */
    finom_ref_log_apply(y, M, x, N, eps, f, q, NULL, NULL, NULL);
    nsum acc = {0.0, 0.0};
    for (int64_t j = 0; j < M; ++j) nadd(&acc, fabs(exp(g[j] / eps + q[j]) - v[j]));
    e = acc.s + acc.c;
    if (it >= maxit || e <= tol) break;
    for (int64_t j = 0; j < M; ++j) g[j] = (v[j] > 0.0) ? eps * (log(v[j]) - q[j]) : -INFINITY;
    finom_ref_log_apply(x, N, y, M, eps, g, q, NULL, NULL, NULL);
    for (int64_t i = 0; i < N; ++i) f[i] = (u[i] > 0.0) ? eps * (log(u[i]) - q[i]) : -INFINITY;
    ++it;
  }
  free(q);
  *err = e;
  return it;
}

/* ------------------------------------------------------------------ 2D --- */
/*
 * Grids: grid 1 = (x1_k, y1_i), grid 2 = (x2_l, y2_j), k, l < N, i, j < M,
 * arrays column-major (k + N i).  out(k, i) = log sum_{l, j} exp((B(l, j) -
 * |x1_k - x2_l| - |y1_i - y2_j|) / eps): the column pass logQ(:, j) =
 * log K_x e^{B(:, j)/eps}, then the row pass log (K_y e^{logQ(k, :)}) (the
 * absorption of the output grid is left to the caller).  With cost_axis = 1
 * (2) the x (y) pass returns the cost-weighted sums instead, so that the
 * result is log sum |x1_k - x2_l| (|y1_i - y2_j|) exp(...).
 */
static void log_apply2d_impl(const double* x1, const double* y1, const double* x2, const double* y2,
                             int64_t N, int64_t M, double eps, const double* B, double* out,
                             int cost_axis) {
  double* Q = (double*)malloc(sizeof(double) * (size_t)(N * M));
  double* col = (double*)malloc(sizeof(double) * (size_t)N);
  double* cst = (double*)malloc(sizeof(double) * (size_t)(N > M ? N : M));
  double* row = (double*)malloc(sizeof(double) * (size_t)M);
  double* rout = (double*)malloc(sizeof(double) * (size_t)M);
  for (int64_t j = 0; j < M; ++j) {
    finom_ref_log_apply(x1, N, x2, N, eps, B + N * j, col, NULL, NULL, cost_axis == 1 ? cst : NULL);
    for (int64_t k = 0; k < N; ++k) Q[k + N * j] = (cost_axis == 1) ? cst[k] : col[k];
  }
  for (int64_t k = 0; k < N; ++k) {
    for (int64_t j = 0; j < M; ++j) row[j] = eps * Q[k + N * j];
    finom_ref_log_apply(y1, M, y2, M, eps, row, rout, NULL, NULL, cost_axis == 2 ? cst : NULL);
    for (int64_t i = 0; i < M; ++i) out[k + N * i] = (cost_axis == 2) ? cst[i] : rout[i];
  }
  free(Q); free(col); free(cst); free(row); free(rout);
}

void finom_ref_log_apply2d(const double* x1, const double* y1, const double* x2, const double* y2,
                           int64_t N, int64_t M, double eps, const double* B, double* out) {
  log_apply2d_impl(x1, y1, x2, y2, N, M, eps, B, out, 0);
}

/* sum | exp(B/eps + log K^T e^{A/eps}) - V | over grid 2 */
double finom_ref_marginal_error2d(const double* x1, const double* y1, const double* x2,
                                  const double* y2, int64_t N, int64_t M, double eps,
                                  const double* A, const double* B, const double* V) {
  double* lt = (double*)malloc(sizeof(double) * (size_t)(N * M));
  log_apply2d_impl(x2, y2, x1, y1, N, M, eps, A, lt, 0);
  nsum acc = {0.0, 0.0};
  for (int64_t t = 0; t < N * M; ++t) nadd(&acc, fabs(exp(B[t] / eps + lt[t]) - V[t]));
  free(lt);
  return acc.s + acc.c;
}

/* <C, Gamma>, Gamma = exp((A(k,i) + B(l,j) - C)/eps), C = |dx| + |dy| */
double finom_ref_cost2d(const double* x1, const double* y1, const double* x2, const double* y2,
                        int64_t N, int64_t M, double eps, const double* A, const double* B) {
  double* r = (double*)malloc(sizeof(double) * (size_t)(N * M));
  nsum acc = {0.0, 0.0};
  for (int axis = 1; axis <= 2; ++axis) {
    log_apply2d_impl(x1, y1, x2, y2, N, M, eps, B, r, axis);
    for (int64_t t = 0; t < N * M; ++t)
      if (A[t] != -INFINITY && r[t] != -INFINITY) nadd(&acc, exp(A[t] / eps + r[t]));
  }
  free(r);
  return acc.s + acc.c;
}

/*
 * Algorithm 2 with absorption after every half step (Appendix A).  A, B
 * (cost units, grid 1 / grid 2, column-major) are outputs; if warm != 0 they
 * are also the start, else Phi = Psi = 1/(NM).  The loop head checks
 * || diag(psi) K^T phi - v ||_1 as Algorithm 2 does.  U, V sum to 1.
 */
int64_t finom_ref_sinkhorn2d(const double* x1, const double* y1, const double* x2, const double* y2,
                             int64_t N, int64_t M, const double* U, const double* V, double eps,
                             double tol, int64_t maxit, int warm, double* A, double* B, double* err) {
  const int64_t NM = N * M;
  double* lt = (double*)malloc(sizeof(double) * (size_t)NM);
  if (!warm) {
    for (int64_t t = 0; t < NM; ++t) A[t] = B[t] = eps * log(1.0 / (double)NM);
  }
  int64_t it = 0;
  double e = 0.0;
  for (;;) {
    log_apply2d_impl(x2, y2, x1, y1, N, M, eps, A, lt, 0);   /* log K^T phi on grid 2 */
    nsum acc = {0.0, 0.0};
    for (int64_t t = 0; t < NM; ++t) nadd(&acc, fabs(exp(B[t] / eps + lt[t]) - V[t]));
    e = acc.s + acc.c;
    if (it >= maxit || e <= tol) break;
    for (int64_t t = 0; t < NM; ++t) B[t] = (V[t] > 0.0) ? eps * (log(V[t]) - lt[t]) : -INFINITY;
    log_apply2d_impl(x1, y1, x2, y2, N, M, eps, B, lt, 0);   /* log K psi on grid 1 */
    for (int64_t t = 0; t < NM; ++t) A[t] = (U[t] > 0.0) ? eps * (log(U[t]) - lt[t]) : -INFINITY;
    ++it;
  }
  free(lt);
  *err = e;
  return it;
}
