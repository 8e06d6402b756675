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
 *     the upper block).
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
