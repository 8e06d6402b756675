// Queries of the transport plan Gamma = diag(phi) K diag(psi) that a solve
// returns (Algorithm 1 ends with Gamma): single rows and columns, and the
// barycentric projections of both measures, from the potentials f = eps log
// phi, g = eps log psi.  Rows and columns are entrywise float64 exponentials;
// the projections are two stabilised kernel products each (eq. decompose to
// p+q in log form), so they cost O(N + M) like one Sinkhorn iteration.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "finom_internal.h"

namespace finom {
namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// out[j] = exp((f[i] + g[j] - |x[i] - y[j]|) / eps), j < n   (row i; a column
// is the same with the roles of the meshes swapped)
__global__ void k_plan_line(const double* x, const double* f, int64_t i, const double* y, const double* g,
                            int64_t n, double inv_eps, double* out) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double fi = f[i], xi = x[i], gj = g[j];
  out[j] = (fi == -INFINITY || gj == -INFINITY) ? 0.0 : exp((fi + gj - fabs(xi - y[j])) * inv_eps);
}

// b[j] = g[j] + eps log(y[j] - y[0] + 1): the weights of the numerator of the
// projection, shifted so that the logarithm's argument is >= 1
__global__ void k_shift_log(const double* g, const double* y, int64_t n, double eps, double* b) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  b[j] = g[j] + eps * log(y[j] - y[0] + 1.0);
}

// t[i] = y[0] - 1 + exp(num[i] - den[i])
__global__ void k_unshift(const double* num, const double* den, const double* y, int64_t n, double* t) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  t[i] = den[i] == -INFINITY ? NAN : y[0] - 1.0 + exp(num[i] - den[i]);
}

bool plain_1d(finom_plan_t p, const char* what) {
  if (!p) {
    set_error(std::string(what) + ": null plan");
    return false;
  }
  if (p->dim != 1 || p->nd || p->B > 0) {
    set_error(std::string(what) + ": 1D single-problem plans only");
    return false;
  }
  return true;
}

}  // namespace
}  // namespace finom

extern "C" {

finom_status finom_transport_row(finom_plan_t p, const double* f, const double* g, int64_t i, double* out,
                                 void* stream) {
  if (!finom::plain_1d(p, "finom_transport_row")) return p ? FINOM_ENOTSUP : FINOM_EINVAL;
  if (!f || !g || !out || i < 0 || i >= p->N) {
    finom::set_error("finom_transport_row: need f, g, out non-null and 0 <= i < N");
    return FINOM_EINVAL;
  }
  finom::k_plan_line<<<finom::nblk(p->M, 256), 256, 0, (cudaStream_t)stream>>>(p->x, f, i, p->y, g, p->M,
                                                                                 1.0 / p->eps, out);
  FINOM_CUDA(cudaGetLastError());
  return FINOM_OK;
}

finom_status finom_transport_col(finom_plan_t p, const double* f, const double* g, int64_t j, double* out,
                                 void* stream) {
  if (!finom::plain_1d(p, "finom_transport_col")) return p ? FINOM_ENOTSUP : FINOM_EINVAL;
  if (!f || !g || !out || j < 0 || j >= p->M) {
    finom::set_error("finom_transport_col: need f, g, out non-null and 0 <= j < M");
    return FINOM_EINVAL;
  }
  finom::k_plan_line<<<finom::nblk(p->N, 256), 256, 0, (cudaStream_t)stream>>>(p->y, g, j, p->x, f, p->N,
                                                                                 1.0 / p->eps, out);
  FINOM_CUDA(cudaGetLastError());
  return FINOM_OK;
}

finom_status finom_barycentric(finom_plan_t p, const double* f, const double* g, double* tx, double* ty,
                               void* stream) {
  if (!finom::plain_1d(p, "finom_barycentric")) return p ? FINOM_ENOTSUP : FINOM_EINVAL;
  if (!f || !g || (!tx && !ty)) {
    finom::set_error("finom_barycentric: need f, g non-null and at least one of tx, ty");
    return FINOM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = p->N, M = p->M, n = N > M ? N : M;
  double* buf = nullptr;
  FINOM_CUDA(cudaMallocAsync(&buf, sizeof(double) * 4 * n, s));
  double *w = buf, *num = buf + n, *den = buf + 2 * n, *zero = buf + 3 * n;
  // the output side's absorption only adds a constant per point, which the
  // ratio cancels: zero keeps the projection defined at points without mass
  FINOM_CUDA(cudaMemsetAsync(zero, 0, sizeof(double) * n, s));
  finom_status rc = FINOM_OK;
  if (tx) {
    // tx_i = sum_j Gamma_ij y_j / sum_j Gamma_ij
    finom::k_shift_log<<<finom::nblk(M, 256), 256, 0, s>>>(g, p->y, M, p->eps, w);
    rc = finom_kv_log(p, zero, w, num, stream);
    if (rc == FINOM_OK) rc = finom_kv_log(p, zero, g, den, stream);
    if (rc == FINOM_OK) finom::k_unshift<<<finom::nblk(N, 256), 256, 0, s>>>(num, den, p->y, N, tx);
  }
  if (ty && rc == FINOM_OK) {
    // ty_j = sum_i Gamma_ij x_i / sum_i Gamma_ij
    finom::k_shift_log<<<finom::nblk(N, 256), 256, 0, s>>>(f, p->x, N, p->eps, w);
    rc = finom_ktu_log(p, w, zero, num, stream);
    if (rc == FINOM_OK) rc = finom_ktu_log(p, f, zero, den, stream);
    if (rc == FINOM_OK) finom::k_unshift<<<finom::nblk(M, 256), 256, 0, s>>>(num, den, p->x, M, ty);
  }
  cudaFreeAsync(buf, s);
  if (rc != FINOM_OK) return rc;
  FINOM_CUDA(cudaGetLastError());
  return FINOM_OK;
}

}  // extern "C"
