// Small float64 vector kernels shared by the plans: mass normalisation with
// validation, fills, the dual sum, and the smooth potentials the float64
// cost kernel takes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "finom_internal.h"

namespace finom {

namespace {

inline unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

// partial sums of masses with validation (deterministic two-level reduction)
__global__ void k_mass_partial(const double* u, int64_t n, double* part, int* bad) {
  __shared__ double sh[256];
  double s = 0.0;
  bool ok = true;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
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
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_mass_total(const double* part, int nblocks, double* total) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[b];
    *total = s;
  }
}

__global__ void k_mass_norm(const double* u, int64_t n, const double* total, double* m64) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) m64[i] = u[i] / *total;
}

// smooth potential from a full potential: P = f / (eps ln 2) - log2 u (0 where u = 0)
__global__ void k_pot_from_f(const double* f, const double* m64, int64_t n, double scale, double* pot) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double w = m64[i];
  const double fv = f[i];
  pot[i] = (w > 0.0 && fv > -INFINITY) ? fv * scale - log2(w) : 0.0;
}

// out += a * sc (ln of a product plus the O side's absorption a / eps)
__global__ void k_add_scaled(double* out, const double* a, double sc, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = out[i] + a[i] * sc;
}

__global__ void k_fill_d(double* f, int64_t n, double v) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) f[i] = v;
}

// sum_i m_i f_i over points with m_i > 0 (one block, deterministic)
__global__ void k_dot_pos(const double* m, const double* f, int64_t n, double* out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
    if (m[i] > 0.0) s += m[i] * f[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

}  // namespace

void pot_from_f(const double* f, const double* m64, int64_t n, double scale, double* pot, cudaStream_t s) {
  k_pot_from_f<<<nb(n), 256, 0, s>>>(f, m64, n, scale, pot);
}
void fill_d(double* f, int64_t n, double v, cudaStream_t s) { k_fill_d<<<nb(n), 256, 0, s>>>(f, n, v); }
void add_scaled(double* out, const double* a, double sc, int64_t n, cudaStream_t s) {
  k_add_scaled<<<nb(n), 256, 0, s>>>(out, a, sc, n);
}
void dot_pos(const double* m, const double* f, int64_t n, double* out, cudaStream_t s) {
  k_dot_pos<<<1, 256, 0, s>>>(m, f, n, out);
}

// Normalise masses u (float64, device) into m64.  scratch: 257 doubles.
// Returns FINOM_EINVAL when u has a negative / non-finite entry or a
// non-positive sum.  Synchronous.
finom_status normalise_masses(const double* u, int64_t n, double* m64, double* scratch, int* bad,
                              double* total_out, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>(256, (n + 255) / 256);
  FINOM_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  k_mass_partial<<<blocks, 256, 0, s>>>(u, n, scratch, bad);
  k_mass_total<<<1, 32, 0, s>>>(scratch, blocks, scratch + 256);
  int hbad = 0;
  double tot = 0.0;
  FINOM_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaMemcpyAsync(&tot, scratch + 256, sizeof(double), cudaMemcpyDeviceToHost, s));
  FINOM_CUDA(cudaStreamSynchronize(s));
  if (hbad || !(tot > 0.0) || !std::isfinite(tot)) {
    set_error("masses must be finite, >= 0 and have a positive sum");
    return FINOM_EINVAL;
  }
  k_mass_norm<<<nb(n), 256, 0, s>>>(u, n, scratch + 256, m64);
  FINOM_CUDA(cudaGetLastError());
  if (total_out) *total_out = tot;
  return FINOM_OK;
}

}  // namespace finom
