// Launchers of the fused half-step kernel and small conversion kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "apply_launch.cuh"
#include "finom_internal.h"

namespace finom {

template <class R>
finom_status launch_apply(const ApplyArgs<R>& a, bool agg_only, cudaStream_t s) {
  const size_t smem = sizeof(TileSmem<R>);
  const int mode = agg_only ? (kModeAgg | (a.flags & (F_FRAME_W | F_WVALID | F_CHECK_DONE))) : a.flags;
  const int64_t units = (int64_t)a.C * (int64_t)(a.lines > 0 ? a.lines : 1);
  // programmatic dependent launch: the kernel stages what the previous
  // kernel does not write before it waits for that kernel to finish
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
#ifndef FINOM_PDL
#define FINOM_PDL 1
#endif
  cfg.attrs = attr;
  cfg.numAttrs = FINOM_PDL ? 1 : 0;
  cudaError_t e = cudaSuccess;
  if (a.elems != 0 && a.elems != kElems) {
    // smaller tiles (1D plans only): instantiated in their own translation units
    if (!launch_apply_small<R>(cfg, a, mode, units, smem, &e)) {
      set_error("k_apply: unsupported launch mode for this tile size");
      return FINOM_EINVAL;
    }
  } else switch (mode) {
#define FINOM_CASE(M)                                \
  case M:                                            \
    e = launch_mode<R, M, kElems>(cfg, a, units, smem); \
    break;
    FINOM_CASE(kModeAgg)
    FINOM_CASE(kModeHalfY)
    FINOM_CASE(kModeHalfX)
    FINOM_CASE(kModeCheck)
    FINOM_CASE(kModeLin)
    FINOM_CASE(kModeLog)
    FINOM_CASE(kMode2Inner)
    FINOM_CASE(kMode2HalfB)
    FINOM_CASE(kMode2HalfA)
    FINOM_CASE(kMode2Check)
    FINOM_CASE(kMode2InnerP)
    FINOM_CASE(kMode2Log)
    FINOM_CASE(kMode2Lin)
    FINOM_CASE(kMode2AggInner)
    FINOM_CASE(kMode2AggOuter)
    FINOM_CASE(kMode2AggInner | F_CHECK_DONE)
    FINOM_CASE(kMode2AggOuter | F_CHECK_DONE)
    FINOM_CASE(kModeBHalfY)
    FINOM_CASE(kModeBHalfX)
    FINOM_CASE(kModeBAgg)
    FINOM_CASE(kModeBCheck)
#undef FINOM_CASE
    default:
      set_error("k_apply: unsupported launch mode");
      return FINOM_EINVAL;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "k_apply launch");
  return FINOM_OK;
}

template finom_status launch_apply<float>(const ApplyArgs<float>&, bool, cudaStream_t);
template finom_status launch_apply<double>(const ApplyArgs<double>&, bool, cudaStream_t);

namespace {

__device__ __forceinline__ void store_pot(float2* p, int64_t i, double v) {
  float hi = (float)v;
  float lo = (float)(v - (double)hi);
  p[i] = make_float2(hi, lo);
}
__device__ __forceinline__ void store_pot(double* p, int64_t i, double v) { p[i] = v; }
__device__ __forceinline__ double load_pot(const float2* p, int64_t i) {
  float2 q = p[i];
  return (double)q.x + (double)q.y;
}
__device__ __forceinline__ double load_pot(const double* p, int64_t i) { return p[i]; }

template <class Pot, class Mass>
__global__ void k_weights_log(const double* b, int64_t n, double scale, Pot* pot, Mass* mass) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = b[i];
  bool ok = v > -INFINITY;
  store_pot(pot, i, ok ? v * scale : 0.0);
  mass[i] = ok ? (Mass)1 : (Mass)0;
}

// linear weights: v = mant * 2^e with the exponent moved into the potential
template <class Pot, class Mass>
__global__ void k_weights_lin(const double* v, int64_t n, Pot* pot, Mass* mass) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double w = v[i];
  if (w > 0.0) {
    int e;
    double m = frexp(w, &e);   // w = m * 2^e, m in [0.5, 1)
    store_pot(pot, i, (double)(e - 1));
    mass[i] = (Mass)(2.0 * m);
  } else {
    store_pot(pot, i, 0.0);
    mass[i] = (Mass)0;
  }
}

template <class Pot>
__global__ void k_pot_scale(const double* a, int64_t n, double scale, Pot* pot) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  store_pot(pot, i, a[i] * scale);
}

template <class Pot>
__global__ void k_pot_fill(Pot* pot, int64_t n, double v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  store_pot(pot, i, v);
}

template <class Mass>
__global__ void k_mass_fill(Mass* m, int64_t n, double v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  m[i] = (Mass)v;
}

// partial sums of masses with validation (deterministic two-level reduction)
__global__ void k_mass_partial(const double* u, int64_t n, double* part, int* bad) {
  __shared__ double sh[256];
  double s = 0.0;
  bool ok = true;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = u[i];
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

__global__ void k_mass_total(const double* part, int nb, double* total) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    *total = s;
  }
}

template <class Mass>
__global__ void k_mass_norm(const double* u, int64_t n, const double* total, Mass* m, double* m64) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = u[i] / *total;
  m64[i] = v;
  m[i] = (Mass)v;
}

// smooth potential from a full potential: P = f / (eps ln 2) - log2 u (0 where u = 0)
template <class Pot>
__global__ void k_pot_from_f(const double* f, const double* m64, int64_t n, double scale, Pot* pot) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double w = m64[i];
  double fv = f[i];
  store_pot(pot, i, (w > 0.0 && fv > -INFINITY) ? fv * scale - log2(w) : 0.0);
}

// full potential f = eps ln2 (P + log2 u), -inf where u = 0
template <class Pot>
__global__ void k_f_from_pot(const Pot* pot, const double* m64, int64_t n, double eps_ln2, double* f,
                             double* p64) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double P = load_pot(pot, i);
  double w = m64[i];
  if (p64) p64[i] = P;
  f[i] = (w > 0.0) ? eps_ln2 * (P + log2(w)) : -INFINITY;
}

// frame for the second pass of a standalone product: c = -ln S0 / ln 2 (0 where S0 = 0)
template <class Pot>
__global__ void k_frame_from_log(const double* t0, int64_t n, Pot* pot) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = t0[i];
  store_pot(pot, i, (v > -INFINITY && v < INFINITY) ? -v * 1.4426950408889634074 : 0.0);
}

// combine the two passes: linear S = e^{t0} S2, log: a/eps + t0 + ln S2
__global__ void k_combine(const double* t0, const double* a, double inv_eps, int64_t n, int lin, double* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t = t0[i];
  double l2 = out[i];
  if (lin) out[i] = (t > -INFINITY) ? exp(t) * l2 : 0.0;
  else out[i] = (t > -INFINITY) ? a[i] * inv_eps + t + l2 : -INFINITY;
}

// out += a * sc (ln of a product plus the O side's absorption a / eps)
__global__ void k_add_scaled(double* out, const double* a, double sc, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = out[i] + a[i] * sc;
}

__global__ void k_fill_d(double* f, int64_t n, double v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
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

// dst(r, c) at c + cols r  <-  src(r, c) at r + rows c  (32 x 32 tiles via shared memory)
template <class T>
__global__ void k_transpose(const T* src, int64_t rows, int64_t cols, T* dst) {
  __shared__ T t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + threadIdx.x, c = c0 + k;
    if (r < rows && c < cols) t[k][threadIdx.x] = src[r + rows * c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t c = c0 + threadIdx.x, r = r0 + k;
    if (r < rows && c < cols) dst[c + cols * r] = t[threadIdx.x][k];
  }
}

inline unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

template <class T>
void transpose(const T* src, int64_t rows, int64_t cols, T* dst, cudaStream_t s) {
  dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32));
  k_transpose<T><<<grid, dim3(32, 8), 0, s>>>(src, rows, cols, dst);
}
template void transpose<double>(const double*, int64_t, int64_t, double*, cudaStream_t);
template void transpose<float>(const float*, int64_t, int64_t, float*, cudaStream_t);
template void transpose<float2>(const float2*, int64_t, int64_t, float2*, cudaStream_t);

template <class R>
void frame_from_log(const double* t0, int64_t n, void* pot, cudaStream_t s) {
  k_frame_from_log<<<nb(n), 256, 0, s>>>(t0, n, (typename Tr<R>::Pot*)pot);
}
void combine_passes(const double* t0, const double* a, double inv_eps, int64_t n, int lin, double* out,
                    cudaStream_t s) {
  k_combine<<<nb(n), 256, 0, s>>>(t0, a, inv_eps, n, lin, out);
}
template <class R>
void conv_weights_log(const double* b, int64_t n, double scale, void* pot, void* mass, cudaStream_t s) {
  k_weights_log<<<nb(n), 256, 0, s>>>(b, n, scale, (typename Tr<R>::Pot*)pot,
                                      (typename Tr<R>::Mass*)mass);
}
template <class R>
void conv_weights_lin(const double* v, int64_t n, void* pot, void* mass, cudaStream_t s) {
  k_weights_lin<<<nb(n), 256, 0, s>>>(v, n, (typename Tr<R>::Pot*)pot, (typename Tr<R>::Mass*)mass);
}
template <class R>
void conv_pot_scale(const double* a, int64_t n, double scale, void* pot, cudaStream_t s) {
  k_pot_scale<<<nb(n), 256, 0, s>>>(a, n, scale, (typename Tr<R>::Pot*)pot);
}
template <class R>
void fill_pot(void* pot, int64_t n, double v, cudaStream_t s) {
  k_pot_fill<<<nb(n), 256, 0, s>>>((typename Tr<R>::Pot*)pot, n, v);
}
template <class R>
void fill_mass(void* m, int64_t n, double v, cudaStream_t s) {
  k_mass_fill<<<nb(n), 256, 0, s>>>((typename Tr<R>::Mass*)m, n, v);
}
template <class R>
void conv_pot_from_f(const double* f, const double* m64, int64_t n, double scale, void* pot,
                     cudaStream_t s) {
  k_pot_from_f<<<nb(n), 256, 0, s>>>(f, m64, n, scale, (typename Tr<R>::Pot*)pot);
}
template <class R>
void conv_f_from_pot(const void* pot, const double* m64, int64_t n, double eps_ln2, double* f,
                     double* p64, cudaStream_t s) {
  k_f_from_pot<<<nb(n), 256, 0, s>>>((const typename Tr<R>::Pot*)pot, m64, n, eps_ln2, f, p64);
}

#define FINOM_INST(R)                                                                        \
  template void frame_from_log<R>(const double*, int64_t, void*, cudaStream_t);                  \
  template void conv_weights_log<R>(const double*, int64_t, double, void*, void*, cudaStream_t); \
  template void conv_weights_lin<R>(const double*, int64_t, void*, void*, cudaStream_t);         \
  template void conv_pot_scale<R>(const double*, int64_t, double, void*, cudaStream_t);          \
  template void fill_pot<R>(void*, int64_t, double, cudaStream_t);                               \
  template void fill_mass<R>(void*, int64_t, double, cudaStream_t);                              \
  template void conv_pot_from_f<R>(const double*, const double*, int64_t, double, void*,         \
                                   cudaStream_t);                                                \
  template void conv_f_from_pot<R>(const void*, const double*, int64_t, double, double*, double*, \
                                   cudaStream_t);
FINOM_INST(float)
FINOM_INST(double)
#undef FINOM_INST

void fill_d(double* f, int64_t n, double v, cudaStream_t s) { k_fill_d<<<nb(n), 256, 0, s>>>(f, n, v); }
void add_scaled(double* out, const double* a, double sc, int64_t n, cudaStream_t s) {
  k_add_scaled<<<nb(n), 256, 0, s>>>(out, a, sc, n);
}
void dot_pos(const double* m, const double* f, int64_t n, double* out, cudaStream_t s) {
  k_dot_pos<<<1, 256, 0, s>>>(m, f, n, out);
}

// Normalise masses u (float64, device) into m (plan precision) and m64.
// Returns FINOM_EINVAL when u has a negative / non-finite entry or a
// non-positive sum.  Synchronous.
template <class R>
finom_status normalise_masses(const double* u, int64_t n, void* m, double* m64, double* scratch,
                              int* bad, double* total_out, cudaStream_t s) {
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
  k_mass_norm<<<nb(n), 256, 0, s>>>(u, n, scratch + 256, (typename Tr<R>::Mass*)m, m64);
  FINOM_CUDA(cudaGetLastError());
  if (total_out) *total_out = tot;
  return FINOM_OK;
}
template finom_status normalise_masses<float>(const double*, int64_t, void*, double*, double*, int*,
                                              double*, cudaStream_t);
template finom_status normalise_masses<double>(const double*, int64_t, void*, double*, double*, int*,
                                               double*, cudaStream_t);

}  // namespace finom
