// Host side of the half-step kernel on absolute levels (half.cuh): launch
// configuration (persistent grid, programmatic dependent launch) and the
// conversions between the ABI's float64 vectors and the kernel's levels.
// Instantiated once per precision (half_f32.cu, half_f64.cu).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "half.cuh"

namespace finom {

// Persistent grid of an instantiation: resident CTAs per SM times SMs, found
// once (a function-local static, so concurrent first launches from several
// host threads initialise it once).
template <class R, int M, int E>
unsigned half_grid(int64_t units, size_t smem) {
  static const int64_t slots = [smem]() -> int64_t {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_half<R, M, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_half<R, M, E>, half_threads<R, E>(), smem) !=
        cudaSuccess)
      n = 1;
    return (int64_t)(n < 1 ? 1 : n) * (sms < 1 ? 1 : sms);
  }();
  return (unsigned)std::min<int64_t>(units, slots);
}

template <class R, int M, int E>
cudaError_t half_launch_me(const HalfArgs<R>& a, cudaStream_t s) {
  const size_t smem = sizeof(HalfSmem<R, E>);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(half_threads<R, E>());
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int64_t units = (M & H_LINES) ? (int64_t)a.lines * a.C : (int64_t)a.C;
  cfg.gridDim = dim3(half_grid<R, M, E>(units, smem));
  return cudaLaunchKernelEx(&cfg, k_half<R, M, E>, a);
}

template <class R, int E>
cudaError_t half_launch_e(const HalfArgs<R>& a, int mode, cudaStream_t s, bool* known) {
  *known = true;
  switch (mode) {
    case kHalfY: return half_launch_me<R, kHalfY, E>(a, s);
    case kHalfX: return half_launch_me<R, kHalfX, E>(a, s);
    case kHalfCheck: return half_launch_me<R, kHalfCheck, E>(a, s);
    case kHalfAgg: return half_launch_me<R, kHalfAgg, E>(a, s);
    case kHalfLog: return half_launch_me<R, kHalfLog, E>(a, s);
    case kHalfLin: return half_launch_me<R, kHalfLin, E>(a, s);
    case kHalfRawAgg: return half_launch_me<R, kHalfRawAgg, E>(a, s);
    case kHalfRawLog: return half_launch_me<R, kHalfRawLog, E>(a, s);
    case kLineAgg: return half_launch_me<R, kLineAgg, E>(a, s);
    case kLineQ: return half_launch_me<R, kLineQ, E>(a, s);
    case kLineY: return half_launch_me<R, kLineY, E>(a, s);
    case kLineX: return half_launch_me<R, kLineX, E>(a, s);
    case kLineCheck: return half_launch_me<R, kLineCheck, E>(a, s);
    case kBatchY: return half_launch_me<R, kBatchY, E>(a, s);
    case kBatchX: return half_launch_me<R, kBatchX, E>(a, s);
    case kBatchAgg: return half_launch_me<R, kBatchAgg, E>(a, s);
    case kBatchCheck: return half_launch_me<R, kBatchCheck, E>(a, s);
    default: break;
  }
  if constexpr (sizeof(R) == sizeof(double)) {
    switch (mode) {
      case kLineFB: return half_launch_me<R, kLineFB, E>(a, s);
      case kLineFBZ: return half_launch_me<R, kLineFBZ, E>(a, s);
      case kLineAggZ: return half_launch_me<R, kLineAggZ, E>(a, s);
      default: break;
    }
  }
  switch (mode) {
    default: *known = false; return cudaSuccess;
  }
}

// Launch one mode with tiles of kind elems (1, 2, 4 or 8 points per thread of
// 256 threads, or kElemsSmall: 64 threads of one point).
template <class R>
finom_status half_launch(const HalfArgs<R>& a, int mode, int elems, cudaStream_t s) {
  bool known = false;
  cudaError_t e = cudaSuccess;
  switch (elems) {
    case 1: e = half_launch_e<R, 1>(a, mode, s, &known); break;
    case 2: e = half_launch_e<R, 2>(a, mode, s, &known); break;
    case 4: e = half_launch_e<R, 4>(a, mode, s, &known); break;
    case 8: e = half_launch_e<R, 8>(a, mode, s, &known); break;
    case kElemsSmall: e = half_launch_e<R, kElemsSmall>(a, mode, s, &known); break;
    default: break;
  }
  if (!known) {
    set_error("k_half: unsupported launch mode or tile size");
    return FINOM_EINVAL;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "k_half launch");
  return FINOM_OK;
}

namespace {

__device__ __forceinline__ void put_level(float2* p, double v) {
  const float hi = (float)v;
  *p = make_float2(hi, (float)(v - (double)hi));
}
__device__ __forceinline__ void put_level(double* p, double v) { *p = v; }
__device__ __forceinline__ void put_beta(float4* p, double bp, double bm) {
  const float ph = (float)bp, mh = (float)bm;
  *p = make_float4(ph, (float)(bp - (double)ph), mh, (float)(bm - (double)mh));
}
__device__ __forceinline__ void put_beta(double2* p, double bp, double bm) { *p = make_double2(bp, bm); }
__device__ __forceinline__ double level_of(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ double level_of(double v) { return v; }
__device__ __forceinline__ double beta_p(float4 b) { return (double)b.x + (double)b.y; }
__device__ __forceinline__ double beta_m(float4 b) { return (double)b.z + (double)b.w; }
__device__ __forceinline__ double beta_p(double2 b) { return b.x; }
__device__ __forceinline__ double beta_m(double2 b) { return b.y; }

// levels of n points at positions pos (cost units, scale = 1 / (eps ln 2)):
// b = f * fscale (f given; -inf gives none), else b = fill
template <class Beta>
__global__ void k_beta_set(Beta* out, const double* pos, int64_t n, double scale, const double* f,
                           double fscale, double fill, double none) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double b = fill;
  if (f) b = (f[i] > -INFINITY) ? f[i] * fscale : none;
  const double z = pos[i] * scale;
  if (b <= 0.5 * none) put_beta(out + i, none, none);
  else put_beta(out + i, b + z, b - z);
}

// levels of linear weights v (b = log2 v; v <= 0 gives none)
template <class Beta>
__global__ void k_beta_lin(Beta* out, const double* pos, int64_t n, double scale, const double* v, double none) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double w = v[i];
  const double z = pos[i] * scale;
  if (w > 0.0) {
    const double b = log2(w);
    put_beta(out + i, b + z, b - z);
  } else {
    put_beta(out + i, none, none);
  }
}

// log2 of normalised masses (none for zero)
template <class Lv>
__global__ void k_log_mass(const double* m64, int64_t n, Lv* lm, double none) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double m = m64[i];
  put_level(lm + i, m > 0.0 ? log2(m) : none);
}

// potential f = eps ln 2 * b (-inf without mass) and the smooth potential
// P = b - log2 m (0 without mass) that the float64 cost kernel takes
template <class Beta>
__global__ void k_f_from_beta(const Beta* in, const double* m64, int64_t n, double eps_ln2, double* f,
                              double* P) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Beta v = in[i];
  const double b = 0.5 * (beta_p(v) + beta_m(v));
  const double m = m64[i];
  if (f) f[i] = (m > 0.0) ? eps_ln2 * b : -INFINITY;
  if (P) P[i] = (m > 0.0) ? b - log2(m) : 0.0;
}

inline unsigned hblk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

template <class R>
void beta_set(void* out, const double* pos, int64_t n, double scale, const double* f, double fscale,
              double fill, cudaStream_t s) {
  k_beta_set<<<hblk(n), 256, 0, s>>>((typename HT<R>::Beta*)out, pos, n, scale, f, fscale, fill,
                                     (double)HT<R>::kNone);
}
template <class R>
void beta_lin(void* out, const double* pos, int64_t n, double scale, const double* v, cudaStream_t s) {
  k_beta_lin<<<hblk(n), 256, 0, s>>>((typename HT<R>::Beta*)out, pos, n, scale, v, (double)HT<R>::kNone);
}
template <class R>
void log_mass(const double* m64, int64_t n, void* lm, cudaStream_t s) {
  k_log_mass<<<hblk(n), 256, 0, s>>>(m64, n, (typename HT<R>::Lv*)lm, (double)HT<R>::kNone);
}
template <class R>
void f_from_beta(const void* in, const double* m64, int64_t n, double eps_ln2, double* f, double* P,
                 cudaStream_t s) {
  k_f_from_beta<<<hblk(n), 256, 0, s>>>((const typename HT<R>::Beta*)in, m64, n, eps_ln2, f, P);
}

#define FINOM_HALF_INST(R)                                                                              \
  template finom_status half_launch<R>(const HalfArgs<R>&, int, int, cudaStream_t);                     \
  template void beta_set<R>(void*, const double*, int64_t, double, const double*, double, double,       \
                            cudaStream_t);                                                               \
  template void beta_lin<R>(void*, const double*, int64_t, double, const double*, cudaStream_t);        \
  template void log_mass<R>(const double*, int64_t, void*, cudaStream_t);                              \
  template void f_from_beta<R>(const void*, const double*, int64_t, double, double*, double*, cudaStream_t);

}  // namespace finom
