// Device-side building blocks of the FINOM scans.
//
// Representation.  A Sinkhorn half step needs, at every output point k of one
// mesh (the "O" side), the stabilised sum
//     S_k = sum_m  2^{ c_k + P_m + log2 w_m - G(k, m) }
// over the points m of the other mesh (the "W" side), where c is a reference
// ("frame") potential, P the absorbed potential of Remark
// log-domain-stabilization, w the mass and G = |z_k - z_m| / (eps ln 2) the
// cost in bits.  In the merged order of both meshes the lower and upper block
// sums (eqs. p/q by dynamic programming) become a forward and a backward
// first-order recurrence
//     fwd:  L_k = (L_{k-1} + A_k) (+) B_k          A_k  =  (c_k - c_{k-1}) - g_k
//     bwd:  R_{k-1} = (R_k (+) B_k) + A'_k          A'_k = -(c_k - c_{k-1}) - g_k
// with g_k the gap to the previous merged point in bits, B_k the log2 weight
// of a W point and (+) the log-sum.  Log-sums are carried as LS {m, s}
// (value s * 2^m, s in [1, 2)) so that adding one term costs one ex2.
// The recurrence maps compose associatively: Agg {D, m, s} is the map
// L -> (L + D) (+) (m, s).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace finom {

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <class R>
struct Tr;

// float path: potentials as unevaluated sums hi + lo of two floats
template <>
struct Tr<float> {
  using Pot = float2;
  using Mass = float;
  static constexpr float kNegBig = -1.0e30f;
  __device__ __forceinline__ static float ex2(float x) { return ex2_approx(x); }
  __device__ __forceinline__ static float lg2(float x) { return lg2_approx(x); }
  // a - b rounded to float (hi parts subtract exactly when close)
  __device__ __forceinline__ static float diff(Pot a, Pot b) { return (a.x - b.x) + (a.y - b.y); }
  // a + b + e rounded to float; e is an integer exponent, added to the hi
  // sum first (exact when a.x + b.x cancels, as it does for matched frames)
  __device__ __forceinline__ static float sum(Pot a, Pot b, float e) {
    return ((a.x + b.x) + e) + (a.y + b.y);
  }
  // a - t as a renormalised pair (two-sum of the hi part, Knuth)
  __device__ __forceinline__ static Pot sub(Pot a, float t) {
    float s = a.x - t;
    float bb = s - a.x;
    float err = (a.x - (s - bb)) + (-t - bb);
    float lo = err + a.y;
    float hi = s + lo;
    lo = lo - (hi - s);
    return make_float2(hi, lo);
  }
  __device__ __forceinline__ static Pot zero() { return make_float2(0.f, 0.f); }
  __device__ __forceinline__ static Pot neg(Pot a) { return make_float2(-a.x, -a.y); }
  __device__ __forceinline__ static float hi(Pot a) { return a.x; }
  // stands for -infinity in a potential (an empty sum)
  __device__ __forceinline__ static Pot none() { return make_float2(kNegBig, 0.f); }
  __device__ __forceinline__ static double to_double(Pot a) { return (double)a.x + (double)a.y; }
  // mass = mant * 2^e, mant in [1, 2); zero (or subnormal) -> (kNegBig, 0)
  __device__ __forceinline__ static void split(float w, float& e, float& mant) {
    uint32_t b = __float_as_uint(w);
    uint32_t ex = (b >> 23) & 0xffu;
    bool z = (ex == 0u);
    e = z ? kNegBig : (float)((int)ex - 127);
    mant = z ? 0.f : __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
  }
};

// double path: plain float64
template <>
struct Tr<double> {
  using Pot = double;
  using Mass = double;
  static constexpr double kNegBig = -1.0e300;
  __device__ __forceinline__ static double ex2(double x) { return exp2(x); }
  __device__ __forceinline__ static double lg2(double x) { return log2(x); }
  __device__ __forceinline__ static double diff(Pot a, Pot b) { return a - b; }
  __device__ __forceinline__ static double sum(Pot a, Pot b, double e) { return (a + b) + e; }
  __device__ __forceinline__ static Pot sub(Pot a, double t) { return a - t; }
  __device__ __forceinline__ static Pot zero() { return 0.0; }
  __device__ __forceinline__ static Pot neg(Pot a) { return -a; }
  __device__ __forceinline__ static double hi(Pot a) { return a; }
  __device__ __forceinline__ static Pot none() { return kNegBig; }
  __device__ __forceinline__ static double to_double(Pot a) { return a; }
  __device__ __forceinline__ static void split(double w, double& e, double& mant) {
    unsigned long long b = (unsigned long long)__double_as_longlong(w);
    int ex = (int)((b >> 52) & 0x7ffull);
    bool z = (ex == 0);
    e = z ? kNegBig : (double)(ex - 1023);
    mant = z ? 0.0 : __longlong_as_double((long long)((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
  }
};

template <class R>
struct LS {
  R m, s;
};

template <class R>
struct Agg {
  R D, m, s;
};

template <class R>
__device__ __forceinline__ LS<R> ls_empty() {
  return {Tr<R>::kNegBig, R(0)};
}

// Move the binary exponent of s into m so that s lands in [1, 2) (exact).
__device__ __forceinline__ void renorm(float& m, float& s) {
  int b = __float_as_int(s);
  int ex = ((b >> 23) & 0xff) - 127;
  if (ex > -127) {   // s > 0 and normal
    s = __int_as_float(b - ex * (1 << 23));
    m += (float)ex;
  }
}
__device__ __forceinline__ void renorm(double& m, double& s) {
  long long b = __double_as_longlong(s);
  long long ex = ((b >> 52) & 0x7ffll) - 1023;
  if (ex > -1023) {
    s = __longlong_as_double(b - ex * (1ll << 52));
    m += (double)ex;
  }
}

// (ma, sa) (+) (mb, sb) without renormalisation (one ex2); used inside the
// per-thread chains, where s grows by at most 2 per added point.
template <class R>
__device__ __forceinline__ void ls_add_fast(R& m, R& s, R mb, R sb) {
  R d = mb - m;
  R e = Tr<R>::ex2(-fabs(d));
  bool gt = d > R(0);
  R s1 = fma(sb, e, s);
  R s2 = fma(s, e, sb);
  s = gt ? s2 : s1;
  m = gt ? mb : m;
}

// (ma, sa) (+) (mb, sb), renormalised.
template <class R>
__device__ __forceinline__ LS<R> ls_add(R ma, R sa, R mb, R sb) {
  ls_add_fast(ma, sa, mb, sb);
  renorm(ma, sa);
  return {ma, sa};
}

template <class R>
__device__ __forceinline__ Agg<R> agg_identity() {
  return {R(0), Tr<R>::kNegBig, R(0)};
}

// map a applied first, then map b
template <class R>
__device__ __forceinline__ Agg<R> agg_then(const Agg<R>& a, const Agg<R>& b) {
  LS<R> t = ls_add(a.m + b.D, a.s, b.m, b.s);
  return {a.D + b.D, t.m, t.s};
}

// state st pushed through map a
template <class R>
__device__ __forceinline__ LS<R> agg_apply(const Agg<R>& a, LS<R> st) {
  return ls_add(st.m + a.D, st.s, a.m, a.s);
}

template <class R>
__device__ __forceinline__ Agg<R> shfl_up_agg(const Agg<R>& a, int o) {
  return {__shfl_up_sync(0xffffffffu, a.D, o), __shfl_up_sync(0xffffffffu, a.m, o),
          __shfl_up_sync(0xffffffffu, a.s, o)};
}
template <class R>
__device__ __forceinline__ Agg<R> shfl_down_agg(const Agg<R>& a, int o) {
  return {__shfl_down_sync(0xffffffffu, a.D, o), __shfl_down_sync(0xffffffffu, a.m, o),
          __shfl_down_sync(0xffffffffu, a.s, o)};
}

template <class R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// exclusive block sum of one int per thread
template <int NT>
__device__ __forceinline__ int block_exclusive_sum(int v, int* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  int wp = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w)
    if (w < warp) wp += sh[w];
  __syncthreads();
  return wp + inc - v;
}

// programmatic dependent launch: wait until the previous kernel of the
// stream has completed and its writes are visible; allow the next kernel of
// the stream to be scheduled (its blocks start as ours exit).  Both are
// no-ops when the launch did not ask for programmatic serialisation.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

}  // namespace finom
