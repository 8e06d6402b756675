// FINOM half step on absolute levels: one launch applies K (or K^T) to the
// weights of one mesh and performs the Sinkhorn division at the other.
//
// Every point k of either mesh carries its log-weight b_k in bits (b = f /
// (eps ln 2) for a potential f in cost units; it includes log2 of the mass)
// and its position Z_k = z_k / (eps ln 2) in bits, stored as the two levels
//     beta+_k = b_k + Z_k,      beta-_k = b_k - Z_k.
// With the merged order of both meshes (y before x on ties), the dividing
// index zeta(k) of an output point k (Definition, Sec. 2.2) counts the
// weight points before it, and the two blocks of eq. decompose to p+q are
//     p_k = sum_{m < zeta(k)} 2^{b_m - (Z_k - Z_m)} = 2^{-Z_k} sum_{m < zeta(k)} 2^{beta+_m}
//     q_k = sum_{m >= zeta(k)} 2^{b_m - (Z_m - Z_k)} = 2^{Z_k}  sum_{m >= zeta(k)} 2^{beta-_m}
// i.e. the first-order recurrences of eqs. p/q by dynamic programming, with
// their decay factors folded into the levels, become a prefix and a suffix
// log-sum over the weight points.  The log-sum is associative and
// commutative, so tile maps and carries are plain log-sum states (M, s):
// value s * 2^M, M a level of the weight points (exact: a float-float pair in
// the float32 path), s in [1, n] a float sum of mantissas.  Levels are large
// numbers; only differences of levels that are moderate wherever they matter
// are rounded to float32, so the float32 path keeps its precision on any
// mesh (large gaps, disjoint supports).
//
// At an output (O) point with the old log-weight b_k as frame, the stabilised
// sum of the Remark on log-domain stabilisation is
//     S_k = 2^{b_k} (p_k + q_k) = 2^{beta-_k} P_k + 2^{beta+_k} Q_k,
// P_k, Q_k the prefix / suffix sums; the division of eq. iteration sets
//     b_k <- log2 mu_k - log2 (p_k + q_k) = b_k - delta_k,
//     delta_k = log2 S_k - log2 mu_k,
// and the marginal error of Algorithm 1's loop head (Sec. 4) is
//     sum_k |S_k - mu_k| = sum_k mu_k |2^{delta_k} - 1|.
//
// One CTA owns one tile of the merged order (E points per thread).  Its weight
// (W) points and output (O) points are handled separately, each as contiguous
// runs of about equal length per thread (no per-point predication):
//   1. every thread records, for each O point of its merged points, the
//      number of W points of the tile before it (its local dividing index);
//   2. W phase: each thread forms the running prefix log-sum of beta+ and the
//      running suffix log-sum of beta- over its W run, in shared memory; two
//      warps scan the 256 run totals, seeded with the tile's carries;
//   3. O phase: each O point combines the entry state of the thread that owns
//      the W point at its dividing index with that thread's local state,
//      forms S_k, divides, adds its marginal-error term and, for the next
//      application (roles swapped), accumulates its new levels into the
//      tile's aggregate;
//   4. the last CTA to finish scans the tile aggregates into the carries of
//      the next launch, reduces the error in float64 and updates the loop
//      control.
#pragma once

#include <cstddef>
#include <cstdint>

#include "dev_common.cuh"
#include "exp2_table.h"
#include "finom_internal.h"

namespace finom {

enum : int {
  H_POT = 1,          // division: write the new O levels
  H_ERR = 2,          // marginal error at the O points + convergence flag
  H_NEXT = 4,         // tile aggregates of the next application (new O levels)
  H_ITER_END = 8,     // this launch ends a Sinkhorn iteration
  H_CHECK_DONE = 16,  // exit at once when the loop is done
  H_AGG = 32,         // only the tile aggregates of this application's W side
  H_LOG = 64,         // products: ln of the sum at the O points (float64)
  H_LIN = 128,        // products: the sum at the O points (float64)
  H_RAW = 256,        // products: levels formed from the caller's float64 vectors and the
                      // plan's positions inside the kernel (no converted copies)
  H_LINES = 512,      // axis pass of a tensor-product grid: units are (line, tile) of an
                      // axis plan; log-weights on the grid, positions per axis node
  H_QOUT = 1024,      // axis pass: write log2 of the product at the O nodes (a level pair)
  H_FB = 2048,        // axis pass: write log2 of the lower and of the upper block sums apart
                      // (float64, out and out + grid size)
  H_ZLOG = 4096,      // axis pass: the W levels carry log2(z - z_min) of their node as well
  H_BATCH = 8192,     // batch of independent 1D problems: units are the tiles of the active
                      // list; carries, errors and loop control per problem come from the
                      // batch end kernel (no launch tail)
};

constexpr int kHalfY = H_POT | H_ERR | H_NEXT | H_CHECK_DONE;       // psi <- nu / K^T phi
constexpr int kHalfX = H_POT | H_NEXT | H_ITER_END | H_CHECK_DONE;  // phi <- mu / K psi
constexpr int kHalfCheck = H_ERR;                                    // loop-head check only
constexpr int kHalfAgg = H_AGG;
constexpr int kHalfLog = H_LOG;
constexpr int kHalfLin = H_LIN;
constexpr int kHalfRawAgg = H_AGG | H_RAW;
constexpr int kHalfRawLog = H_LOG | H_RAW;
// axis passes of a d-dimensional application (Sec. 3, applied axis by axis)
constexpr int kLineAgg = H_AGG | H_LINES;                    // tile aggregates of the W side
constexpr int kLineQ = H_QOUT | H_LINES;                     // a pass before the last one
constexpr int kLineY = H_POT | H_ERR | H_CHECK_DONE | H_LINES;  // last pass of K^T phi: divide + check
constexpr int kLineX = H_POT | H_ITER_END | H_CHECK_DONE | H_LINES;  // last pass of K psi
constexpr int kLineCheck = H_ERR | H_LINES;
// the cost-weighted pass of <C, Gamma> (float64): both block sums apart,
// with plain and with distance-weighted levels
constexpr int kLineFB = H_FB | H_LINES;
constexpr int kLineFBZ = H_FB | H_ZLOG | H_LINES;
constexpr int kLineAggZ = H_AGG | H_ZLOG | H_LINES;
// batches of independent 1D problems (Algorithm 1 per problem)
constexpr int kBatchY = H_POT | H_ERR | H_NEXT | H_BATCH;
constexpr int kBatchX = H_POT | H_NEXT | H_BATCH;
constexpr int kBatchAgg = H_AGG | H_BATCH;
constexpr int kBatchCheck = H_ERR | H_BATCH;

// Level arithmetic per precision.  Beta holds (beta+, beta-) of one point.
template <class R>
struct HT;

template <>
struct HT<float> {
  using Lv = float2;    // unevaluated sum hi + lo
  using Beta = float4;  // (beta+.hi, beta+.lo, beta-.hi, beta-.lo)
  static constexpr int kSt = 3;   // values of a stored state: M.hi, M.lo, s
  static constexpr float kNone = -1.0e30f;
  __device__ __forceinline__ static Lv bp(const Beta& b) { return make_float2(b.x, b.y); }
  __device__ __forceinline__ static Lv bm(const Beta& b) { return make_float2(b.z, b.w); }
  __device__ __forceinline__ static Beta pack(Lv p, Lv m) { return make_float4(p.x, p.y, m.x, m.y); }
  __device__ __forceinline__ static Lv none() { return make_float2(kNone, 0.f); }
  __device__ __forceinline__ static bool valid(Lv a) { return a.x > 0.5f * kNone; }
  __device__ __forceinline__ static float ex2(float x) { return ex2_approx(x); }
  __device__ __forceinline__ static float lg2(float x) { return lg2_approx(x); }
  // log2 with a relative error of about one ulp of the result: the division
  // step takes log2 of a mantissa sum in [1, 4), where lg2.approx has an
  // absolute error of ~2^-22 (not small against a result near 0)
  __device__ __forceinline__ static float lg2_acc(float x) { return log2f(x); }
  // a - b rounded once (exact where the hi parts are within a factor 2)
  __device__ __forceinline__ static float diff(Lv a, Lv b) { return (a.x - b.x) + (a.y - b.y); }
  // (a + b) + k - c for a small integer k: the hi parts are added with
  // their rounding error kept (two-sum), and k and c enter before anything
  // is rounded, so the result is accurate wherever it is moderate
  __device__ __forceinline__ static float sum_minus(Lv a, Lv b, Lv c, float k) {
    const float s = a.x + b.x;
    const float bb = s - a.x;
    const float e = (a.x - (s - bb)) + (b.x - bb);
    return (((s + k) - c.x) + e) + ((a.y + b.y) - c.y);
  }
  // s = m 2^k with m in [1, 2) (s = 0: m = 0, k = 0)
  __device__ __forceinline__ static float mant_exp(float s, float& m) {
    const uint32_t b = __float_as_uint(s);
    const int ex = (int)((b >> 23) & 0xffu);
    m = ex ? __uint_as_float((b & 0x007fffffu) | 0x3f800000u) : 0.f;
    return ex ? (float)(ex - 127) : 0.f;
  }
  __device__ __forceinline__ static Lv zero() { return make_float2(0.f, 0.f); }
  __device__ __forceinline__ static float hi(Lv a) { return a.x; }
  __device__ __forceinline__ static float lo(Lv a) { return a.y; }
  __device__ __forceinline__ static Lv mk(float h, float l) { return make_float2(h, l); }
  // a - t as a renormalised pair
  __device__ __forceinline__ static Lv sub(Lv a, float t) {
    const float s = a.x - t;
    const float bb = s - a.x;
    const float err = (a.x - (s - bb)) + (-t - bb);
    float lo = err + a.y;
    const float hi = s + lo;
    lo = lo - (hi - s);
    return make_float2(hi, lo);
  }
  // (b + z, b - z) of two level pairs, the hi parts added with their
  // rounding error kept (b none: none)
  __device__ __forceinline__ static Beta beta_of(Lv b, Lv z) {
    if (!(b.x > 0.5f * kNone)) return make_float4(kNone, 0.f, kNone, 0.f);
    const float s = b.x + z.x, bs = s - b.x, e = (b.x - (s - bs)) + (z.x - bs);
    const float d = b.x - z.x, bd = d - b.x, f = (b.x - (d - bd)) + (-z.x - bd);
    return make_float4(s, e + (b.y + z.y), d, f + (b.y - z.y));
  }
  // a + b for level pairs (b may be none)
  __device__ __forceinline__ static Lv add_lv(Lv a, Lv b) {
    const float s = a.x + b.x, bs = s - a.x, e = (a.x - (s - bs)) + (b.x - bs);
    return make_float2(s, e + (a.y + b.y));
  }
  // a float64 value as a level pair
  __device__ __forceinline__ static Lv from_double(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
  }
  // a - t with the rounding error of the hi part moved to lo (exact when
  // |a.x| >= |t|, the case of a division step near the fixed point); the pair
  // is not renormalised
  __device__ __forceinline__ static Lv sub_fast(Lv a, float t) {
    const float s = a.x - t;
    return make_float2(s, a.y + ((a.x - s) - t));
  }
  __device__ __forceinline__ static double to_double(Lv a) { return (double)a.x + (double)a.y; }
  // the levels b + z, b - z of float64 values as pairs (b = -inf: none)
  __device__ __forceinline__ static Beta make_beta(double b, double z) {
    if (!(b > -INFINITY)) return make_float4(kNone, 0.f, kNone, 0.f);
    const double p = b + z, m = b - z;
    const float ph = (float)p, mh = (float)m;
    return make_float4(ph, (float)(p - (double)ph), mh, (float)(m - (double)mh));
  }
  __device__ __forceinline__ static void put(float* p, Lv M, float s) { p[0] = M.x; p[1] = M.y; p[2] = s; }
  // a state from global memory written by another CTA (L2, not L1)
  __device__ __forceinline__ static void get(const float* p, Lv& M, float& s) {
    M = make_float2(__ldcg(p), __ldcg(p + 1));
    s = __ldcg(p + 2);
  }
  // a state from shared memory
  __device__ __forceinline__ static void get_s(const float* p, Lv& M, float& s) {
    M = make_float2(p[0], p[1]);
    s = p[2];
  }
  __device__ __forceinline__ static Lv shfl_up(Lv a, int o) {
    return make_float2(__shfl_up_sync(0xffffffffu, a.x, o), __shfl_up_sync(0xffffffffu, a.y, o));
  }
  __device__ __forceinline__ static Lv shfl_down(Lv a, int o) {
    return make_float2(__shfl_down_sync(0xffffffffu, a.x, o), __shfl_down_sync(0xffffffffu, a.y, o));
  }
  __device__ __forceinline__ static Lv shfl_idx(Lv a, int l) {
    return make_float2(__shfl_sync(0xffffffffu, a.x, l), __shfl_sync(0xffffffffu, a.y, l));
  }
};

// 2^x in float64 for the scans, table-driven (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989, in base 2): x = n + k/64 + r with n =
// floor(x), k in 0..63 and 0 <= r < 1/64 read off the fixed-point bits of x
// by integer operations; 2^(k/64) from a 64-entry table (exp2_table.h) and
// 2^r = e^t, t = r ln 2 < 0.0109, as its Taylor series to degree 6 (remainder
// below 4e-18 relative); n is added to the binary exponent.  Within about 3
// ulp.  Nine float64 instructions: on GB300 every float64 warp instruction
// occupies its sub-partition's float64 pipe for 64 cycles, so the scans'
// combines are counted in these (a plain range reduction and a degree-13
// series take about eighteen).  Arguments below -1021 (and NaN) give 0,
// above 1023 infinity.
__device__ __forceinline__ double exp2_tab(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((u >> 52) & 0x7ff);
  const bool neg = (u >> 63) != 0;
  if (ex >= 1023 + 11) {   // |x| >= 2048, infinities, NaN
    const bool nan = ex == 0x7ff && (u << 12) != 0;
    return (neg || nan) ? 0.0 : INFINITY;
  }
  if (ex < 1023 - 53) return 1.0;   // |x| < 2^-53
  // |x| 2^52 as an integer (bits below 2^-52 dropped: an error below 2^-52 in x)
  const unsigned long long m = (u & 0xfffffffffffffull) | (1ull << 52);
  const int sh = ex - 1023;   // -53 .. 10
  const unsigned long long X = sh >= 0 ? (m << sh) : (m >> (-sh));
  const long long Xs = neg ? -(long long)X : (long long)X;
  const long long n = Xs >> 52;   // floor(x)
  if (n < -1021) return 0.0;
  if (n > 1023) return INFINITY;
  const unsigned long long F = (unsigned long long)Xs & 0xfffffffffffffull;   // (x - n) 2^52
  const int k = (int)(F >> 46);
  const double r = (double)(long long)(F & 0x3fffffffffffull);   // r 2^52, exact
  const double t = r * (0.69314718055994530942 * 0x1p-52);
  // 1/j! for j = 6 .. 2
  double p = 1.3888888888888888889e-03;
  p = fma(p, t, 8.3333333333333333333e-03);
  p = fma(p, t, 4.1666666666666666667e-02);
  p = fma(p, t, 1.6666666666666666667e-01);
  p = fma(p, t, 0.5);
  p = fma(p, t, 1.0);
  p = fma(p, t, 1.0);
  const double v = __ldg(&kExp2Tab[k]) * p;   // in [1, 2)
  return __longlong_as_double(__double_as_longlong(v) + (n << 52));
}

template <>
struct HT<double> {
  using Lv = double;
  using Beta = double2;  // (beta+, beta-)
  static constexpr int kSt = 2;
  static constexpr double kNone = -1.0e300;
  __device__ __forceinline__ static Lv bp(const Beta& b) { return b.x; }
  __device__ __forceinline__ static Lv bm(const Beta& b) { return b.y; }
  __device__ __forceinline__ static Beta pack(Lv p, Lv m) { return make_double2(p, m); }
  __device__ __forceinline__ static Lv none() { return kNone; }
  __device__ __forceinline__ static bool valid(Lv a) { return a > 0.5 * kNone; }
  __device__ __forceinline__ static double ex2(double x) { return exp2_tab(x); }
  __device__ __forceinline__ static double lg2(double x) { return log2(x); }
  __device__ __forceinline__ static double lg2_acc(double x) { return log2(x); }
  __device__ __forceinline__ static double diff(Lv a, Lv b) { return a - b; }
  __device__ __forceinline__ static double sum_minus(Lv a, Lv b, Lv c, double k) { return ((a + b) + k) - c; }
  __device__ __forceinline__ static double mant_exp(double s, double& m) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(s);
    const int ex = (int)((b >> 52) & 0x7ffull);
    m = ex ? __longlong_as_double((long long)((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull)) : 0.0;
    return ex ? (double)(ex - 1023) : 0.0;
  }
  __device__ __forceinline__ static Lv zero() { return 0.0; }
  __device__ __forceinline__ static double hi(Lv a) { return a; }
  __device__ __forceinline__ static double lo(Lv) { return 0.0; }
  __device__ __forceinline__ static Lv mk(double h, double) { return h; }
  __device__ __forceinline__ static Lv sub(Lv a, double t) { return a - t; }
  __device__ __forceinline__ static Lv sub_fast(Lv a, double t) { return a - t; }
  __device__ __forceinline__ static Beta beta_of(Lv b, Lv z) {
    if (!(b > 0.5 * kNone)) return make_double2(kNone, kNone);
    return make_double2(b + z, b - z);
  }
  __device__ __forceinline__ static Lv from_double(double v) { return v; }
  __device__ __forceinline__ static Lv add_lv(Lv a, Lv b) { return a + b; }
  __device__ __forceinline__ static double to_double(Lv a) { return a; }
  __device__ __forceinline__ static Beta make_beta(double b, double z) {
    if (!(b > -INFINITY)) return make_double2(kNone, kNone);
    return make_double2(b + z, b - z);
  }
  __device__ __forceinline__ static void put(double* p, Lv M, double s) { p[0] = M; p[1] = s; }
  __device__ __forceinline__ static void get(const double* p, Lv& M, double& s) {
    M = __ldcg(p);
    s = __ldcg(p + 1);
  }
  __device__ __forceinline__ static void get_s(const double* p, Lv& M, double& s) {
    M = p[0];
    s = p[1];
  }
  __device__ __forceinline__ static Lv shfl_up(Lv a, int o) { return __shfl_up_sync(0xffffffffu, a, o); }
  __device__ __forceinline__ static Lv shfl_down(Lv a, int o) { return __shfl_down_sync(0xffffffffu, a, o); }
  __device__ __forceinline__ static Lv shfl_idx(Lv a, int l) { return __shfl_sync(0xffffffffu, a, l); }
};

// log-sum state: value s * 2^M (s = 0: empty)
template <class R>
struct St {
  typename HT<R>::Lv M;
  R s;
};

template <class R>
__device__ __forceinline__ St<R> st_empty() {
  return {HT<R>::none(), R(0)};
}

// a (+) b
template <class R>
__device__ __forceinline__ St<R> st_comb(const St<R>& a, const St<R>& b) {
  using H = HT<R>;
  const R d = H::diff(b.M, a.M);
  const bool gt = d > R(0);
  const R e = H::ex2(-fabs(d));
  St<R> r;
  r.s = gt ? fma(a.s, e, b.s) : fma(b.s, e, a.s);
  r.M = gt ? b.M : a.M;
  return r;
}

// a (+) 2^lv (lv = none adds nothing)
template <class R>
__device__ __forceinline__ void st_term(St<R>& a, typename HT<R>::Lv lv) {
  using H = HT<R>;
  const R d = H::diff(lv, a.M);
  const bool gt = d > R(0);
  const R e = H::ex2(-fabs(d));
  a.s = gt ? fma(a.s, e, R(1)) : a.s + e;
  a.M = gt ? lv : a.M;
}

// Float64 states keep M a whole number of bits, so that the factor between
// two states is an exact power of two, built from the bits of the
// difference of their levels: a combine is one float64 fused multiply-add
// and an add instead of a 2^x (GB300 runs float64 at a 64th of the float32
// rate, and the scans chain their combines).  A term 2^lv enters as
// 2^(lv - floor lv) 2^floor(lv).  The value s 2^M of a state is the same as
// with a fractional M; s then lies in [1, 2 n) for n terms.

// 2^-|d| for a whole number d (0 when |d| > 1022, and for d = +-none)
__device__ __forceinline__ double pow2_neg(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const int ex = (int)((u >> 52) & 0x7ff);
  if (ex < 1023) return 1.0;            // d = 0
  if (ex >= 1023 + 10) return 0.0;      // |d| >= 1024
  const int k = (int)(((u & 0xfffffffffffffull) | (1ull << 52)) >> (52 - (ex - 1023)));   // |d|
  return k > 1022 ? 0.0 : __longlong_as_double((long long)(1023 - k) << 52);
}

// d > 0 from the bits of d (no float64 instruction)
__device__ __forceinline__ bool pos_bits(double d) {
  const long long b = __double_as_longlong(d);
  return b > 0;   // sign clear and not +0 (NaN does not occur)
}

// 2^x = v 2^n with n = floor(x) and v = 2^(x - n) in [1, 2), by the steps of
// exp2_tab on the fraction; v = 0 (and n = 0) for a level below -2^900 (none)
__device__ __forceinline__ double exp2_split(double x, double& n) {
  const unsigned long long ux = (unsigned long long)__double_as_longlong(x);
  if ((ux >> 63) && ((ux >> 52) & 0x7ff) >= 1023 + 900) {
    n = 0.0;
    return 0.0;
  }
  n = floor(x);
  const double f = x - n;   // in [0, 1], exact unless it rounds up to 1 (x just below a whole number)
  const unsigned long long u = (unsigned long long)__double_as_longlong(f);
  const int ex = (int)((u >> 52) & 0x7ff);
  if (ex < 1023 - 53) return 1.0;   // f < 2^-53
  if (ex >= 1023) {                 // f = 1
    n += 1.0;
    return 1.0;
  }
  const unsigned long long F = ((u & 0xfffffffffffffull) | (1ull << 52)) >> (1023 - ex);   // f 2^52
  const int k = (int)(F >> 46);
  const double r = (double)(long long)(F & 0x3fffffffffffull);
  const double t = r * (0.69314718055994530942 * 0x1p-52);
  double p = 1.3888888888888888889e-03;
  p = fma(p, t, 8.3333333333333333333e-03);
  p = fma(p, t, 4.1666666666666666667e-02);
  p = fma(p, t, 1.6666666666666666667e-01);
  p = fma(p, t, 0.5);
  p = fma(p, t, 1.0);
  p = fma(p, t, 1.0);
  return __ldg(&kExp2Tab[k]) * p;
}

template <>
__device__ __forceinline__ St<double> st_comb(const St<double>& a, const St<double>& b) {
  const double d = b.M - a.M;   // a whole number, or +-none
  const bool gt = pos_bits(d);
  const double e = pow2_neg(d);
  St<double> r;
  r.s = gt ? fma(a.s, e, b.s) : fma(b.s, e, a.s);
  r.M = gt ? b.M : a.M;
  return r;
}

template <>
__device__ __forceinline__ void st_term(St<double>& a, double lv) {
  double n;
  const double v = exp2_split(lv, n);
  const double d = n - a.M;
  const bool gt = __double_as_longlong(v) != 0 && pos_bits(d);
  const double e = pow2_neg(d);
  a.s = gt ? fma(a.s, e, v) : fma(v, e, a.s);
  a.M = gt ? n : a.M;
}

template <class R>
__device__ __forceinline__ St<R> st_shfl_up(const St<R>& a, int o) {
  return {HT<R>::shfl_up(a.M, o), __shfl_up_sync(0xffffffffu, a.s, o)};
}
template <class R>
__device__ __forceinline__ St<R> st_shfl_down(const St<R>& a, int o) {
  return {HT<R>::shfl_down(a.M, o), __shfl_down_sync(0xffffffffu, a.s, o)};
}
template <class R>
__device__ __forceinline__ St<R> st_shfl_idx(const St<R>& a, int l) {
  return {HT<R>::shfl_idx(a.M, l), __shfl_sync(0xffffffffu, a.s, l)};
}

template <class R>
struct HalfArgs {
  using Beta = typename HT<R>::Beta;
  const uint32_t* tbits;   // merged type bits (bit set = x point)
  const int32_t* tile_x0;  // C + 1: x points before each tile
  int64_t L;               // merged points
  int C;                   // tiles
  int o_is_x;              // 1: outputs at x (K psi), 0: outputs at y (K^T phi)
  const Beta* bO;          // O levels (frames)
  const typename HT<R>::Lv* lmO;   // O log2 masses (none for a zero mass); H_POT / H_ERR
  const double* mO;                // H_ERR, float64 kernels: the O masses (may be null)
  Beta* bO_out;            // new O levels (H_POT)
  const Beta* bW;          // W levels
  double* out;             // H_LOG / H_LIN: per O point
  const R* carry_in;       // 2 kSt per tile: forward state entering it | backward state entering it
  R* agg_out;              // 2 kSt per tile: tile aggregates (forward beta+ | backward beta-)
  R* carry_out;            // 2 kSt per tile: carries of the target application (last CTA)
  double* part;            // per tile: partial error sum
  double* scal;            // [0] error of the last check
  int32_t* ctrl;           // [0] ticket [1] done [2] iteration [3] iterations at exit [4] converged
  double tol;
  int64_t maxit;
  // H_RAW: W levels from rawW (cost units) at positions posW, O frames 0 at
  // posO, and the output ln of the product plus rawO / eps
  const double* rawW;
  const double* rawO;
  const double* posW;
  const double* posO;
  double scale;       // 1 / (eps ln 2)
  double inv_eps;
  // H_LINES: lines of the launch; line l's node i sits at grid index
  // (l % inner) + (l / inner) * inner * nk + i * inner
  int lines;
  int pair;                        // lines of exactly two tiles: each tile forms its carry
                                   // from the other tile's W points (no aggregate launch)
  int64_t inner, nk;
  const typename HT<R>::Lv* gW;    // W log-weights on the grid (bits)
  const typename HT<R>::Lv* gO;    // O log-weights on the grid (frames; H_POT / H_ERR)
  typename HT<R>::Lv* gO_out;      // new O log-weights (H_POT)
  typename HT<R>::Lv* q_out;       // H_QOUT: log2 of the product at the O nodes
  const typename HT<R>::Lv* zW;    // positions of the axis nodes in bits (W, O side)
  const typename HT<R>::Lv* zO;
  const typename HT<R>::Lv* zlogW; // H_ZLOG: log2(z - z_min) of the W axis nodes (bits)
  int64_t grid;                    // H_FB: grid points (the upper sums follow the lower ones)
  // H_BATCH: problem b owns the packed tiles itile[b] .. itile[b+1] - 1 (the
  // first point of each on a tile boundary) and the points ioffx[b] ..
  // ioffx[b+1] - 1 of x (ioffy of y); tile_x0 holds, from itile[b] + b on,
  // the x points of problem b before each of its tile boundaries; the
  // launch handles the acount tiles listed in alist
  const int32_t* tinst;
  const int32_t* itile;
  const int64_t* ioffx;
  const int64_t* ioffy;
  const int32_t* alist;
  const int32_t* acount;
};

// The template parameter E of the kernel is the tile kind of tile_threads:
// points per thread, or kElemsSmall for 64-thread tiles of one point each.
template <class R, int E>
constexpr int half_threads() { return tile_threads(E); }
template <int E>
constexpr int half_e() { return tile_elems(E); }

__device__ __forceinline__ int hslot(int t) { return t + (t >> 5); }

template <class R, int E>
struct HalfSmem {
  using Lv = typename HT<R>::Lv;
  static constexpr int NT = half_threads<R, E>();
  static constexpr int T = half_e<E>() * NT;
  static constexpr int kSlots = NT + NT / 32;
  static_assert((NT & (NT - 1)) == 0 && NT >= 64 && NT <= 256, "own[] holds thread indices as bytes");
  Lv pfM[T];      // W phase: running prefix states of the owning thread (levels ...
  R pfs[T];       //   ... and mantissas)
  Lv sfM[T];      // running suffix states
  R sfs[T];
  // per thread: run totals, then entry states ([0] forward, [1] backward);
  // level hi / lo parts and mantissas as separate 4-byte arrays so that the
  // raking lanes (8 consecutive slots each, padded) hit distinct banks
  R slh[2][kSlots];
  R sll[2][kSlots];
  R sls[2][kSlots];
  int16_t zl[T];        // per O point of the tile: W points of the tile before it
  uint8_t own[T];       // per W point of the tile: the thread whose run holds it
  double red[NT / 32];
  int iscan[NT / 32];
  int last;
  typename HT<R>::Lv totM;   // launch tail: the running carry of a chunk of tiles
  R tots;
};


template <class R, int E>
__device__ __forceinline__ void hslot_put(HalfSmem<R, E>& sm, int dir, int t, const St<R>& a) {
  const int i = hslot(t);
  sm.slh[dir][i] = HT<R>::hi(a.M);
  if (sizeof(R) == 4) sm.sll[dir][i] = HT<R>::lo(a.M);
  sm.sls[dir][i] = a.s;
}
template <class R, int E>
__device__ __forceinline__ St<R> hslot_get(const HalfSmem<R, E>& sm, int dir, int t) {
  const int i = hslot(t);
  return {HT<R>::mk(sm.slh[dir][i], sizeof(R) == 4 ? sm.sll[dir][i] : R(0)), sm.sls[dir][i]};
}

// Warps 0 (forward) and 1 (backward): turn the run totals of the threads in the
// slots into entry states: forward, the carry cf and the totals of threads
// 0 .. t-1; backward, the carry cb and the totals of threads t+1 .. end.
template <class R, int E>
__device__ __forceinline__ void hrake_scan(HalfSmem<R, E>& sm, const St<R>& cf, const St<R>& cb) {
  constexpr int kHPer = half_threads<R, E>() / 32;   // slots raked per lane
  const int lane = threadIdx.x & 31;
  const int dir = threadIdx.x >> 5;   // 0 or 1
  St<R> f = st_empty<R>();
#pragma unroll
  for (int k = 0; k < kHPer; ++k) f = st_comb(f, hslot_get(sm, dir, lane * kHPer + k));
  if (dir == 0) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const St<R> u = st_shfl_up(f, o);
      if (lane >= o) f = st_comb(u, f);
    }
    St<R> ex = st_shfl_up(f, 1);
    if (lane == 0) ex = st_empty<R>();
    St<R> st = st_comb(cf, ex);
#pragma unroll
    for (int k = 0; k < kHPer; ++k) {
      const St<R> a = hslot_get(sm, 0, lane * kHPer + k);
      hslot_put(sm, 0, lane * kHPer + k, st);
      st = st_comb(st, a);
    }
  } else {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const St<R> u = st_shfl_down(f, o);
      if (lane + o < 32) f = st_comb(u, f);
    }
    St<R> ex = st_shfl_down(f, 1);
    if (lane == 31) ex = st_empty<R>();
    St<R> st = st_comb(cb, ex);
#pragma unroll
    for (int k = kHPer - 1; k >= 0; --k) {
      const St<R> a = hslot_get(sm, 1, lane * kHPer + k);
      hslot_put(sm, 1, lane * kHPer + k, st);
      st = st_comb(st, a);
    }
  }
}

// Warps 0 and 1: log-sum of the threads' partial states of slot direction 0
// (warp 0) and 1 (warp 1); lane 0 stores it at out + dir * kSt.
template <class R, int E>
__device__ __forceinline__ void hrake_reduce(HalfSmem<R, E>& sm, R* out) {
  constexpr int kHPer = half_threads<R, E>() / 32;   // slots raked per lane
  const int lane = threadIdx.x & 31;
  const int dir = threadIdx.x >> 5;
  St<R> f = st_empty<R>();
#pragma unroll
  for (int k = 0; k < kHPer; ++k) f = st_comb(f, hslot_get(sm, dir, lane * kHPer + k));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f = st_comb(f, st_shfl_down(f, o));
  if (lane == 0) HT<R>::put(out + dir * HT<R>::kSt, f.M, f.s);
}


// Warp dir (0: forward, 1: backward) alone: exclusive scan of the run
// totals in slot direction dir, seeded with seed; the slots receive the entry
// states and (totM, tots) the log-sum of seed and every slot.
template <class R, int E, int dir>
__device__ __forceinline__ void hrake_one(HalfSmem<R, E>& sm, const St<R>& seed) {
  constexpr int kHPer = half_threads<R, E>() / 32;   // slots raked per lane
  const int lane = threadIdx.x & 31;
  St<R> f = st_empty<R>();
#pragma unroll
  for (int k = 0; k < kHPer; ++k) f = st_comb(f, hslot_get(sm, dir, lane * kHPer + k));
  if (dir == 0) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const St<R> u = st_shfl_up(f, o);
      if (lane >= o) f = st_comb(u, f);
    }
  } else {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const St<R> u = st_shfl_down(f, o);
      if (lane + o < 32) f = st_comb(u, f);
    }
  }
  St<R> ex = dir == 0 ? st_shfl_up(f, 1) : st_shfl_down(f, 1);
  if (lane == (dir == 0 ? 0 : 31)) ex = st_empty<R>();
  if (lane == (dir == 0 ? 31 : 0)) {
    const St<R> t = st_comb(seed, f);
    sm.totM = t.M;
    sm.tots = t.s;
  }
  St<R> st = st_comb(seed, ex);
#pragma unroll
  for (int kk = 0; kk < kHPer; ++kk) {
    const int k = dir == 0 ? kk : kHPer - 1 - kk;
    const St<R> a = hslot_get(sm, dir, lane * kHPer + k);
    hslot_put(sm, dir, lane * kHPer + k, st);
    st = st_comb(st, a);
  }
}

// S - 1 for S = 2^x without the cancellation near x = 0: the series of
// e^t - 1, t = x ln 2, for |t| < 0.03 (float32: degree 4, branch-free;
// float64: degree 9, which leaves a relative error below 1e-17, and a
// branch, since near the fixed point every point takes the series and the
// float64 exp2 is skipped), else 2^x - 1
template <class R>
__device__ __forceinline__ R pow2m1(R x) {
  const R t = x * R(0.69314718055994530942);
  if constexpr (sizeof(R) == sizeof(double)) {
    if (fabs(t) < 0.03) {
      double p = 2.7557319223985890653e-06;   // 1/9!
      p = fma(p, t, 2.4801587301587301587e-05);
      p = fma(p, t, 1.9841269841269841270e-04);
      p = fma(p, t, 1.3888888888888888889e-03);
      p = fma(p, t, 8.3333333333333333333e-03);
      p = fma(p, t, 4.1666666666666666667e-02);
      p = fma(p, t, 1.6666666666666666667e-01);
      p = fma(p, t, 0.5);
      p = fma(p, t, 1.0);
      return p * t;
    }
    return HT<R>::ex2(x) - 1.0;
  } else {
    const R p = t * (R(1) + t * (R(0.5) + t * (R(1.0 / 6) + t * R(1.0 / 24))));
    const R q = HT<R>::ex2(x) - R(1);
    return (fabs(t) < R(0.03)) ? p : q;
  }
}

// One tile of a launch: steps 1-3 of the header comment.  Returns false when
// the loop is already done (the launch does nothing).  Per-thread runs have a
// fixed trip count E; indices past a thread's run are clamped to a valid
// point of the tile and its contributions masked, so the loops do not branch.
template <class R, int kFlags, int EK>
__device__ __forceinline__ bool half_unit(const HalfArgs<R>& a, HalfSmem<R, EK>& sm, int unit, bool first) {
  constexpr int E = half_e<EK>();   // points per thread
  using H = HT<R>;
  using Lv = typename H::Lv;
  using Beta = typename H::Beta;
  constexpr int NT = half_threads<R, EK>();
  constexpr int kT = E * NT;
  constexpr bool kAgg = (kFlags & H_AGG) != 0;
  constexpr bool kLines = (kFlags & H_LINES) != 0;
  constexpr bool kProd = (kFlags & (H_LOG | H_LIN | H_QOUT | H_FB)) != 0;
  constexpr bool kDiv = (kFlags & (H_POT | H_ERR)) != 0;
  constexpr bool kBatch = (kFlags & H_BATCH) != 0;
  const int tid = threadIdx.x;

  // The unit's tile: its merged points [k0, kend) in its problem's own
  // numbering (pk0: the packed position of k0 in the type bits), its x and y
  // points, and the index of the first x / y point in the point arrays.
  // Line mode: unit = line * C + tile; grid index of node i of the line:
  // gbase + i * inner.  Batches: unit = entry of the active tile list.
  int line = 0, tile, x0, x1;
  int64_t k0, kend, pk0, xb = 0, yb = 0;
  if constexpr (kBatch) {
    tile = a.alist[unit];
    const int b = a.tinst[tile];
    const int lt = tile - a.itile[b];
    const int32_t* tx = a.tile_x0 + a.itile[b] + b;
    x0 = tx[lt];
    x1 = tx[lt + 1];
    xb = a.ioffx[b];
    yb = a.ioffy[b];
    const int64_t Lb = (a.ioffx[b + 1] - xb) + (a.ioffy[b + 1] - yb);
    k0 = (int64_t)lt * kT;
    kend = min(k0 + (int64_t)kT, Lb);
    pk0 = (int64_t)tile * kT;
  } else {
    line = kLines ? unit / a.C : 0;
    tile = unit - line * a.C;
    x0 = a.tile_x0[tile];
    x1 = a.tile_x0[tile + 1];
    k0 = (int64_t)tile * kT;
    kend = min(k0 + (int64_t)kT, a.L);
    pk0 = k0;
  }
  // per-tile slots of the aggregates, carries and error partials
  const int64_t slot = kBatch ? (int64_t)tile : (int64_t)unit;
  const int64_t inner = kLines ? a.inner : 1;
  const int64_t gbase = kLines ? (line % inner) + (line / inner) * inner * a.nk : 0;
  const int y0 = (int)(k0 - x0), y1 = (int)(kend - x1);
  const int64_t o_start = a.o_is_x ? xb + x0 : yb + y0;
  const int n_o = a.o_is_x ? (x1 - x0) : (y1 - y0);
  const int64_t w_start = a.o_is_x ? yb + y0 : xb + x0;
  const int n_w = a.o_is_x ? (y1 - y0) : (x1 - x0);
  const Beta* bO = a.bO + o_start;
  const Beta* bW = a.bW + w_start;

  // 1. local dividing index of the O points of this thread's merged points
  if (!kAgg) {
    const int64_t segl = k0 + (int64_t)tid * E;
    const int64_t seg = pk0 + (int64_t)tid * E;
    uint32_t omask = 0;
    if (segl < kend) {
      const int64_t nv = kend - segl;
      const uint32_t vmask = nv >= E ? ((1u << E) - 1u) : ((1u << nv) - 1u);
      const uint32_t bits = (a.tbits[seg >> 5] >> (seg & 31)) & ((1u << E) - 1u);
      omask = (a.o_is_x ? bits : ~bits) & vmask;
    }
    int r = block_exclusive_sum<NT>(__popc(omask), sm.iscan);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if ((omask >> e) & 1u) sm.zl[r] = (int16_t)(tid * E + e - r);
      r += (omask >> e) & 1u;
    }
  }
  if (first) {
    griddep_wait();
    if ((kFlags & H_CHECK_DONE) && *(volatile int32_t*)(a.ctrl + 1)) return false;
    griddep_launch_dependents();
  }

  // 2. W phase: running log-sums over this thread's W run
  const int wlo = (int)(((int64_t)tid * n_w) / NT);
  const int qw = (int)(((int64_t)(tid + 1) * n_w) / NT) - wlo;
  St<R> tf = st_empty<R>(), tb = st_empty<R>();
  auto wbeta = [&](int i) -> Beta {
    if constexpr ((kFlags & H_RAW) != 0) {
      return H::make_beta(a.rawW[w_start + i] * a.scale, a.posW[w_start + i] * a.scale);
    } else if constexpr (kLines) {
      Lv b = a.gW[gbase + (int64_t)(w_start + i) * inner];
      if constexpr ((kFlags & H_ZLOG) != 0) b = H::add_lv(b, a.zlogW[w_start + i]);
      return H::beta_of(b, a.zW[w_start + i]);
    } else {
      return bW[i];
    }
  };
  if constexpr (kAgg) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (e < qw) {
        const Beta b = wbeta(wlo + e);
        st_term(tf, H::bp(b));
        st_term(tb, H::bm(b));
      }
    }
    hslot_put(sm, 0, tid, tf);
    hslot_put(sm, 1, tid, tb);
    __syncthreads();
    if (tid < 64) hrake_reduce(sm, a.agg_out + 2 * H::kSt * slot);
    return true;
  } else {
  // longest run of the tile (block-uniform trip count); the loads of a run
  // are all in flight before its chain starts
  const int qwm = (n_w + NT - 1) / NT;
  const int wl = max(n_w - 1, 0);
  Beta bw[E];
#pragma unroll
  for (int e = 0; e < E; ++e)
    if (e < qwm) bw[e] = wbeta(min(wlo + e, wl));
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (e < qwm) {
      const bool v = e < qw;
      st_term(tf, v ? H::bp(bw[e]) : H::none());
      if (v) {
        sm.pfM[wlo + e] = tf.M;
        sm.pfs[wlo + e] = tf.s;
        sm.own[wlo + e] = (uint8_t)tid;
      }
    }
  }
#pragma unroll
  for (int e = E - 1; e >= 0; --e) {
    if (e < qwm) {
      const bool v = e < qw;
      st_term(tb, v ? H::bm(bw[e]) : H::none());
      if (v) {
        sm.sfM[wlo + e] = tb.M;
        sm.sfs[wlo + e] = tb.s;
      }
    }
  }
  const int wlast = max(n_w - 1, 0);
  // O run of this thread
  const int olo = (int)(((int64_t)tid * n_o) / NT);
  const int qo = (int)(((int64_t)(tid + 1) * n_o) / NT) - olo;
  St<R> cf = st_empty<R>(), cb = st_empty<R>();
  if (a.carry_in) {
    const R* c = a.carry_in + 2 * H::kSt * slot;
    H::get(c, cf.M, cf.s);
    H::get(c + H::kSt, cb.M, cb.s);
  }
  if constexpr (kLines) {
    if (a.pair) {
      // A line of two tiles: the carry entering this tile is the log-sum of
      // the other tile's W levels (beta- of tile 1 for tile 0's backward
      // sums, beta+ of tile 0 for tile 1's forward sums), formed here from
      // its W points, a run per thread and one warp's scan of the run totals.
      const int t2 = tile ^ 1;
      const int64_t k0b = (int64_t)t2 * kT, kendb = min(k0b + (int64_t)kT, a.L);
      const int x0b = a.tile_x0[t2], x1b = a.tile_x0[t2 + 1];
      const int y0b = (int)(k0b - x0b), y1b = (int)(kendb - x1b);
      const int wsb = a.o_is_x ? y0b : x0b;
      const int nwb = a.o_is_x ? (y1b - y0b) : (x1b - x0b);
      const int lo2 = (int)(((int64_t)tid * nwb) / NT);
      const int q2 = (int)(((int64_t)(tid + 1) * nwb) / NT) - lo2;   // at most E
      St<R> pt = st_empty<R>();
#pragma unroll
      for (int e = 0; e < E; ++e) {
        if (e < q2) {
          const Beta b = wbeta(wsb + lo2 + e - (int)w_start);
          st_term(pt, tile == 0 ? H::bm(b) : H::bp(b));
        }
      }
      hslot_put(sm, 0, tid, pt);
      __syncthreads();
      if (tid < 32) hrake_one<R, EK, 0>(sm, st_empty<R>());
      __syncthreads();
      const St<R> tot{sm.totM, sm.tots};
      if (tile == 0) cb = tot;
      else cf = tot;
    }
  }
  hslot_put(sm, 0, tid, tf);
  hslot_put(sm, 1, tid, tb);
  __syncthreads();
  if (tid < 64) hrake_scan(sm, cf, cb);
  __syncthreads();

  // 3. O phase (block-uniform trip count; a thread past its run repeats its
  // last point with the results masked)
  R err = R(0);
  St<R> nf = st_empty<R>(), nb = st_empty<R>();
  const int qom = (n_o + NT - 1) / NT;
  const int ol = max(n_o - 1, 0);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (e >= qom) break;
    const bool v = e < qo;
    const int j = min(olo + e, ol);
    Beta bo;
    Lv lm;
    const int64_t gi = gbase + (int64_t)(o_start + j) * inner;   // line mode: grid index
    if constexpr ((kFlags & H_RAW) != 0) bo = H::make_beta(0.0, a.posO[o_start + j] * a.scale);
    else if constexpr (kLines) bo = H::beta_of(kDiv ? a.gO[gi] : H::zero(), a.zO[o_start + j]);
    else bo = bO[j];
    if constexpr (kDiv) lm = kLines ? a.lmO[gi] : a.lmO[o_start + j];
    const int z = sm.zl[j];
    // forward: the W points before z (entry of the owner of W point z-1
    // and its local prefix); backward: the W points from z on
    const int i1 = max(z - 1, 0), i2 = min(z, wlast);
    // (a tile without W points leaves own[] stale or unset; Fo / Bo are not
    // used then, and the mask keeps the slot index inside the slot arrays)
    const St<R> Fo = st_comb(hslot_get(sm, 0, sm.own[i1] & (NT - 1)), St<R>{sm.pfM[i1], sm.pfs[i1]});
    const St<R> Bo = st_comb(hslot_get(sm, 1, sm.own[i2] & (NT - 1)), St<R>{sm.sfM[i2], sm.sfs[i2]});
    const St<R> F = z > 0 ? Fo : cf;
    const St<R> B = z < n_w ? Bo : cb;
    {
      const Lv op = H::bp(bo), om = H::bm(bo);
      if constexpr ((kFlags & H_QOUT) != 0 && sizeof(R) == 4) {
        // log2 of p + q with the O frame 0 (levels +-Z) as a level pair, in
        // float arithmetic: each block's level, with the binary exponent of
        // its mantissa sum joined exactly, then the larger one plus log2 of
        // the mantissas in its frame
        R m1, m2;
        const R k1 = H::mant_exp(F.s, m1), k2 = H::mant_exp(B.s, m2);
        const bool e1 = F.s > R(0) && H::valid(F.M), e2 = B.s > R(0) && H::valid(B.M);
        const Lv A1 = H::add_lv(H::add_lv(F.M, om), H::mk(k1, R(0)));
        const Lv A2 = H::add_lv(H::add_lv(B.M, op), H::mk(k2, R(0)));
        const R D = e1 && e2 ? H::diff(A2, A1) : (e1 ? R(-1000) : R(1000));
        const bool g2 = D > R(0);
        const R t = H::lg2_acc(g2 ? fma(m1, H::ex2(-D), m2) : fma(m2, H::ex2(D), m1));
        if (v) a.q_out[gi] = (e1 || e2) ? H::sub(g2 ? A2 : A1, -t) : H::none();
      } else if constexpr (kProd) {
        // ln of p + q with the O frame 0 (levels +-Z), in float64
        const double a1 = H::to_double(F.M) + H::to_double(om);
        const double a2 = H::to_double(B.M) + H::to_double(op);
        const bool g1 = a1 >= a2;
        const double big = g1 ? a1 : a2;
        const R d = (R)(g1 ? a2 - a1 : a1 - a2);
        const R sb = g1 ? F.s : B.s, so = g1 ? B.s : F.s;
        const bool none = !(sb > R(0)) || big < 0.5 * (double)H::kNone;
        const double l2 = big + (double)H::lg2_acc(fma(so, H::ex2(d), sb));
        if constexpr ((kFlags & H_FB) != 0) {
          if (v) {
            a.out[gi] = (F.s > R(0) && a1 > 0.5 * (double)H::kNone) ? a1 + (double)H::lg2_acc(F.s) : -INFINITY;
            a.out[a.grid + gi] = (B.s > R(0) && a2 > 0.5 * (double)H::kNone) ? a2 + (double)H::lg2_acc(B.s) : -INFINITY;
          }
        } else if constexpr ((kFlags & H_QOUT) != 0) {
          if (v) a.q_out[gi] = none ? H::none() : H::from_double(l2);
        } else {
          double val;
          if constexpr ((kFlags & H_LOG) != 0) val = none ? -INFINITY : 0.69314718055994530942 * l2;
          else val = none ? 0.0 : exp2(l2);
          if constexpr ((kFlags & H_RAW) != 0) val += a.rawO[o_start + j] * a.inv_eps;
          if (v) a.out[o_start + j] = val;
        }
      } else {
        const bool has_mass = H::valid(lm);
        const Lv c = has_mass ? lm : H::zero();
        // delta = log2 S - c, S = 2^{beta-} P + 2^{beta+} Q; the binary
        // exponents of the mantissa sums join the level sums before rounding,
        // so the dominant part is near 0 and keeps full float precision
        R m1, m2;
        const R k1 = H::mant_exp(F.s, m1), k2 = H::mant_exp(B.s, m2);
        const R a1 = H::sum_minus(F.M, om, c, k1);
        const R a2 = H::sum_minus(B.M, op, c, k2);
        const R dd = a1 - a2;
        const bool g1 = dd > R(0);
        const R ed = H::ex2(-fabs(dd));
        const R big = g1 ? a1 : a2;
        const R mb = g1 ? m1 : m2, mo = g1 ? m2 : m1;
        const R delta = big + H::lg2_acc(fma(mo, ed, mb));
        if constexpr ((kFlags & H_ERR) != 0) {
          // the mass mu_k: 2^{log2 mu} (float32), or the float64 mass itself
          // where the plan passes it (a float64 exp2 saved per point)
          R mu;
          if constexpr (sizeof(R) == sizeof(double))
            mu = a.mO ? a.mO[kLines ? gi : o_start + j] : H::ex2(H::hi(lm));
          else
            mu = H::ex2(H::hi(lm));
          const R term = has_mass ? mu * fabs(pow2m1(delta)) : H::ex2(delta);
          err += v ? term : R(0);
        }
        if constexpr ((kFlags & H_POT) != 0) {
          const bool ok = v && has_mass && delta > R(0.5) * H::kNone;
          if constexpr (kLines) {
            if (v) a.gO_out[gi] = ok ? H::sub_fast(a.gO[gi], delta) : H::none();
          } else {
          const Lv np = ok ? H::sub_fast(op, delta) : H::none();
          const Lv nm = ok ? H::sub_fast(om, delta) : H::none();
          if (v) a.bO_out[o_start + j] = H::pack(np, nm);
          if constexpr ((kFlags & H_NEXT) != 0) {
            // the tile aggregate of the next application (new levels)
            st_term(nf, np);
            st_term(nb, nm);
          }
          }
        }
      }
    }
  }

  if constexpr ((kFlags & H_ERR) != 0) {
    const double e64 = warp_sum((double)err);
    if ((tid & 31) == 0) sm.red[tid >> 5] = e64;
  }
  __syncthreads();   // the entry states in the slots are no longer read
  if constexpr ((kFlags & H_ERR) != 0) {
    if (tid == 0) {
      double tot = 0.0;
#pragma unroll
      for (int w = 0; w < NT / 32; ++w) tot += sm.red[w];
      a.part[slot] = tot;
    }
  }
  if constexpr ((kFlags & H_NEXT) != 0) {
    hslot_put(sm, 0, tid, nf);
    hslot_put(sm, 1, tid, nb);
    __syncthreads();
    if (tid < 64) hrake_reduce(sm, a.agg_out + 2 * H::kSt * slot);
  }
  return true;
  }
}

// Last CTA: carries of every tile from the tile aggregates (forward: the
// log-sum of the tiles before it; backward: of the tiles after it).  Chunks
// of E tiles per thread are staged in the (now free) prefix / suffix arrays
// with coalesced loads, eight in flight per thread; the state leaving a chunk
// enters the next one in each direction.
template <class R, int E>
__device__ __forceinline__ void half_stage(const HalfArgs<R>& a, R* buf, int c0, int nq) {
  constexpr int kS2 = 2 * HT<R>::kSt;
  const R* src = a.agg_out + kS2 * (int64_t)c0;
  const int nv = kS2 * nq;
  constexpr int NT = half_threads<R, E>();
#pragma unroll 1
  for (int r0 = threadIdx.x; r0 < nv; r0 += 8 * NT) {
    R v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int i = r0 + k * NT;
      v[k] = i < nv ? __ldcg(src + i) : R(0);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int i = r0 + k * NT;
      if (i < nv) buf[i] = v[k];
    }
  }
}

template <class R, int E, int dir>
__device__ __forceinline__ void half_carry_chunk(const HalfArgs<R>& a, HalfSmem<R, E>& sm, const R* buf, int c0,
                                                 int nq, St<R>& run) {
  using H = HT<R>;
  constexpr int kS = H::kSt;
  constexpr int kQ = half_e<E>();
  const int tid = threadIdx.x;
  const int j0 = tid * kQ;
  St<R> f = st_empty<R>();
#pragma unroll 1
  for (int k = 0; k < kQ; ++k) {
    const int j = j0 + k;
    if (j < nq) {
      St<R> u;
      H::get_s(buf + 2 * kS * j + dir * kS, u.M, u.s);
      f = st_comb(f, u);
    }
  }
  hslot_put(sm, dir, tid, f);
  __syncthreads();
  if ((tid >> 5) == dir) hrake_one<R, E, dir>(sm, run);
  __syncthreads();
  St<R> st = hslot_get(sm, dir, tid);
#pragma unroll 1
  for (int kk = 0; kk < kQ; ++kk) {
    const int k = dir == 0 ? kk : kQ - 1 - kk;
    const int j = j0 + k;
    if (j < nq) {
      H::put(a.carry_out + 2 * kS * (int64_t)(c0 + j) + dir * kS, st.M, st.s);
      St<R> u;
      H::get_s(buf + 2 * kS * j + dir * kS, u.M, u.s);
      st = st_comb(st, u);
    }
  }
  run = {sm.totM, sm.tots};
}

// Both directions of one chunk that holds every tile (no running state
// enters it): each thread forms the forward and backward log-sums of its kQ
// tiles, warps 0 and 1 scan the two directions at the same time (as a
// tile's W phase does), and each thread writes its tiles' carries.
template <class R, int E>
__device__ __forceinline__ void half_carry_chunk2(const HalfArgs<R>& a, HalfSmem<R, E>& sm, const R* buf, int nq) {
  using H = HT<R>;
  constexpr int kS = H::kSt;
  constexpr int kQ = half_e<E>();
  const int tid = threadIdx.x;
  const int j0 = tid * kQ;
  St<R> f = st_empty<R>(), b = st_empty<R>();
#pragma unroll 1
  for (int k = 0; k < kQ; ++k) {
    const int j = j0 + k;
    if (j < nq) {
      St<R> u, w;
      H::get_s(buf + 2 * kS * j, u.M, u.s);
      H::get_s(buf + 2 * kS * j + kS, w.M, w.s);
      f = st_comb(f, u);
      b = st_comb(b, w);
    }
  }
  hslot_put(sm, 0, tid, f);
  hslot_put(sm, 1, tid, b);
  __syncthreads();
  if (tid < 64) hrake_scan(sm, st_empty<R>(), st_empty<R>());
  __syncthreads();
  St<R> sf = hslot_get(sm, 0, tid), sb = hslot_get(sm, 1, tid);
#pragma unroll 1
  for (int kk = 0; kk < kQ; ++kk) {
    const int jf = j0 + kk, jb = j0 + kQ - 1 - kk;
    if (jf < nq) {
      H::put(a.carry_out + 2 * kS * (int64_t)jf, sf.M, sf.s);
      St<R> u;
      H::get_s(buf + 2 * kS * jf, u.M, u.s);
      sf = st_comb(sf, u);
    }
    if (jb < nq) {
      H::put(a.carry_out + 2 * kS * (int64_t)jb + kS, sb.M, sb.s);
      St<R> w;
      H::get_s(buf + 2 * kS * jb + kS, w.M, w.s);
      sb = st_comb(sb, w);
    }
  }
}

// Last CTA, line mode: each thread scans the tiles of whole lines (a line
// spans a few tiles); a line starts and ends empty.
template <class R>
__device__ void half_carries_lines(const HalfArgs<R>& a) {
  using H = HT<R>;
  constexpr int kS = H::kSt;
  const int C = a.C;
#pragma unroll 1
  for (int l = threadIdx.x; l < a.lines; l += blockDim.x) {
    const int64_t u0 = (int64_t)l * C;
    St<R> st = st_empty<R>();
#pragma unroll 1
    for (int t = 0; t < C; ++t) {
      H::put(a.carry_out + 2 * kS * (u0 + t), st.M, st.s);
      St<R> u;
      H::get(a.agg_out + 2 * kS * (u0 + t), u.M, u.s);
      st = st_comb(st, u);
    }
    st = st_empty<R>();
#pragma unroll 1
    for (int t = C - 1; t >= 0; --t) {
      H::put(a.carry_out + 2 * kS * (u0 + t) + kS, st.M, st.s);
      St<R> u;
      H::get(a.agg_out + 2 * kS * (u0 + t) + kS, u.M, u.s);
      st = st_comb(st, u);
    }
  }
}

template <class R, int E>
__device__ void half_carries(const HalfArgs<R>& a, HalfSmem<R, E>& sm) {
  constexpr int K = half_e<E>() * half_threads<R, E>();   // tiles per chunk
  static_assert(sizeof(sm.pfM) + sizeof(sm.pfs) + sizeof(sm.sfM) + sizeof(sm.sfs) >=
                    sizeof(R) * 2 * HT<R>::kSt * K, "staging");
  R* buf = reinterpret_cast<R*>(sm.pfM);   // pfM, pfs, sfM, sfs are adjacent
  const int C = a.C;
  if (C <= 32) {
    // a few tiles: warp 0 scans the forward aggregates and warp 1 the
    // backward ones at the same time, one tile per lane (five shuffle
    // levels instead of the chunked rake; float64 combines on GB300 cost
    // their pipe time per warp instruction, so the depth is what counts)
    using H = HT<R>;
    constexpr int kS = H::kSt;
    const int tid = threadIdx.x, lane = tid & 31, dir = tid >> 5;
    if (tid < 64) {
      const int t = dir == 0 ? lane : C - 1 - lane;   // tile of this lane (dir 1: right to left)
      const bool in = lane < C;
      St<R> inc = st_empty<R>();
      if (in) H::get(a.agg_out + 2 * kS * (int64_t)t + dir * kS, inc.M, inc.s);
      for (int o = 1; o < C; o <<= 1) {   // (C is uniform: whole levels are skipped)
        const St<R> u = st_shfl_up(inc, o);
        if (lane >= o) inc = st_comb(u, inc);
      }
      St<R> ex = st_shfl_up(inc, 1);
      if (lane == 0) ex = st_empty<R>();
      if (in) H::put(a.carry_out + 2 * kS * (int64_t)t + dir * kS, ex.M, ex.s);
    }
    return;
  }
  const int nch = (C + K - 1) / K;
  if (nch == 1) {
    __syncthreads();
    half_stage<R, E>(a, buf, 0, C);
    __syncthreads();
    half_carry_chunk2<R, E>(a, sm, buf, C);
    return;
  }
  St<R> runF = st_empty<R>(), runB = st_empty<R>();
#pragma unroll 1
  for (int ch = 0; ch < nch; ++ch) {
    const int c0 = ch * K, nq = min(K, C - c0);
    __syncthreads();
    half_stage<R, E>(a, buf, c0, nq);
    __syncthreads();
    half_carry_chunk<R, E, 0>(a, sm, buf, c0, nq, runF);
  }
#pragma unroll 1
  for (int ch = nch - 1; ch >= 0; --ch) {
    const int c0 = ch * K, nq = min(K, C - c0);
    __syncthreads();
    half_stage<R, E>(a, buf, c0, nq);
    __syncthreads();
    half_carry_chunk<R, E, 1>(a, sm, buf, c0, nq, runB);
  }
}

// Last CTA: carries of the next launch, the float64 error sum, the loop
// control.  Runs once per launch on one SM: loops stay rolled.
template <class R, int kFlags, int E>
__device__ void half_finish(const HalfArgs<R>& a, HalfSmem<R, E>& sm, int units) {
  const int tid = threadIdx.x;
  double ep = 0.0;
  if (kFlags & H_ERR) {
#pragma unroll 4
    for (int i = tid; i < units; i += (int)blockDim.x) ep += __ldcg(a.part + i);
  }
  if (kFlags & (H_NEXT | H_AGG)) {
    if (kFlags & H_LINES) half_carries_lines<R>(a);
    else half_carries<R, E>(a, sm);
  }
  double errsum = 0.0;
  if (kFlags & H_ERR) {
    ep = warp_sum(ep);
    __syncthreads();
    if ((tid & 31) == 0) sm.red[tid >> 5] = ep;
    __syncthreads();
#pragma unroll
    for (int w = 0; w < half_threads<R, E>() / 32; ++w) errsum += sm.red[w];
  }
  if (tid == 0) {
    int32_t* c = a.ctrl;
    if (kFlags & H_ERR) {
      a.scal[0] = errsum;
      if (errsum <= a.tol) {
        c[1] = 1;
        c[3] = c[2];
        c[4] = 1;
      }
    }
    if ((kFlags & H_ITER_END) && !c[1]) {
      c[2] += 1;
      if ((int64_t)c[2] >= a.maxit) {
        c[1] = 1;
        c[3] = c[2];
      }
    }
    c[0] = 0;
  }
}

template <class R, int E>
__device__ __forceinline__ bool half_last_cta(int32_t* ticket, int G, HalfSmem<R, E>& sm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const int t = atomicAdd(ticket, 1);
    sm.last = (t == G - 1);
  }
  __syncthreads();
  if (sm.last) __threadfence();
  return sm.last != 0;
}

// resident CTAs per SM the registers are budgeted for (float32)
#ifndef FINOM_HALF_MINB8
#define FINOM_HALF_MINB8 3
#endif
template <class R, int E>
constexpr int half_min_blocks() {
  return sizeof(R) != 4 ? 1 : (E >= 8 ? FINOM_HALF_MINB8 : (E == 4 ? 3 : (E == kElemsSmall ? 8 : 4)));
}

// Persistent CTAs: CTA b handles the tiles b, b + G, b + 2G, ... (G = grid
// size); the last CTA to finish (ticket ctrl[0]) runs half_finish.
template <class R, int kFlags, int E>
__global__ void __launch_bounds__(half_threads<R, E>(), half_min_blocks<R, E>()) k_half(HalfArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  HalfSmem<R, E>& sm = *reinterpret_cast<HalfSmem<R, E>*>(smem_raw);
  if constexpr ((kFlags & H_BATCH) != 0) {
    // the active list and the done flag come from the preceding launch
    griddep_wait();
    if (*(volatile int32_t*)(a.ctrl + 1)) return;   // every problem retired
    griddep_launch_dependents();
    const int units = *(volatile const int32_t*)a.acount;
    for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
      half_unit<R, kFlags, E>(a, sm, unit, false);
      __syncthreads();
    }
    return;
  }
  const int units = (kFlags & H_LINES) ? a.lines * a.C : a.C;
  for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
    if (!half_unit<R, kFlags, E>(a, sm, unit, unit == (int)blockIdx.x)) return;   // the loop is done
    __syncthreads();
  }
  griddep_wait();   // (a no-op after the first unit's wait)
  if (half_last_cta<R, E>(a.ctrl, (int)gridDim.x, sm)) half_finish<R, kFlags, E>(a, sm, units);
}

}  // namespace finom
