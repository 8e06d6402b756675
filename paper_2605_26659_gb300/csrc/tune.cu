// Tile-size tuning of 1D plans: points per thread of the fused half-step
// kernel by size bucket and precision, and the autotuner that measures it.
//
// The kernel's tile is kThreads threads x E points, or for E = kElemsSmall
// 64 threads x 1 point.  Large problems want the full tile (E = kElems:
// fewer tiles, fewer carries, longer per-thread runs); small ones want more,
// smaller tiles, so that a problem of a few thousand points spreads over
// more SMs (float64 arithmetic on one SM is slow) and each tile's serial
// chains are shorter.  The table maps the bucket
// ceil(log2(N + M)) to E; finom_plan reads it.  finom_autotune times a few
// Sinkhorn iterations of a synthetic problem of the bucket's size for every
// E and installs the fastest; finom_tune_set / finom_tune_get let a caller
// persist and restore the table.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "finom_internal.h"

namespace finom {
namespace {

constexpr int kBuckets = 40;
std::mutex g_tune_mu;

// Defaults from a tuning run on GB300 (finom_autotune, 64 iterations per
// candidate, buckets 2^10 .. 2^22; E = -1 is the 64-point tile).  float64:
// 2^10-2^13 take E = -1 (24.9-39.8 us per iteration against 40.9-41.9 with
// E = 1 and 61.6-112.6 with E = 8), 2^14-2^15 E = 1, 2^16 E = 2, 2^17 E = 4,
// from 2^18 on E = 8.  float32: 2^10-2^12 E = -1 (9.7-10.5 us against
// 11.0-11.3 with E = 1), 2^13 E = 1, 2^14 E = 2, 2^15 E = 4, 2^16 E = 2,
// 2^17-2^20 E = 4, from 2^21 on E = 8.  Smaller buckets take E = -1, larger
// ones E = 8.
struct Table {
  int e[2][kBuckets];
  int batch[2] = {kElems, kElems};   // batch plans (finom_tune_set_batch)
  Table() {
    //                           2^10 .. 2^22
    const int f64[13] = {kElemsSmall, kElemsSmall, kElemsSmall, kElemsSmall, 1, 1, 2, 4, 8, 8, 8, 8, 8};
    const int f32[13] = {kElemsSmall, kElemsSmall, kElemsSmall, 1, 2, 4, 2, 4, 4, 4, 4, 8, 8};
    for (int b = 0; b < kBuckets; ++b) {
      const int k = b < 10 ? 0 : (b > 22 ? 12 : b - 10);
      e[FINOM_F64][b] = b < 10 ? kElemsSmall : (b > 22 ? kElems : f64[k]);
      e[FINOM_F32_LOG][b] = b < 10 ? kElemsSmall : (b > 22 ? kElems : f32[k]);
    }
  }
};
Table g_table;

int bucket_of(int64_t L) {
  int b = 0;
  while (b < kBuckets - 1 && ((int64_t)1 << b) < L) ++b;
  return b;
}

bool valid_elems(int e) { return tile_kind_ok(e); }

}  // namespace

int tune_pick(finom_precision prec, int64_t L) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_table.e[prec == FINOM_F64 ? FINOM_F64 : FINOM_F32_LOG][bucket_of(L)];
}

int tune_pick_batch(finom_precision prec) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_table.batch[prec == FINOM_F64 ? FINOM_F64 : FINOM_F32_LOG];
}

}  // namespace finom

extern "C" {

finom_status finom_tune_set_batch(finom_precision prec, int32_t elems) {
  if ((prec != FINOM_F64 && prec != FINOM_F32_LOG) || !finom::valid_elems(elems)) {
    finom::set_error("finom_tune_set_batch: need a known precision and elems in {-1, 1, 2, 4, 8}");
    return FINOM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(finom::g_tune_mu);
  finom::g_table.batch[prec] = elems;
  return FINOM_OK;
}

finom_status finom_tune_get_batch(finom_precision prec, int32_t* elems) {
  if ((prec != FINOM_F64 && prec != FINOM_F32_LOG) || !elems) {
    finom::set_error("finom_tune_get_batch: need a known precision and elems non-null");
    return FINOM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(finom::g_tune_mu);
  *elems = finom::g_table.batch[prec];
  return FINOM_OK;
}

finom_status finom_tune_set(finom_precision prec, int32_t log2_bucket, int32_t elems) {
  if ((prec != FINOM_F64 && prec != FINOM_F32_LOG) || log2_bucket < 0 || log2_bucket >= finom::kBuckets ||
      !finom::valid_elems(elems)) {
    finom::set_error("finom_tune_set: need a known precision, 0 <= log2_bucket < 40, elems in {-1, 1, 2, 4, 8}");
    return FINOM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(finom::g_tune_mu);
  finom::g_table.e[prec][log2_bucket] = elems;
  return FINOM_OK;
}

finom_status finom_tune_get(finom_precision prec, int32_t log2_bucket, int32_t* elems) {
  if ((prec != FINOM_F64 && prec != FINOM_F32_LOG) || log2_bucket < 0 || log2_bucket >= finom::kBuckets || !elems) {
    finom::set_error("finom_tune_get: need a known precision, 0 <= log2_bucket < 40, elems non-null");
    return FINOM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(finom::g_tune_mu);
  *elems = finom::g_table.e[prec][log2_bucket];
  return FINOM_OK;
}

finom_status finom_autotune(finom_precision prec, int32_t log2_bucket, int32_t iters, int32_t* best,
                            double* us_per_iter, void* stream) {
  if ((prec != FINOM_F64 && prec != FINOM_F32_LOG) || log2_bucket < 4 || log2_bucket > 26 || iters < 1 ||
      iters > 100000 || !best) {
    finom::set_error("finom_autotune: need a known precision, 4 <= log2_bucket <= 26, 1 <= iters <= 1e5, best");
    return FINOM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // the synthetic problem: N = M = 2^(bucket-1) sorted points of a fixed
  // pseudo-random sequence on [0, 1], eps = 1e-2, masses from the same sequence
  const int64_t n = (int64_t)1 << (log2_bucket - 1);
  std::vector<double> h(4 * n);
  uint64_t st = 0x9E3779B97F4A7C15ull;
  for (auto& v : h) {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    v = (double)(st >> 11) * (1.0 / 9007199254740992.0);
  }
  std::sort(h.begin(), h.begin() + n);
  std::sort(h.begin() + n, h.begin() + 2 * n);
  for (int64_t i = 2 * n; i < 4 * n; ++i) h[i] = 0.1 + h[i];
  double* d = nullptr;
  FINOM_CUDA(cudaMalloc(&d, sizeof(double) * 6 * n));
  finom_plan_t p = nullptr;
  finom_status rc = FINOM_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const int cand[5] = {finom::kElemsSmall, 1, 2, 4, finom::kElems};
  double t[5] = {0, 0, 0, 0, 0};
  if (cudaMemcpyAsync(d, h.data(), sizeof(double) * 4 * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = finom::cuda_fail(cudaGetLastError(), "finom_autotune setup");
  }
  if (rc == FINOM_OK) rc = finom_plan(d, n, d + n, n, 1e-2, prec, stream, &p);
  const int warm = std::min(16, iters);
  for (int k = 0; k < 5 && rc == FINOM_OK; ++k) {
    rc = finom_plan_set_elems(p, cand[k], stream);
    if (rc == FINOM_OK) rc = finom_solve_begin(p, d + 2 * n, d + 3 * n, 0.0, 1 + warm + iters, nullptr, nullptr,
                                               stream);
    if (rc == FINOM_OK) rc = finom_solve_step(p, warm, stream);
    if (rc != FINOM_OK) break;
    cudaEventRecord(e0, s);
    rc = finom_solve_step(p, iters, stream);
    cudaEventRecord(e1, s);
    if (rc == FINOM_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = finom::cuda_fail(cudaGetLastError(), "tune");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    t[k] = 1e3 * ms / iters;
    if (rc == FINOM_OK) rc = finom_solve_end(p, d + 4 * n, d + 5 * n, nullptr, stream);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  finom_plan_destroy(p);
  cudaFree(d);
  if (rc != FINOM_OK) return rc;
  int bi = 0;
  for (int k = 1; k < 5; ++k)
    if (t[k] < t[bi]) bi = k;
  *best = cand[bi];
  if (us_per_iter)
    for (int k = 0; k < 5; ++k) us_per_iter[k] = t[k];
  return finom_tune_set(prec, log2_bucket, cand[bi]);
}

}  // extern "C"
