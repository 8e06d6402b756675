// Internal host-side declarations of libfinom (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "finom.h"

namespace finom {

// Scan geometry: one CTA handles a tile of kThreads * kElems merged points;
// each thread walks kElems consecutive points.  The tile size is fixed for
// both precisions so a plan's tile table serves every kernel.
#ifndef FINOM_THREADS
#define FINOM_THREADS 256
#endif
#ifndef FINOM_ELEMS
#define FINOM_ELEMS 8
#endif
constexpr int kThreads = FINOM_THREADS;
constexpr int kElems = FINOM_ELEMS;
constexpr int kTile = kThreads * kElems;   // merged points per tile (2048 by default)

void set_error(const std::string& msg);
finom_status cuda_fail(cudaError_t e, const char* what);

#define FINOM_CUDA(call)                                           \
  do {                                                             \
    cudaError_t e__ = (call);                                      \
    if (e__ != cudaSuccess) return ::finom::cuda_fail(e__, #call); \
  } while (0)

// Device state of the Sinkhorn loop of one plan (allocated on first use).
struct SolveState {
  bool ready = false;
  void* px[2] = {nullptr, nullptr};   // absorbed x-side potential (log2 units), ping-pong
  void* py[2] = {nullptr, nullptr};   // absorbed y-side potential
  void* mu = nullptr;                 // x masses, plan precision (normalised)
  void* nu = nullptr;                 // y masses
  double* mu64 = nullptr;             // x masses, float64 (normalised)
  double* nu64 = nullptr;
  double* tx = nullptr;               // float64 scratch, N
  double* ty = nullptr;               // float64 scratch, M
  void* aggs = nullptr;               // 6 * C tile maps
  void* carries = nullptr;            // 4 * C tile carries
  double* part = nullptr;             // C per-tile partial sums
  double* scal = nullptr;             // 512 + 8 float64 scalars
  int32_t* ctrl = nullptr;            // loop control words (see apply.cuh)
  int* bad = nullptr;
  void* qo = nullptr;                 // products: O-side frame potentials
  void* qom = nullptr;                // products: O-side masses (read, unused)
  void* qw = nullptr;                 // products: W-side potentials
  void* qwm = nullptr;                // products: W-side masses
  cudaStream_t stream = nullptr;      // internal stream (graph capture needs a non-legacy stream)
  cudaGraphExec_t body = nullptr;     // two Sinkhorn iterations
  // the solve in progress
  bool active = false;
  bool warm = false;
  double tol = 0.0;
  int64_t maxit = 0;
  int64_t launched = 0;               // iterations launched so far (host count)
};

}  // namespace finom

struct finom_plan_s {
  int64_t N = 0, M = 0, L = 0;   // L = N + M merged points
  int64_t C = 0;                 // number of tiles
  double eps = 0.0;
  finom_precision prec = FINOM_F64;
  int device = 0;
  double* x = nullptr;           // copies of the meshes
  double* y = nullptr;
  int32_t* zeta = nullptr;       // #{j : y_j <= x_i}
  int32_t* zetaT = nullptr;      // #{i : x_i <= y_j}
  uint32_t* tbits = nullptr;     // merged type bits, bit set = x point
  void* gap = nullptr;           // per merged point: (z_k - z_{k-1}) / (eps ln 2), plan precision
  double* gap64 = nullptr;       // float64 gaps (the cost kernel uses them)
  int32_t* tile_x0 = nullptr;    // C + 1 entries: number of x points before each tile
  finom::SolveState st;
};

namespace finom {
finom_status build_plan(finom_plan_s* p, const double* x, const double* y, cudaStream_t s);
void free_plan(finom_plan_s* p);
finom_status cost64(finom_plan_s* p, const double* px, const double* py, const double* u,
                    const double* v, double* err, double* w1, cudaStream_t s);
}  // namespace finom
