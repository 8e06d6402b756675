// Internal host-side declarations of libfinom (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

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
// iterations per graph launch of the stepwise solves (an even number)
constexpr int kChunkIters = 16;

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
  void* q2 = nullptr;                 // 2D: log2 sums between the two passes of an application
  int32_t* ictl = nullptr;            // batch: 4 x B per-instance control (done | iteration | at exit | converged)
  double* ierr = nullptr;             // batch: per instance, the error of its last check
  double* itol = nullptr;             // batch: per instance, the loop tolerance
  void* iuni = nullptr;               // batch: per instance (1/N, 1/M) for the start phi, psi
  int32_t* alist = nullptr;           // batch: the tiles of the active instances
  double* t2 = nullptr;               // 2D: float64 scratch, one grid
  double* z = nullptr;                // 2D: float64 moments between the two cost passes (2 grids)
  cudaStream_t stream = nullptr;      // internal stream (graph capture needs a non-legacy stream)
  cudaGraphExec_t body = nullptr;     // two Sinkhorn iterations
  cudaGraphExec_t chunk = nullptr;    // kChunkIters iterations (stepwise solves)
  double chunk_tol = -1.0;            // loop tolerance and iteration limit the
  int64_t chunk_maxit = -1;           //   chunk was captured with
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
  // tiles of the fused half-step kernel on a 1D plan: elems points per thread
  // (kElems, or 1, 2, 4 for small problems), Ce tiles of elems * kThreads
  // points, tile_x0e the number of x points before each (tile_x0 when elems
  // = kElems)
  int elems = finom::kElems;
  int64_t Ce = 0;
  int32_t* tile_x0e = nullptr;
  int32_t* fw[2] = {nullptr, nullptr};  // per tile, [o_is_x]: the W point before the O point
                                        // that precedes the tile (frames of 2D first passes)
  // 2D plans (Sec. 3): grids x1 (x) y1 and x2 (x) y2 with N points on the x
  // axis and M on the y axis; ax merges x1 with x2, ay merges y1 with y2
  int dim = 1;
  finom_plan_s* ax = nullptr;
  finom_plan_s* ay = nullptr;
  // batches of independent 1D instances (batch.cu): instance b owns x[offx[b] ..
  // offx[b+1]), y[offy[b] .. offy[b+1]) and the tiles itile[b] .. itile[b+1]-1
  // of the packed merged arrays (every instance starts on a tile boundary)
  int64_t B = 0;                 // instances (0: not a batch plan)
  std::vector<int64_t> hoffx, hoffy;
  std::vector<int32_t> hitile;
  std::vector<double> heps;
  int64_t* ioffx = nullptr;      // device copies (B + 1)
  int64_t* ioffy = nullptr;
  int32_t* itile = nullptr;
  int32_t* tinst = nullptr;      // per tile: its instance
  int64_t btile = finom::kTile;  // merged points per tile of the packing (256 x points per thread)
  std::vector<int32_t> hitilec;  // per instance: first 2048-point tile of the float64 evaluation
  int32_t* tile_x0c = nullptr;   // the evaluation's tile tables (as tile_x0, 2048-point tiles)
  double* ieps = nullptr;        // per instance
  // d-dimensional tensor-product plans (nd.cu; finom_plan_nd): grids of
  // nd_n[0] x ... x nd_n[d-1] points, axis 0 fastest; one 1D plan per axis
  // merging mu's nodes (x side) with nu's (y side); per axis the node
  // positions in bits (level pairs in the plan precision, float64 copies)
  // and log2 of their distance to the axis minimum (float64, the cost)
  static constexpr int kMaxDim = 8;
  bool nd = false;
  int64_t nd_n[kMaxDim] = {};
  int64_t nd_G = 0;
  finom_plan_s* nd_ax[kMaxDim] = {};
  void* nd_zx[kMaxDim] = {};
  void* nd_zy[kMaxDim] = {};
  double* nd_zx64[kMaxDim] = {};
  double* nd_zy64[kMaxDim] = {};
  double* nd_lx64[kMaxDim] = {};
  double* nd_ly64[kMaxDim] = {};
  double nd_z0s[kMaxDim] = {};   // axis minimum over both meshes, in bits
  double* nd_w64 = nullptr;      // float64 workspace of the checks (grids, aggregates)
  finom::SolveState st;
};

namespace finom {
finom_status build_plan(finom_plan_s* p, const double* x, const double* y, cudaStream_t s);
// tile table of a 1D plan for elems points per thread (plan.cu); the solve
// state must be released by the caller when Ce changes
finom_status build_tiles_e(finom_plan_s* p, int elems, cudaStream_t s);
// points per thread that the tuning table gives a 1D plan of L merged points,
// and batch plans
int tune_pick(finom_precision prec, int64_t L);
int tune_pick_batch(finom_precision prec);
void free_plan(finom_plan_s* p);
finom_status cost64(finom_plan_s* p, const double* px, const double* py, const double* u,
                    const double* v, double* err, double* w1, cudaStream_t s);
finom_status cost64_2d(finom_plan_s* p, const double* pa, const double* pb, const double* u,
                       const double* v, double* err, double* w1, cudaStream_t s);
// 2D plans (api2d.cu)
finom_status plan2d_build(finom_plan_s* p, const double* x1, const double* x2, int64_t N,
                          const double* y1, const double* y2, int64_t M, cudaStream_t s);
void plan2d_free(finom_plan_s* p);
finom_status kv2d(finom_plan_s* p, bool transpose_k, bool logmode, const double* a, const double* b,
                  double* out, cudaStream_t s);
finom_status solve2d(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                     double* f, double* g, int32_t warm, finom_result* res, cudaStream_t s);
finom_status solve2d_begin(finom_plan_s* p, const double* u, const double* v, double tol,
                           int64_t maxit, const double* f0, const double* g0, cudaStream_t s);
finom_status solve2d_step(finom_plan_s* p, int64_t iters, cudaStream_t s);
finom_status solve2d_end(finom_plan_s* p, double* f, double* g, finom_result* res, cudaStream_t s);
finom_status cost2d(finom_plan_s* p, const double* u, const double* v, const double* f,
                    const double* g, double* w1, double* err, cudaStream_t s);
// batches of 1D instances (batch.cu)
finom_status plan_batch_build(finom_plan_s* p, const double* x, const int64_t* offx, const double* y,
                              const int64_t* offy, int64_t B, const double* eps, cudaStream_t s);
void plan_batch_free(finom_plan_s* p);
finom_status solve_batch(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                         double* f, double* g, finom_result* res, cudaStream_t s);
finom_status solve_batch_begin(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                               cudaStream_t s);
finom_status solve_batch_step(finom_plan_s* p, int64_t iters, cudaStream_t s);
finom_status solve_batch_end(finom_plan_s* p, double* f, double* g, finom_result* res, cudaStream_t s);
// d-dimensional plans (nd.cu)
finom_status plan_nd_build(finom_plan_s* p, int d, const int64_t* n, const double* const* xs,
                           const double* const* ys, cudaStream_t s);
void plan_nd_free(finom_plan_s* p);
finom_status kv_nd(finom_plan_s* p, bool transpose_k, bool logmode, const double* a, const double* b,
                   double* out, cudaStream_t s);
finom_status solve_nd(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                      double* f, double* g, int32_t warm, finom_result* res, cudaStream_t s);
finom_status solve_nd_begin(finom_plan_s* p, const double* u, const double* v, double tol, int64_t maxit,
                            const double* f0, const double* g0, cudaStream_t s);
finom_status solve_nd_step(finom_plan_s* p, int64_t iters, cudaStream_t s);
finom_status solve_nd_end(finom_plan_s* p, double* f, double* g, finom_result* res, cudaStream_t s);
finom_status cost_nd(finom_plan_s* p, const double* u, const double* v, const double* f, const double* g,
                     double* w1, double* err, cudaStream_t s);
}  // namespace finom
