// Internal host-side declarations of libfinom (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
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

// Tiles of the half-step kernel: `elems` points per thread of kThreads
// threads (1, 2, 4 or kElems), or kElemsSmall: 64 threads with one point
// each.  Small problems want many small tiles on many SMs with short scans
// over few run totals; on GB300 a float64 warp instruction holds its
// sub-partition's float64 pipe for 64 cycles, so small float64 plans most.
constexpr int kElemsSmall = -1;
constexpr bool tile_kind_ok(int elems) {
  return elems == kElemsSmall || elems == 1 || elems == 2 || elems == 4 || elems == kElems;
}
constexpr int tile_threads(int elems) { return elems == kElemsSmall ? 64 : kThreads; }
constexpr int tile_elems(int elems) { return elems == kElemsSmall ? 1 : elems; }
constexpr int64_t tile_points(int elems) { return (int64_t)tile_elems(elems) * tile_threads(elems); }

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
// The float32 loop's own marginal-error check stops no lower than this: the
// float32 estimate of the error sum has a rounding floor of about this size
// (an error of a few float32 roundings in each log-sum); a solve to a tighter
// tol continues in float64 from the float32 potentials.
constexpr double kF32LoopFloor = 2e-7;

struct SolveState {
  bool ready = false;
  void* px[2] = {nullptr, nullptr};   // x-side (mu) levels of the loop, ping-pong: 1D plans and
  void* py[2] = {nullptr, nullptr};   //   batches (beta+, beta-) per point; grid plans log-weights
  double* mu64 = nullptr;             // x masses, float64 (normalised)
  double* nu64 = nullptr;
  double* tx = nullptr;               // float64 scratch, N
  double* ty = nullptr;               // float64 scratch, M
  void* aggs = nullptr;               // per tile (unit): two log-sum states of the tile aggregates
  void* carries = nullptr;            // per tile (unit): two log-sum states entering the tile
  double* part = nullptr;             // per tile (unit): marginal-error partial sums
  double* scal = nullptr;             // 512 + 8 float64 scalars ([0]: error of the last check)
  int32_t* ctrl = nullptr;            // loop control: [0] ticket [1] done [2] iteration [3] iterations at
                                      //   exit [4] converged (batches: [2] active instances [3] active
                                      //   tiles [6] an instance retired since the last compaction)
  int* bad = nullptr;
  void* qo = nullptr;                 // products: O-side frame levels
  void* qom = nullptr;                // log2 masses of x (products: unused)
  void* qw = nullptr;                 // products: W-side levels
  void* qwm = nullptr;                // log2 masses of y
  void* q2 = nullptr;                 // grid plans: partial products between the axis passes (2 grids)
  int32_t* ictl = nullptr;            // batch: 6 x B per-instance control (done | iteration | at exit |
                                      //   converged | parity flip | iteration budget)
  double* ierr = nullptr;             // batch: per instance, the error of its last check
  double* itol = nullptr;             // batch: per instance, the loop tolerance
  int32_t* alist = nullptr;           // batch: the tiles of the active instances
  cudaStream_t stream = nullptr;      // internal stream (graph capture needs a non-legacy stream)
  cudaGraphExec_t body = nullptr;     // two Sinkhorn iterations
  cudaGraphExec_t chunk = nullptr;    // kChunkIters iterations (stepwise solves)
  double chunk_tol = -1.0;            // loop tolerance and iteration limit the
  int64_t chunk_maxit = -1;           //   chunk was captured with
  // the solve in progress
  bool active = false;
  bool warm = false;
  double tol = 0.0;                   // the loop's own check (device)
  double tol_user = 0.0;              // the solve's tol (float64 verification)
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
  double* gap64 = nullptr;       // per merged point: (z_k - z_{k-1}) / (eps ln 2) (the float64 cost kernel)
  int32_t* tile_x0 = nullptr;    // C + 1 entries: number of x points before each tile
  // tiles of the fused half-step kernel on a 1D plan: elems points per thread
  // (kElems, or 1, 2, 4 for small problems), Ce tiles of elems * kThreads
  // points, tile_x0e the number of x points before each (tile_x0 when elems
  // = kElems)
  int elems = finom::kElems;
  int64_t Ce = 0;
  int32_t* tile_x0e = nullptr;
  int dim = 1;                   // axes of a grid plan (1: a 1D or batch plan)
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
  // batch solves stop early (between rounds of launches, before the float64
  // resumes) once *stop is non-zero: the serving loop's cancellation of a
  // batch whose requests were all cancelled (not owned; null: never)
  const std::atomic<int>* stop = nullptr;
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
// float64 vector helpers (vec.cu)
finom_status normalise_masses(const double* u, int64_t n, double* m64, double* scratch, int* bad,
                              double* total_out, cudaStream_t s);
void pot_from_f(const double* f, const double* m64, int64_t n, double scale, double* pot, cudaStream_t s);
void fill_d(double* f, int64_t n, double v, cudaStream_t s);
void add_scaled(double* out, const double* a, double sc, int64_t n, cudaStream_t s);
void dot_pos(const double* m, const double* f, int64_t n, double* out, cudaStream_t s);
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
