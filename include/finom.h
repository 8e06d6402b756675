/*
 * finom.h -- C ABI of libfinom, a GB300 (sm_103a) implementation of FINOM,
 * the fast Sinkhorn algorithm for the entropic Wasserstein-1 distance on
 * non-uniform meshes (Cheng, Liao, Wu, Yang).
 *
 * Problem (Sec. 1, eq. w1Definition; Sec. 2.1, eq. regularized problem):
 * mu = sum_i u_i delta_{x_i} and nu = sum_j v_j delta_{y_j} on sorted meshes,
 * cost c_ij = |x_i - y_j|, kernel K = exp(-C / eps).  The Sinkhorn iteration
 * (eq. iteration) needs K psi and K^T phi; FINOM evaluates them in O(N + M)
 * through the dividing index (Definition, Sec. 2.2) and two first-order
 * recurrences (eqs. p/q by dynamic programming, Sec. 2.3).
 *
 * Conventions for every entry point
 *   - Array arguments are DEVICE pointers (cudaMalloc / torch CUDA tensors) on
 *     the device that was current when the plan was made, unless the name
 *     says "_host".  The caller owns every array it passes; the library never
 *     keeps a caller pointer after the call returns.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous on it unless stated otherwise.
 *   - Every call returns a finom_status.  On failure nothing is written to the
 *     outputs, and finom_last_error() gives a one-line message (per thread).
 *   - A plan may be used by one host thread / one stream at a time.
 *   - Coordinates: float64, sorted non-decreasing, finite.  Duplicates and
 *     ties between x and y are allowed: a tie x_i = y_j belongs to the lower
 *     block of K (Definition, first bullet: y_zeta <= x_i).
 *   - Potentials are in cost units: f = eps * log(phi), g = eps * log(psi)
 *     (-inf where the mass is zero).
 */
#ifndef FINOM_H
#define FINOM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FINOM_OK = 0,
  FINOM_EINVAL = 1,           /* invalid argument: sizes, eps, unsorted or non-finite meshes, bad masses */
  FINOM_ENOMEM = 2,           /* a device (or, in the serving calls, host) allocation failed */
  FINOM_ECUDA = 3,            /* a CUDA runtime call failed (message in finom_last_error) */
  FINOM_EDEVICE_TIMEOUT = 4,  /* a bounded device-side wait gave up */
  FINOM_ENOTSUP = 5,          /* the plan's precision or kind does not support the call */
  FINOM_EPENDING = 6,         /* finom_server_result: the request has not finished (or is unknown) */
  FINOM_ECANCELED = 7         /* a served request was cancelled (finom_server_cancel) */
} finom_status;

typedef enum {
  FINOM_F64 = 0,      /* float64 throughout (the plain form) */
  FINOM_F32_LOG = 1   /* float32 log-domain scans with absorbed potentials (Remark
                         log-domain-stabilization); float64 for the cost <C,Gamma>
                         and the final marginal-error check */
} finom_precision;

typedef struct finom_plan_s* finom_plan_t;

typedef struct {
  double w1;              /* <C, Gamma> of the returned plan, float64 (objective of eq. w1Definition) */
  double marginal_err;    /* || diag(psi) K^T phi - v ||_1 of the returned potentials, float64 */
  double marginal_err_loop; /* the same quantity as computed by the loop's own check (plan precision) */
  double dual;            /* <f, u> + <g, v> */
  int64_t iters;          /* completed Sinkhorn iterations (the paper's l at loop exit) */
  int32_t converged;      /* 1 if the loop stopped because its check was <= tol */
  int32_t status;         /* finom_status of the solve */
} finom_result;

/* Library version (major*10000 + minor*100 + patch). */
int finom_version(void);

/* Last error message of the calling host thread ("" if none). */
const char* finom_last_error(void);

/*
 * finom_plan -- build the plan for the mesh pair (x, y): the merged order of
 * the two meshes (ties: y before x), the dividing index zeta of K and zeta^T
 * of K^T (Definition, Sec. 2.2; Algorithm 1 first step), and the decay
 * factors between consecutive merged points (the ratio vectors r, r' of the
 * Theorems on the vector representation of K_L and K_U, eq. ratio, split at
 * every merged point).
 *   x: N doubles, y: M doubles (device), sorted non-decreasing and finite.
 *   N, M >= 1.  eps > 0 and finite.
 *   prec: FINOM_F64 or FINOM_F32_LOG.
 *   out: receives the plan handle (owned by the library until finom_plan_destroy).
 * Synchronous: returns after the plan is built.  Errors: FINOM_EINVAL for
 * bad sizes/eps or unsorted/non-finite coordinates, FINOM_ENOMEM, FINOM_ECUDA.
 */
finom_status finom_plan(const double* x, int64_t N, const double* y, int64_t M, double eps,
                        finom_precision prec, void* stream, finom_plan_t* out);

/*
 * finom_plan_2d -- plan for two tensor-product grids (Sec. 3, Algorithm 2):
 *   grid 1 = { (x1_k, y1_i) }, grid 2 = { (x2_l, y2_j) },  k, l < N;  i, j < M,
 * with cost |x1_k - x2_l| + |y1_i - y2_j|, so that K = K_y (x) K_x
 * (eq. 2d-kron) with K_x the 1D kernel of (x1, x2) and K_y that of (y1, y2).
 * The plan holds the two axis plans (merged order, dividing indices, decay
 * factors of each axis).
 *   x1, x2: N doubles; y1, y2: M doubles (device), each sorted non-decreasing
 *   and finite.  N, M >= 1, N * M <= 2^31.  eps > 0 and finite.
 * Grid arrays passed to the other entry points hold N * M values in the
 * paper's column-major order: point (k, i) of grid 1 at k + N i, point (l, j)
 * of grid 2 at l + N j (vec() of Sec. 3.2).  On a 2D plan finom_kv is
 * K v (v on grid 2, out on grid 1), finom_ktu is K^T u, finom_kv_log /
 * finom_ktu_log the stabilised products of Appendix A (eq. K'bpsi), and
 * finom_solve / finom_solve_* / finom_cost run Algorithm 2 with that
 * stabilisation (Phi = Psi = 1/(NM) at the start).  finom_dividing_index and
 * finom_kv_log_noalloc return FINOM_ENOTSUP.  finom_plan_info reports N*M for
 * both sizes.  Synchronous.  Errors as finom_plan.
 */
finom_status finom_plan_2d(const double* x1, const double* x2, int64_t N, const double* y1,
                           const double* y2, int64_t M, double eps, finom_precision prec,
                           void* stream, finom_plan_t* out);

/*
 * finom_plan_nd -- plan for two d-dimensional tensor-product grids (Sec. 3.2,
 * the closing remark on higher dimensions: with the separable L1 cost
 * sum_k |x^k - y^k| the kernel is K = K_d (x) ... (x) K_1, and a product
 * with K is d batches of 1D products, one axis after the other):
 *   mu's grid = { (x^1_{i1}, ..., x^d_{id}) }, nu's grid = { (y^1_{j1}, ...,
 *   y^d_{jd}) }, i_k, j_k < n[k].
 *   d: 1 .. 8; n: d sizes (HOST array), each >= 1, product < 2^31.
 *   xs, ys: HOST arrays of d DEVICE pointers; xs[k], ys[k]: n[k] doubles,
 *   each sorted non-decreasing and finite.  eps > 0 and finite.
 * Grid arrays passed to the other entry points hold prod(n) values with axis
 * 0 fastest: point (i_1, ..., i_d) at i_1 + n_1 (i_2 + n_2 (i_3 + ...)) (the
 * paper's vec() for d = 2).  finom_kv (v on nu's grid, out on mu's),
 * finom_ktu, finom_kv_log, finom_ktu_log, finom_solve, finom_solve_begin /
 * step / poll / end, finom_cost and finom_solve_eps_scaling take these plans
 * and run Algorithm 2's loop (Phi = Psi = 1 / prod(n) at the start) with the
 * products done axis by axis by the half-step kernel, every 1D product in
 * log-domain levels; W1 = <C, Gamma> and the marginal error are evaluated in
 * float64.  finom_plan_shape reports dim = d, N = n[0], M = prod(n) / n[0];
 * finom_plan_axes returns n.  Synchronous.  Errors as finom_plan.
 */
finom_status finom_plan_nd(int32_t d, const int64_t* n, const double* const* xs, const double* const* ys,
                           double eps, finom_precision prec, void* stream, finom_plan_t* out);

/*
 * finom_plan_axes -- the number of axes d and the axis sizes n[0 .. d) (host
 * array of at least d entries) of a plan made by finom_plan_nd; other plans:
 * FINOM_ENOTSUP.  Either pointer may be NULL.
 */
finom_status finom_plan_axes(finom_plan_t plan, int32_t* d, int64_t* n);

/*
 * finom_plan_shape -- dimension of a plan and its sizes: dim = 1 with the
 * mesh sizes (N, M), or dim = 2 with the grid sides (N points along x, M
 * along y).  Any pointer may be NULL.
 */
finom_status finom_plan_shape(finom_plan_t plan, int32_t* dim, int64_t* N, int64_t* M);

/*
 * finom_plan_batch -- plan for B independent 1D problems solved together
 * (batching: one launch per half step covers every instance; not a form the
 * paper describes, its arithmetic per instance is Algorithm 1's).
 *   x: sum of N_b doubles, y: sum of M_b doubles (device), instance b's points
 *      at x[offx[b] .. offx[b+1]) and y[offy[b] .. offy[b+1]), each run sorted
 *      non-decreasing and finite.
 *   offx, offy: B + 1 int64 offsets (HOST arrays), offx[0] = offy[0] = 0,
 *      every instance with N_b >= 1 and M_b >= 1.
 *   eps: B doubles (HOST array), each > 0 and finite.
 *   1 <= B <= 2^24; the padded merged length (each instance rounded up to
 *   whole tiles of 2048 points, or 256 * elems with finom_plan_batch_elems)
 *   and each of sum N_b, sum M_b must stay below 2^31.
 * Only finom_solve_batch, finom_plan_info / finom_plan_shape (totals),
 * finom_plan_instances and finom_plan_destroy take a batch plan; the other
 * calls return FINOM_ENOTSUP.  Synchronous.  Errors as finom_plan.
 */
finom_status finom_plan_batch(const double* x, const int64_t* offx, const double* y, const int64_t* offy,
                              int64_t B, const double* eps, finom_precision prec, void* stream,
                              finom_plan_t* out);

/*
 * Queries of the transport plan Gamma = diag(phi) K diag(psi) that a solve
 * returns (Algorithm 1 and Sec. 2.1: Gamma_ij = exp((f_i + g_j - |x_i - y_j|)
 * / eps)), from potentials f (N), g (M) in cost units as finom_solve returns
 * them (-inf where a mass is zero).  1D single-problem plans only (other
 * plans: FINOM_ENOTSUP).  All arrays are device arrays; asynchronous on
 * `stream`.
 *   finom_transport_row  out (M doubles) = row i of Gamma, 0 <= i < N.
 *   finom_transport_col  out (N doubles) = column j of Gamma, 0 <= j < M.
 *   finom_barycentric    barycentric projections: tx (N doubles, may be
 *                        NULL) tx_i = sum_j Gamma_ij y_j / sum_j Gamma_ij,
 *                        ty (M doubles, may be NULL) ty_j = sum_i Gamma_ij
 *                        x_i / sum_i Gamma_ij; two stabilised kernel
 *                        products per side, O(N + M), in the plan's
 *                        precision (float32 plans: absolute error ~1e-5 of
 *                        the mesh extent).  Uses the plan's product scratch:
 *                        a solve in progress on the plan ends.
 */
finom_status finom_transport_row(finom_plan_t plan, const double* f, const double* g, int64_t i, double* out,
                                 void* stream);
finom_status finom_transport_col(finom_plan_t plan, const double* f, const double* g, int64_t j, double* out,
                                 void* stream);
finom_status finom_barycentric(finom_plan_t plan, const double* f, const double* g, double* tx, double* ty,
                               void* stream);

/*
 * Tile size of 1D plans (not a form of the paper: a property of the GPU
 * kernel).  The half-step kernel processes tiles of 256 threads x E points,
 * E in {1, 2, 4, 8}, or, for E = -1, tiles of 64 threads x 1 point (many
 * short tiles on many SMs: the choice of small problems, float64 above all,
 * whose warp instructions hold GB300's float64 pipe for 64 cycles each).
 * finom_plan picks E from a tuning table indexed by precision and the bucket
 * b = ceil(log2(N + M)); results of different E agree to rounding (float64)
 * or within the float32 bounds.
 *   finom_plan_set_elems  forces E on a 1D plan (2D and batch plans: ENOTSUP);
 *                         releases the plan's solve state (a solve in
 *                         progress ends).  Synchronises `stream`.
 *   finom_plan_elems      E and the number of tiles of a plan.
 *   finom_tune_set/get    one entry of the table (b in 0..39; process-wide).
 *   finom_autotune        the autotuner of one bucket: times `iters` Sinkhorn
 *                         iterations (after 16 warm-up ones) of a synthetic
 *                         problem with N = M = 2^(b-1) (sorted pseudo-random
 *                         points, eps = 1e-2) for E = -1, 1, 2, 4, 8 with
 *                         CUDA events on `stream`, installs the fastest in
 *                         the table, returns it in *best and the five times
 *                         (us per iteration, in that order, HOST array of
 *                         5, may be NULL) in us_per_iter.  4 <= b <= 26.
 *                         Synchronous.
 */
finom_status finom_plan_set_elems(finom_plan_t plan, int32_t elems, void* stream);
finom_status finom_plan_elems(finom_plan_t plan, int32_t* elems, int64_t* tiles);
finom_status finom_tune_set(finom_precision prec, int32_t log2_bucket, int32_t elems);
finom_status finom_tune_get(finom_precision prec, int32_t log2_bucket, int32_t* elems);
finom_status finom_autotune(finom_precision prec, int32_t log2_bucket, int32_t iters, int32_t* best,
                            double* us_per_iter, void* stream);

/*
 * finom_plan_batch_elems -- finom_plan_batch with the kernel's points per
 * thread chosen: each instance is packed into tiles of 256 * elems points
 * (elems in {1, 2, 4, 8}, or -1: tiles of 64 points on 64 threads; 0 takes
 * the process-wide batch entry of the tuning
 * table, 8 unless finom_tune_set_batch changed it).  Smaller tiles waste less
 * padding on small instances; results agree to rounding across elems.
 * finom_tune_set_batch / finom_tune_get_batch set and read that entry
 * (paper_2605_26659_gb300/autotune.py times the candidates on a batch).
 */
finom_status finom_plan_batch_elems(const double* x, const int64_t* offx, const double* y, const int64_t* offy,
                                    int64_t B, const double* eps, finom_precision prec, int32_t elems,
                                    void* stream, finom_plan_t* out);
finom_status finom_tune_set_batch(finom_precision prec, int32_t elems);
finom_status finom_tune_get_batch(finom_precision prec, int32_t* elems);

/* Number of instances of a batch plan (0 for other plans). */
finom_status finom_plan_instances(finom_plan_t plan, int64_t* B);

/*
 * finom_solve_batch -- Algorithm 1 for every instance of a batch plan, each
 * with its own masses and eps: the start phi = 1/N_b, psi = 1/M_b, the
 * check || diag(psi) K^T phi - v ||_1 <= tol at every loop head, at most
 * maxit iterations.  An instance retires at its own stop (its tiles are
 * skipped from then on); the call returns when the last one has retired.
 *   u, v: masses in the layout of x, y (device), normalised per instance.
 *   f, g: outputs in the same layout (cost units, -inf where the mass is 0),
 *      the potentials of each instance's stop state.
 *   res: B finom_result (HOST array): per instance W1 and the marginal error
 *      of the returned potentials in float64, the loop's own error, the dual,
 *      the iterations; converged = the float64 error is <= tol (FP32 plans)
 *      or the loop's check passed (FP64 plans).
 * Synchronous.  FINOM_EINVAL for bad masses (any instance).
 */
finom_status finom_solve_batch(finom_plan_t plan, const double* u, const double* v, double tol,
                               int64_t maxit, double* f, double* g, finom_result* res, void* stream);

/*
 * Stepwise form of finom_solve_batch (the loop without the float64 resume):
 *   finom_solve_batch_begin  masses, start state, iteration 0 on `stream`
 *                            (synchronous mass validation only);
 *   finom_solve_batch_step   `iterations` more iterations of every active
 *                            instance (four kernels each); asynchronous;
 *   finom_solve_poll         on a batch plan: *done = every instance retired,
 *                            *iters = iterations launched;
 *   finom_solve_batch_end    f, g and res (as finom_solve_batch) for the state
 *                            of each instance; synchronous.
 */
finom_status finom_solve_batch_begin(finom_plan_t plan, const double* u, const double* v, double tol,
                                     int64_t maxit, void* stream);
finom_status finom_solve_batch_step(finom_plan_t plan, int64_t iterations, void* stream);
finom_status finom_solve_batch_end(finom_plan_t plan, double* f, double* g, finom_result* res, void* stream);

/*
 * Serving loop: continuous batching of 1D and 2D solves (Algorithm 1 and
 * Algorithm 2) of mixed sizes in one process on one GPU.  The paper has no
 * counterpart; each solve's arithmetic is that of finom_solve, so a request's
 * result does not depend on what else is being served.
 *
 * A server owns max_active CUDA streams (slots).  finom_server_submit_* copy a
 * request's HOST arrays and queue it.  finom_server_step runs one scheduling
 * round, without waiting for the GPU:
 *   - admission (first come first served by default; see
 *     finom_server_set_policy): the queue head is admitted while a
 *     slot is free and the estimated device footprint of the active solves
 *     plus its own stays within mem_budget_bytes (a request larger than the
 *     budget is admitted alone); admission copies its inputs to the device,
 *     builds its plan and launches iteration 0 on its slot's stream;
 *   - progress: every active solve whose launches have completed and whose
 *     loop is still running gets more iterations (1, 2, 4, ... up to 64 per
 *     round; CUDA graphs of 16 iterations); the potentials stay on the device;
 *   - retirement: a solve whose loop stopped (check <= tol, or maxit) is
 *     finished: float64 W1 and marginal error; with FINOM_F32_LOG, a float64
 *     error above tol (before maxit) continues the loop in float64 from the
 *     float32 potentials, on a float64 plan of the same meshes, in later
 *     rounds; then f, g are copied to the host and the slot and its memory
 *     are freed.
 *   - batching (finom_server_set_batching; on by default for FINOM_F32_LOG
 *     servers): a 1D request with N + M at most the batching limit is
 *     admitted together with the queued requests compatible with it (the
 *     same tol and maxit, eps within a factor 2), as far as the memory
 *     budget allows (footprint: 240 B per merged point, each request rounded
 *     up to whole 2048-point tiles, plus 1 MiB per batch).  The batch takes
 *     one slot and counts as one active solve; it is solved as by
 *     finom_plan_batch + finom_solve_batch on a host thread of the server
 *     (its plan building and its blocking solve do not hold up the rounds),
 *     and its requests finish together when the last of them retires.  A
 *     batched request's result does not depend on what it was batched with.
 *     The mesh and mass checks of a batched request are made on the host; a
 *     bad one finishes with FINOM_EINVAL without joining a batch.
 * Solves on different slots overlap on the GPU.  All calls on one server
 * must come from one host thread at a time; the server uses the device that
 * was current at finom_server_create.
 */
typedef struct finom_server_s* finom_server_t;

typedef struct {
  int64_t id;             /* request id returned by finom_server_submit_* */
  int32_t kind;           /* 1: 1D, 2: 2D */
  int32_t status;         /* finom_status of the solve (plan, loop, cost) */
  finom_result result;    /* as finom_solve; iters counts every iteration run */
  double latency_s;       /* submit -> result ready (host wall clock) */
  double queue_s;         /* submit -> admission */
} finom_server_done;

/*
 * finom_server_create -- mem_budget_bytes > 0 (device bytes for the active
 * solves), 1 <= max_active <= 256 slots, prec the precision of every solve.
 */
finom_status finom_server_create(int64_t mem_budget_bytes, int32_t max_active, finom_precision prec,
                                 finom_server_t* out);

/*
 * finom_server_set_policy -- admission order of queued requests:
 * FINOM_SERVE_FIFO (default; arrival order) or FINOM_SERVE_SMALLEST_FIRST
 * (the queued request with the smallest estimated footprint first, which
 * keeps short solves from waiting behind long ones; a large request can wait
 * as long as smaller ones keep arriving).
 */
enum { FINOM_SERVE_FIFO = 0, FINOM_SERVE_SMALLEST_FIRST = 1 };
finom_status finom_server_set_policy(finom_server_t srv, int32_t policy);

/*
 * finom_server_set_eps_scaling -- requests admitted from now on first solve
 * their problem at eps / factor^stages, eps / factor^(stages-1), ...,
 * eps / factor, each to tol_stage (or tol if larger) on a plan of its own and
 * warm-started from the previous stage, then at their own eps to tol (as
 * finom_solve_eps_scaling).  The fixed point is unchanged; at small eps it
 * takes fewer iterations.  `iters` of a result counts every stage.  stages = 0
 * (the default) turns it off.  0 <= stages <= 30, 0 < factor < 1,
 * tol_stage > 0.
 */
finom_status finom_server_set_eps_scaling(finom_server_t srv, int32_t stages, double factor, double tol_stage);

/*
 * finom_server_set_batching -- 1D requests admitted from now on with N + M <=
 * max_points are batched (see above); 0 turns batching off.  Default: 65536
 * for FINOM_F32_LOG servers, 0 for FINOM_F64 ones.  Requests are not batched
 * while eps scaling is on.  0 <= max_points <= 2^22, else FINOM_EINVAL.
 */
finom_status finom_server_set_batching(finom_server_t srv, int64_t max_points);

/*
 * finom_server_submit_1d -- queue a 1D solve (arguments as finom_plan and
 * finom_solve; x, y, u, v are HOST arrays of N, M, N, M doubles, copied before
 * the call returns).  *id receives the request id.  Sorting and mass checks
 * happen at admission; a bad request finishes with that status.
 */
finom_status finom_server_submit_1d(finom_server_t srv, const double* x, int64_t N, const double* y, int64_t M,
                                    const double* u, const double* v, double eps, double tol, int64_t maxit,
                                    int64_t* id);

/*
 * finom_server_submit_2d -- queue a 2D solve (arguments as finom_plan_2d and
 * finom_solve on it; x1, x2: N, y1, y2: M, U, V: N * M column-major doubles,
 * HOST arrays, copied before the call returns).
 */
finom_status finom_server_submit_2d(finom_server_t srv, const double* x1, const double* x2, int64_t N,
                                    const double* y1, const double* y2, int64_t M, const double* U,
                                    const double* V, double eps, double tol, int64_t maxit, int64_t* id);

/*
 * finom_server_step -- one scheduling round (see above).  Returns the number
 * of queued, active and finished-but-not-collected requests (any pointer may
 * be NULL).  Errors of a request are reported through its result, not here:
 * a request whose admission or finish fails (device memory, or host memory
 * for its result) is released with that status and can be collected.
 * FINOM_ENOMEM when the round's own host bookkeeping cannot be allocated;
 * then nothing has changed and the round can be retried.
 */
finom_status finom_server_step(finom_server_t srv, int32_t* n_pending, int32_t* n_active, int32_t* n_finished);

/*
 * finom_server_result -- collect a finished request: *out, and its potentials
 * into f (N doubles for 1D, N * M for 2D, HOST, may be NULL) and g (M, or
 * N * M).  The request is forgotten afterwards.  FINOM_EPENDING if it has
 * not finished (or the id is unknown).
 */
finom_status finom_server_result(finom_server_t srv, int64_t id, finom_server_done* out, double* f, double* g);

/*
 * finom_server_cancel -- stop a request: a queued one is dropped, an active
 * one is stopped after its launched work completes (its stream is
 * synchronised) and its memory and slot are freed; a batched one finishes
 * when its batch ends (a batch whose requests are all cancelled stops after
 * its current round of launches).  Each then finishes with status
 * FINOM_ECANCELED (collect it with finom_server_result).  A finished request
 * is left as it is.  FINOM_EINVAL for an unknown id.
 */
finom_status finom_server_cancel(finom_server_t srv, int64_t id);

/* Release the server: stops its batches, waits for its active solves and
 * drops every request. */
finom_status finom_server_destroy(finom_server_t srv);

/* Release the plan and all device memory it owns.  NULL is accepted. */
finom_status finom_plan_destroy(finom_plan_t plan);

/* Sizes of a plan (any pointer may be NULL). */
finom_status finom_plan_info(finom_plan_t plan, int64_t* N, int64_t* M, double* eps,
                             int32_t* precision);

/*
 * finom_dividing_index -- copy the dividing indices out (Definition, Sec. 2.2).
 *   zeta:  N int32 (device), zeta[i] = #{j : y_j <= x_i} in 0..M (the paper's
 *          zeta(i) for row i of K).  May be NULL.
 *   zetaT: M int32 (device), zetaT[j] = #{i : x_i <= y_j} in 0..N (the same
 *          definition applied to K^T).  May be NULL.
 */
finom_status finom_dividing_index(finom_plan_t plan, int32_t* zeta, int32_t* zetaT, void* stream);

/*
 * finom_kv -- out = K v (eq. decompose to p+q: p + q from the forward and the
 * backward recurrence).  v: M doubles, out: N doubles (device), v >= 0 and
 * finite (the recurrences run on log-weights in both precisions).
 * Relative error vs the dense product: <= 1e-12 (F64), <= 1e-5 (F32_LOG) on
 * entries above 1e-30 of the largest.
 */
finom_status finom_kv(finom_plan_t plan, const double* v, double* out, void* stream);

/* finom_ktu -- out = K^T u.  u: N doubles, out: M doubles (device). */
finom_status finom_ktu(finom_plan_t plan, const double* u, double* out, void* stream);

/*
 * finom_kv_log -- the stabilised product of Remark log-domain-stabilization:
 *   out_i = log( sum_j exp((a_i + b_j - |x_i - y_j|) / eps) ),
 * i.e. log( diag(e^{a/eps}) K diag(e^{b/eps}) 1 ).  a: N doubles, b: M
 * doubles (absorption vectors, cost units, finite or -inf in b), out: N
 * doubles (natural log).  For both precisions.
 */
finom_status finom_kv_log(finom_plan_t plan, const double* a, const double* b, double* out,
                          void* stream);

/* finom_ktu_log -- out_j = log( sum_i exp((a_i + b_j - |x_i - y_j|)/eps) ); out: M doubles. */
finom_status finom_ktu_log(finom_plan_t plan, const double* a, const double* b, double* out,
                           void* stream);

/*
 * finom_solve -- Sinkhorn loop of Algorithm 1 (psi first, then phi), started
 * from phi = 1/N, psi = 1/M, or from warm-start potentials.  Stops at the loop
 * head when the marginal error || diag(psi) K^T phi - v ||_1 <= tol or after
 * maxit iterations.
 *   u: N doubles, v: M doubles (device), >= 0, finite, positive sums; they are
 *      normalised to sum 1 internally.
 *   tol >= 0, maxit >= 0.
 *   f: N doubles, g: M doubles (device, outputs; f, g in cost units).  If
 *      warm != 0 they are also inputs (warm-start potentials).
 *   res: host struct, filled on return.
 * FINOM_F32_LOG plans (1D): the float32 loop's own check stops no lower than
 * 2e-7 (its rounding floor); the marginal error is then verified in float64,
 * and a solve whose float64 error is above tol continues, first in float32
 * with a tightened check while that stays above the floor, then in float64
 * on a float64 plan of the same meshes, warm-started from the float32
 * potentials (res->iters counts every iteration).
 * Synchronous (returns when the solve is done).  Non-convergence is not an
 * error: res->converged = 0, res->iters = maxit.
 */
finom_status finom_solve(finom_plan_t plan, const double* u, const double* v, double tol,
                         int64_t maxit, double* f, double* g, int32_t warm, finom_result* res,
                         void* stream);

/*
 * finom_solve_trace -- the marginal error against time (the measurement
 * behind the time-to-error curves of Sec. 4): runs the loop of finom_solve
 * without a stopping tolerance for maxit iterations, started from
 * phi = 1/N, psi = 1/M, and after every `every` iterations records, without
 * synchronising, the loop-head error || diag(psi) K^T phi - v ||_1 (plan
 * precision) and a CUDA event.
 *   err, ms: HOST arrays of ceil(maxit / every) doubles; entry i holds the
 *            error at the head of iteration min((i + 1) * every, maxit - 1)
 *            and the GPU time in ms since iteration 0 was launched.
 *   *n:      number of entries written.
 * The solve state is left ended (use finom_solve for potentials).  1D and
 * 2D plans; synchronous.
 */
finom_status finom_solve_trace(finom_plan_t plan, const double* u, const double* v, int64_t maxit, int64_t every,
                               double* err, double* ms, int64_t* n, void* stream);

/*
 * finom_solve_eps_scaling -- finom_solve preceded by solves of the same
 * problem at eps0, eps0 * factor, eps0 * factor^2, ... (while above the
 * plan's eps), each to tol_stage on a plan of its own and warm-started from
 * the previous stage's potentials; the last stage is finom_solve on `plan`
 * (warm-started) to tol.  Not a form of the paper: the fixed point at the
 * plan's eps is unchanged, only the starting potentials differ, which cuts
 * the iterations at small eps.  res->iters counts the iterations of every
 * stage (all within maxit); res->converged is the last stage's.  1D and 2D
 * plans.  Arguments as finom_solve; eps0 > eps, 0 < factor < 1,
 * tol_stage >= tol.  Synchronous.
 */
finom_status finom_solve_eps_scaling(finom_plan_t plan, const double* u, const double* v, double tol,
                                     int64_t maxit, double eps0, double factor, double tol_stage, double* f,
                                     double* g, finom_result* res, void* stream);

/*
 * Stepwise form of finom_solve (same loop, driven by the caller):
 *   finom_solve_begin  normalises u, v, sets phi = 1/N, psi = 1/M (or the
 *                      warm start f0, g0 when both are non-NULL) and launches
 *                      iteration 0 on `stream`.  Asynchronous except for the
 *                      mass validation (one small device->host read).
 *   finom_solve_step   launches `iterations` more Sinkhorn iterations (two
 *                      kernels each) on `stream`; asynchronous.  Iterations
 *                      after the loop has stopped return at once.
 *   finom_solve_poll   *done = 1 once the loop stopped (check <= tol or maxit;
 *                      1D float32 plans: check <= max(tol, 2e-7));
 *                      *iters = completed iterations.  Synchronises `stream`.
 *   finom_solve_end    writes f, g (device, cost units) and res (host) for the
 *                      state at the loop exit, or after the last completed
 *                      iteration if the loop is still running; res->converged
 *                      is the float64 error <= tol for float32 plans (a caller
 *                      may continue in float64, warm-started, as the serving
 *                      loop does).  Synchronous.
 * Any kernel product or finom_cost on the same plan in between ends the solve.
 */
finom_status finom_solve_begin(finom_plan_t plan, const double* u, const double* v, double tol,
                               int64_t maxit, const double* f0, const double* g0, void* stream);
finom_status finom_solve_step(finom_plan_t plan, int64_t iterations, void* stream);
finom_status finom_solve_poll(finom_plan_t plan, int32_t* done, int64_t* iters, void* stream);
finom_status finom_solve_end(finom_plan_t plan, double* f, double* g, finom_result* res,
                             void* stream);

/*
 * finom_cost -- W1 and marginal error of given potentials, float64:
 *   w1  = <C, Gamma>, Gamma_ij = exp((f_i + g_j - |x_i - y_j|)/eps)
 *   err = sum_j | sum_i Gamma_ij - v_j |
 * u, f: N doubles; v, g: M doubles (device); w1, err: host doubles.
 * Synchronous.
 */
finom_status finom_cost(finom_plan_t plan, const double* u, const double* v, const double* f,
                        const double* g, double* w1, double* err, void* stream);

/*
 * finom_kv_log_noalloc -- the same product as finom_kv_log, for callers that
 * must not allocate device memory (their memory is owned by a fixed pool or
 * another allocator, they run under a hard memory budget, or they cannot
 * afford the allocator's locks and implicit synchronisation).  The paper has
 * no counterpart; this is a property of the library, not of the method.
 *   - Allocates nothing: no cudaMalloc/cudaFree and no allocating library
 *     call.  The working memory of the scan (tile aggregates, tile carries,
 *     the last-block ticket) is one static device array of 262,400 bytes
 *     that every GPU loading the library keeps until the process exits.
 *   - Limit: at most 4096 tiles of the plan, i.e. N + M <= 8,388,608 merged
 *     points at the default 8 points per thread (finom_plan_elems reports a
 *     plan's tile count); larger plans return FINOM_EINVAL with a message,
 *     and nothing is launched.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call shares the array and leaves its contents behind; the ticket
 *     is reset at the start of each call.  Calls that overlap on the GPU (on
 *     different streams, or from different host threads) race and must not
 *     be issued.
 *   - The levels are formed inside the kernel from a, b and the plan's
 *     positions, in one pass; the result is the one finom_kv_log computes,
 *     with the same error bound (1e-5 relative in float32, 1e-12 in
 *     float64), for any a and b.
 * Arguments as finom_kv_log (device pointers; out: N doubles, natural log).
 */
finom_status finom_kv_log_noalloc(finom_plan_t plan, const double* a, const double* b, double* out,
                                  void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FINOM_H */
