// Serving loop: continuous batching of 1D and 2D solves of mixed sizes.
//
// Requests are queued on the host; a scheduling round (finom_server_step)
// admits queued requests (first come first served, or smallest first) while their estimated
// device footprint fits the memory budget and a stream slot is free, builds
// their plans and starts their solves on their own stream; for every active
// solve whose previous launches have completed it either launches more
// iterations (doubling, up to 64 per round) or, once the loop has stopped,
// finishes it (float64 W1 and marginal error, potentials copied back; with
// float32 scans, a float64 error above tol first continues in float64) and
// frees its memory and slot.  Potentials stay resident on the device for
// the whole solve, and the kernels of all active solves run concurrently on
// the GPU from their streams; each solve's arithmetic is that of finom_solve,
// whatever else is running.
//
// Small 1D requests (N + M up to the server's batching limit) are admitted
// together instead: the queued requests compatible with the next one (same
// tol and maxit, eps within a factor 2) form one batch (finom_plan_batch /
// finom_solve_batch: one launch per half step for all of them, each retiring
// at its own stop), which takes one slot and runs on a host thread of its
// own, so that its plan building, its blocking solve and its plan release
// never hold up the scheduling rounds.  An instance's arithmetic in a batch
// does not depend on the other instances, so a batched request's result is
// the same whatever it was batched with.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <chrono>
#include <cmath>
#include <deque>
#include <atomic>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "finom_internal.h"

struct finom_server_s {
  struct Group;
  struct Req {
    int64_t id = 0;
    int kind = 1;                     // 1: 1D, 2: 2D
    int64_t N = 0, M = 0;             // 1D: mesh sizes; 2D: grid sides
    double eps = 0.0, tol = 0.0;
    int64_t maxit = 0;
    std::vector<double> in[6];        // 1D: x, y, u, v; 2D: x1, x2, y1, y2, U, V
    int64_t footprint = 0;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    // while active
    int slot = -1;
    finom_plan_t plan = nullptr;
    finom_plan_t plan64 = nullptr;    // after a switch to float64: the float32 plan
    int64_t iters_before = 0;         // iterations before that switch (or the current stage)
    int stages_left = 0;              // eps-scaling stages still to come before the final eps
    double* dev = nullptr;            // device inputs, then f and g
    cudaEvent_t ev = nullptr;
    int64_t step = 1;
    // when finished
    int32_t status = FINOM_OK;
    finom_result res{};
    std::vector<double> f, g;
    // batching: host checks of a 1D request (done at submit), the batch it
    // runs in, and a cancellation that takes effect when that batch ends
    bool valid = true;
    Group* group = nullptr;
    bool cancelled = false;
  };
  // A batch of small 1D requests, solved by a host thread on the batch's
  // slot.  The thread writes the members' results, then sets ready (the
  // members are no longer touched by it), releases the plan and the device
  // memory, then sets done.
  struct Group {
    std::vector<Req*> members;
    int slot = -1;
    int64_t footprint = 0;
    double tol = 0.0;
    int64_t maxit = 0;
    std::atomic<int> stop{0};
    std::atomic<int> ready{0};
    std::atomic<int> done{0};
    bool collected = false;     // members moved to finished
    std::thread worker;
  };
  int64_t budget = 0, used = 0;
  int max_active = 8;
  // eps scaling (finom_server_set_eps_scaling): stages at eps / factor^k,
  // k = stages .. 1, each to tol_stage, before the request's own eps
  int sc_stages = 0;
  double sc_factor = 0.5, sc_tol = 1e-4;
  int policy = FINOM_SERVE_FIFO;        // admission order
  // 1D requests with N + M <= batch_points are batched (0: never); the
  // default for float32 servers, float64 servers solve every request alone
  int64_t batch_points = 0;
  finom_precision prec = FINOM_F32_LOG;
  int device = 0;
  int64_t next_id = 1;
  // Containers only grow where capacity was reserved beforehand (submit
  // reserves room in finished for every request in flight, step reserves
  // active, its successor list and the graveyard before it changes any
  // state), so that a host allocation failure surfaces as FINOM_ENOMEM
  // before any request changes hands.
  std::deque<Req*> pending;
  std::vector<Req*> active;
  std::vector<Group*> groups;   // active batches
  int64_t grouped = 0;          // requests in active batches, not yet finished
  std::vector<Req*> finished;
  std::vector<cudaStream_t> streams;
  std::vector<int> free_slots;
  // plans of retired requests, destroyed together: freeing device memory
  // waits for the whole device, so it is done once per batch of plans (or
  // when their memory is needed) rather than at every retirement, and on a
  // host thread (a reaper), so that the scheduling rounds never wait for it;
  // their bytes count as used until the reaper is done
  std::vector<finom_plan_t> graveyard;
  int64_t dead_bytes = 0;
  struct Reaper {
    std::vector<finom_plan_t> plans;
    int64_t bytes = 0;
    std::atomic<int> done{0};
    std::thread worker;
  };
  std::vector<Reaper*> reapers;
};

namespace {

using Req = finom_server_s::Req;

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// device bytes of a solve (plan, state, scratch), an estimate for admission
int64_t footprint(int kind, int64_t N, int64_t M) {
  if (kind == 1) return (N + M) * 240 + (1 << 20);
  return N * M * 260 + (N + M) * 240 + (1 << 20);
}

int64_t npoints(const Req* r, int side) {   // points of the first (side 0) or second measure
  (void)side;
  return r->kind == 1 ? (side == 0 ? r->N : r->M) : r->N * r->M;
}

constexpr size_t kGraveyard = 32;

// Destroy the plans of the graveyard: on a reaper thread, or here when
// `wait` is set or no thread can be had.
void flush_graveyard(finom_server_s* s, bool wait = false) {
  if (!wait && !s->graveyard.empty()) {
    auto* k = new (std::nothrow) finom_server_s::Reaper();
    if (k) {
      try {
        s->reapers.reserve(s->reapers.size() + 1);
        k->plans.assign(s->graveyard.begin(), s->graveyard.end());
        k->bytes = s->dead_bytes;
        const int dev = s->device;
        k->worker = std::thread([k, dev] {
          cudaSetDevice(dev);
          for (finom_plan_t p : k->plans) finom_plan_destroy(p);
          k->done.store(1, std::memory_order_release);
        });
        s->reapers.push_back(k);   // (reserved above)
        s->graveyard.clear();      // (keeps its capacity for the round)
        s->dead_bytes = 0;
        return;
      } catch (...) {   // no memory or thread: destroy them here
        delete k;
      }
    }
  }
  for (finom_plan_t p : s->graveyard) finom_plan_destroy(p);
  s->graveyard.clear();
  s->used -= s->dead_bytes;
  s->dead_bytes = 0;
}

// reapers that are done: their plans' bytes are free again (all of them
// when `wait` is set)
void collect_reapers(finom_server_s* s, bool wait) {
  for (size_t k = 0; k < s->reapers.size();) {
    finom_server_s::Reaper* r = s->reapers[k];
    if (!wait && !r->done.load(std::memory_order_acquire)) {
      ++k;
      continue;
    }
    r->worker.join();
    s->used -= r->bytes;
    s->reapers[k] = s->reapers.back();
    s->reapers.pop_back();
    delete r;
  }
}

void release(finom_server_s* s, Req* r) {
  if (r->plan) s->graveyard.push_back(r->plan);
  if (r->plan64) s->graveyard.push_back(r->plan64);
  s->dead_bytes += r->footprint;   // still counted in used until the plans are destroyed
  if (r->dev) cudaFreeAsync(r->dev, s->streams[r->slot]);
  if (r->ev) cudaEventDestroy(r->ev);
  r->plan = nullptr;
  r->plan64 = nullptr;
  r->dev = nullptr;
  r->ev = nullptr;
  if (r->slot >= 0) s->free_slots.push_back(r->slot);
  r->slot = -1;
  for (auto& v : r->in) std::vector<double>().swap(v);
}

void fail(finom_server_s* s, Req* r, finom_status rc) {
  r->status = rc;
  r->res.status = rc;
  r->t_done = now_s();
  release(s, r);
  s->finished.push_back(r);   // (capacity reserved by submit)
}

std::vector<Req*>::iterator find_finished(finom_server_s* s, int64_t id) {
  return std::find_if(s->finished.begin(), s->finished.end(), [id](const Req* r) { return r->id == id; });
}

// batching
constexpr int64_t kBatchPoints = (int64_t)1 << 16;   // default limit of float32 servers (N + M)
constexpr size_t kGroupMax = 1024;                   // requests per batch
constexpr int64_t kGroupPoints = (int64_t)1 << 24;   // padded merged points per batch
constexpr int64_t kPad = 2048;                       // a batch packs each request into whole tiles of
                                                     // at most this many merged points

int64_t padded(const Req* r) { return (r->N + r->M + kPad - 1) / kPad * kPad; }

// the footprint a batch adds for one more member, and that of a batch of one
int64_t member_bytes(const Req* r) { return padded(r) * 240; }
int64_t group_bytes(const Req* r) { return member_bytes(r) + (1 << 20); }

// the checks finom_plan and finom_solve make on the device, on the host: a
// batch plan refuses the whole batch for one bad request, so bad requests
// are finished before they join one
bool check_1d(const Req* r) {
  auto mesh = [](const std::vector<double>& a) {
    for (size_t i = 0; i < a.size(); ++i)
      if (!std::isfinite(a[i]) || (i > 0 && a[i] < a[i - 1])) return false;
    return true;
  };
  auto mass = [](const std::vector<double>& a) {
    double t = 0.0;
    for (double v : a) {
      if (!std::isfinite(v) || v < 0.0) return false;
      t += v;
    }
    return t > 0.0 && std::isfinite(t);
  };
  return std::isfinite(r->eps) && mesh(r->in[0]) && mesh(r->in[1]) && mass(r->in[2]) && mass(r->in[3]);
}

bool batchable(const finom_server_s* s, const Req* r) {
  return s->batch_points > 0 && s->sc_stages == 0 && r->kind == 1 && r->N + r->M <= s->batch_points;
}

// requests that share a batch: the same stop rule, and eps within a factor 2
// (similar iteration counts, so that members retire at similar times)
bool compatible(const Req* a, const Req* b) {
  return a->tol == b->tol && a->maxit == b->maxit && std::max(a->eps, b->eps) <= 2.0 * std::min(a->eps, b->eps);
}

// The host thread of a batch: packed inputs to the device, the batch plan,
// the blocking batch solve (float64 verification and finish included), the
// members' potentials and results; then ready, then the plan and the device
// memory are released, then done.
void run_group(finom_server_s::Group* g, int device, cudaStream_t st, finom_precision prec) {
  const size_t B = g->members.size();
  finom_status rc = FINOM_OK;
  std::vector<finom_result> res;
  finom_plan_t plan = nullptr;
  double* d = nullptr;
  cudaSetDevice(device);
  try {
    std::vector<int64_t> offx(B + 1, 0), offy(B + 1, 0);
    std::vector<double> eps(B);
    for (size_t b = 0; b < B; ++b) {
      offx[b + 1] = offx[b] + g->members[b]->N;
      offy[b + 1] = offy[b] + g->members[b]->M;
      eps[b] = g->members[b]->eps;
    }
    const int64_t X = offx[B], Y = offy[B];
    // x | y | u | v of every member, packed; f | g follow on the device
    std::vector<double> h(2 * (X + Y));
    for (size_t b = 0; b < B; ++b) {
      const Req* r = g->members[b];
      std::copy(r->in[0].begin(), r->in[0].end(), h.begin() + offx[b]);
      std::copy(r->in[1].begin(), r->in[1].end(), h.begin() + X + offy[b]);
      std::copy(r->in[2].begin(), r->in[2].end(), h.begin() + (X + Y) + offx[b]);
      std::copy(r->in[3].begin(), r->in[3].end(), h.begin() + (2 * X + Y) + offy[b]);
    }
    res.resize(B);
    cudaError_t e = cudaMallocAsync(&d, sizeof(double) * 3 * (X + Y), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rc = finom::cuda_fail(e, "finom_server_step: batch inputs");
    if (rc == FINOM_OK)
      rc = finom_plan_batch(d, offx.data(), d + X, offy.data(), (int64_t)B, eps.data(), prec, st, &plan);
    double* fg = d ? d + 2 * (X + Y) : nullptr;
    if (rc == FINOM_OK) {
      plan->stop = &g->stop;
      rc = finom_solve_batch(plan, d + (X + Y), d + (2 * X + Y), g->tol, g->maxit, fg, fg + X, res.data(), st);
    }
    if (rc == FINOM_OK) {
      for (Req* r : g->members) {
        r->f.resize(r->N);
        r->g.resize(r->M);
      }
      h.resize(X + Y);
      e = cudaMemcpyAsync(h.data(), fg, sizeof(double) * (X + Y), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = finom::cuda_fail(e, "finom_server_step: batch results");
      for (size_t b = 0; b < B && rc == FINOM_OK; ++b) {
        Req* r = g->members[b];
        std::copy(h.begin() + offx[b], h.begin() + offx[b + 1], r->f.begin());
        std::copy(h.begin() + X + offy[b], h.begin() + X + offy[b + 1], r->g.begin());
      }
    }
  } catch (const std::bad_alloc&) {
    finom::set_error("finom_server_step: out of host memory for a batch");
    rc = FINOM_ENOMEM;
  }
  const double t = now_s();
  for (size_t b = 0; b < B; ++b) {
    Req* r = g->members[b];
    r->status = rc;
    if (rc == FINOM_OK) {
      r->res = res[b];
    } else {
      r->res = finom_result{};
      r->res.status = rc;
      std::vector<double>().swap(r->f);
      std::vector<double>().swap(r->g);
    }
    r->t_done = t;
  }
  g->ready.store(1, std::memory_order_release);   // the members are the server's again
  if (plan) finom_plan_destroy(plan);
  if (d) {
    cudaFreeAsync(d, st);
    cudaStreamSynchronize(st);
  }
  g->done.store(1, std::memory_order_release);
}

// Admission of a batch headed by *pick: the head and the queued requests
// compatible with it (in admission order) while the memory budget allows.
// FINOM_ENOMEM, with nothing changed, when the host bookkeeping or the
// thread cannot be had.
finom_status admit_group(finom_server_s* s, std::deque<Req*>::iterator pick) {
  using Group = finom_server_s::Group;
  Req* head = *pick;
  Group* g = new (std::nothrow) Group();
  if (!g) return FINOM_ENOMEM;
  std::deque<Req*> rest;
  try {
    g->members.push_back(head);
    g->footprint = group_bytes(head);
    int64_t pts = padded(head);
    std::vector<Req*> cand;
    for (Req* q : s->pending)
      if (q != head && q->valid && batchable(s, q) && compatible(head, q)) cand.push_back(q);
    if (s->policy == FINOM_SERVE_SMALLEST_FIRST)
      std::stable_sort(cand.begin(), cand.end(), [](const Req* a, const Req* b) { return a->footprint < b->footprint; });
    for (Req* q : cand) {
      if (g->members.size() >= kGroupMax) break;
      if (s->used + g->footprint + member_bytes(q) > s->budget || pts + padded(q) > kGroupPoints) continue;
      g->members.push_back(q);
      g->footprint += member_bytes(q);
      pts += padded(q);
    }
    for (Req* q : g->members) q->group = g;
    for (Req* q : s->pending)
      if (q->group != g) rest.push_back(q);
    g->slot = s->free_slots.back();
    g->tol = head->tol;
    g->maxit = head->maxit;
    g->worker = std::thread(run_group, g, s->device, s->streams[g->slot], s->prec);
  } catch (...) {   // std::bad_alloc, or std::system_error from the thread
    for (Req* q : g->members) q->group = nullptr;
    delete g;
    return FINOM_ENOMEM;
  }
  // nothing below throws (the round reserved room in groups)
  s->free_slots.pop_back();
  s->pending.swap(rest);
  s->used += g->footprint;
  s->grouped += (int64_t)g->members.size();
  const double t = now_s();
  for (Req* q : g->members) {
    q->t_admit = t;
    q->slot = g->slot;
  }
  s->groups.push_back(g);
  return FINOM_OK;
}

// a batch whose thread has written its results: the members to finished;
// once the thread is done, the slot and the memory are free again
bool retire_group(finom_server_s* s, finom_server_s::Group* g) {
  if (!g->collected && g->ready.load(std::memory_order_acquire)) {
    for (Req* q : g->members) {
      if (q->cancelled) q->status = q->res.status = FINOM_ECANCELED;
      q->group = nullptr;
      q->slot = -1;
      for (auto& v : q->in) std::vector<double>().swap(v);
      s->finished.push_back(q);   // (capacity reserved by submit)
    }
    s->grouped -= (int64_t)g->members.size();
    g->collected = true;
  }
  if (!g->collected || !g->done.load(std::memory_order_acquire)) return false;
  g->worker.join();
  s->free_slots.push_back(g->slot);
  s->used -= g->footprint;
  return true;
}

// a queued request that fails the host checks of batching
void finish_invalid(finom_server_s* s, Req* r) {
  r->status = r->res.status = FINOM_EINVAL;
  r->t_admit = r->t_done = now_s();
  for (auto& v : r->in) std::vector<double>().swap(v);
  s->finished.push_back(r);   // (capacity reserved by submit)
}

// a plan of the request's meshes (device copies in r->dev) at eps e
finom_status plan_at(finom_server_s* s, Req* r, double e, finom_precision prec, finom_plan_t* out) {
  (void)s;
  const double* d = r->dev;
  cudaStream_t st = s->streams[r->slot];
  if (r->kind == 1) return finom_plan(d, r->N, d + r->N, r->M, e, prec, st, out);
  return finom_plan_2d(d, d + r->N, r->N, d + 2 * r->N, d + 2 * r->N + r->M, r->M, e, prec, st, out);
}

// admit: device copies of the inputs, the plan, the start of the solve
finom_status admit(finom_server_s* s, Req* r) {
  r->slot = s->free_slots.back();
  s->free_slots.pop_back();
  s->used += r->footprint;
  r->t_admit = now_s();
  cudaStream_t st = s->streams[r->slot];
  const int64_t n1 = npoints(r, 0), n2 = npoints(r, 1);
  int64_t total = 0;
  for (auto& v : r->in) total += (int64_t)v.size();
  total += n1 + n2;   // f, g
  FINOM_CUDA(cudaMallocAsync(&r->dev, sizeof(double) * total, st));
  FINOM_CUDA(cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming));
  double* d[6];
  int64_t off = 0;
  for (int k = 0; k < 6; ++k) {
    d[k] = r->dev + off;
    if (!r->in[k].empty())
      FINOM_CUDA(cudaMemcpyAsync(d[k], r->in[k].data(), sizeof(double) * r->in[k].size(),
                                 cudaMemcpyHostToDevice, st));
    off += (int64_t)r->in[k].size();
  }
  r->stages_left = s->sc_stages;
  const double e0 = r->eps / std::pow(s->sc_factor, r->stages_left);
  const double tol0 = r->stages_left > 0 ? std::max(r->tol, s->sc_tol) : r->tol;
  finom_status rc = plan_at(s, r, e0, s->prec, &r->plan);
  if (rc == FINOM_OK)
    rc = finom_solve_begin(r->plan, d[r->kind == 1 ? 2 : 4], d[r->kind == 1 ? 3 : 5], tol0, r->maxit, nullptr,
                           nullptr, st);
  if (rc != FINOM_OK) return rc;
  FINOM_CUDA(cudaEventRecord(r->ev, st));
  return FINOM_OK;
}

// A solve whose loop has stopped: its float64 result; with float32 scans, a
// float64 marginal error above tol (the float32 check passed, or the float32
// precision floor is above tol) continues in float64 from the float32
// potentials on a float64 plan of the same meshes (*more = true); otherwise
// the potentials go to the host and the request is released.
finom_status finish(finom_server_s* s, Req* r, bool* more) {
  *more = false;
  cudaStream_t st = s->streams[r->slot];
  const int64_t n1 = npoints(r, 0), n2 = npoints(r, 1);
  int64_t off = 0;
  for (auto& v : r->in) off += (int64_t)v.size();
  double* f = r->dev + off;
  double* g = f + n1;
  const double* u = r->dev + (r->kind == 1 ? r->N + r->M : 2 * (r->N + r->M));
  const double* v = u + n1;
  finom_status rc = finom_solve_end(r->plan, f, g, &r->res, st);
  if (rc != FINOM_OK) return rc;
  r->res.iters += r->iters_before;
  if (r->stages_left > 0) {
    // eps scaling: the next stage (or the request's own eps) on a plan of its
    // own, warm-started from this stage's potentials
    --r->stages_left;
    const double e = r->eps / std::pow(s->sc_factor, r->stages_left);
    const double tol = r->stages_left > 0 ? std::max(r->tol, s->sc_tol) : r->tol;
    s->graveyard.push_back(r->plan);   // an extra plan alive until the next flush
    s->used += r->footprint;
    s->dead_bytes += r->footprint;
    r->plan = nullptr;
    rc = plan_at(s, r, e, s->prec, &r->plan);
    if (rc != FINOM_OK) return rc;
    rc = finom_solve_begin(r->plan, u, v, tol, std::max<int64_t>(r->maxit - r->res.iters, 0), f, g, st);
    if (rc != FINOM_OK) return rc;
    r->iters_before = r->res.iters;
    r->step = 1;
    FINOM_CUDA(cudaEventRecord(r->ev, st));
    *more = true;
    return FINOM_OK;
  }
  if (!r->res.converged && r->res.iters < r->maxit && !r->plan64 && s->prec != FINOM_F64) {
    rc = plan_at(s, r, r->eps, FINOM_F64, &r->plan64);
    if (rc != FINOM_OK) return rc;
    rc = finom_solve_begin(r->plan64, u, v, r->tol, r->maxit - r->res.iters, f, g, st);
    if (rc != FINOM_OK) return rc;
    std::swap(r->plan, r->plan64);   // the float32 plan is released with the request
    r->iters_before = r->res.iters;
    r->step = 1;
    FINOM_CUDA(cudaEventRecord(r->ev, st));
    *more = true;
    return FINOM_OK;
  }
  try {
    r->f.resize(n1);
    r->g.resize(n2);
  } catch (const std::bad_alloc&) {
    finom::set_error("finom_server_step: out of host memory for a result");
    return FINOM_ENOMEM;
  }
  FINOM_CUDA(cudaMemcpyAsync(r->f.data(), f, sizeof(double) * n1, cudaMemcpyDeviceToHost, st));
  FINOM_CUDA(cudaMemcpyAsync(r->g.data(), g, sizeof(double) * n2, cudaMemcpyDeviceToHost, st));
  FINOM_CUDA(cudaStreamSynchronize(st));
  r->t_done = now_s();
  release(s, r);
  return FINOM_OK;
}

finom_status submit(finom_server_s* s, Req* r, int64_t* id) {
  try {
    // room for every request in flight to finish without a reallocation
    s->finished.reserve(s->finished.size() + s->pending.size() + s->active.size() + (size_t)s->grouped + 1);
    s->pending.push_back(r);
  } catch (const std::bad_alloc&) {
    delete r;
    finom::set_error("finom_server_submit: out of host memory");
    return FINOM_ENOMEM;
  }
  r->id = s->next_id++;
  r->footprint = footprint(r->kind, r->N, r->M);
  if (r->kind == 1) r->valid = check_1d(r);
  r->t_submit = now_s();
  if (id) *id = r->id;
  return FINOM_OK;
}

}  // namespace

extern "C" {

finom_status finom_server_create(int64_t mem_budget_bytes, int32_t max_active, finom_precision prec,
                                 finom_server_t* out) {
  if (!out || mem_budget_bytes <= 0 || max_active < 1 || max_active > 256 ||
      (prec != FINOM_F64 && prec != FINOM_F32_LOG)) {
    finom::set_error("finom_server_create: need out, a positive budget, 1 <= max_active <= 256, known precision");
    return FINOM_EINVAL;
  }
  finom_server_s* s = new (std::nothrow) finom_server_s();
  if (!s) return FINOM_ENOMEM;
  s->budget = mem_budget_bytes;
  s->max_active = max_active;
  s->prec = prec;
  s->batch_points = prec == FINOM_F32_LOG ? kBatchPoints : 0;
  cudaGetDevice(&s->device);
  try {
    s->streams.resize(max_active);
    s->free_slots.reserve(max_active);
  } catch (const std::bad_alloc&) {
    delete s;
    finom::set_error("finom_server_create: out of host memory");
    return FINOM_ENOMEM;
  }
  for (int k = 0; k < max_active; ++k) {
    cudaError_t e = cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (int j = 0; j < k; ++j) cudaStreamDestroy(s->streams[j]);
      delete s;
      return finom::cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    s->free_slots.push_back(max_active - 1 - k);
  }
  *out = s;
  return FINOM_OK;
}

finom_status finom_server_set_policy(finom_server_t s, int32_t policy) {
  if (!s || (policy != FINOM_SERVE_FIFO && policy != FINOM_SERVE_SMALLEST_FIRST)) {
    finom::set_error("finom_server_set_policy: need a server and FINOM_SERVE_FIFO or FINOM_SERVE_SMALLEST_FIRST");
    return FINOM_EINVAL;
  }
  s->policy = policy;
  return FINOM_OK;
}

finom_status finom_server_set_batching(finom_server_t s, int64_t max_points) {
  if (!s || max_points < 0 || max_points > ((int64_t)1 << 22)) {
    finom::set_error("finom_server_set_batching: need a server and 0 <= max_points <= 2^22");
    return FINOM_EINVAL;
  }
  s->batch_points = max_points;
  return FINOM_OK;
}

finom_status finom_server_set_eps_scaling(finom_server_t s, int32_t stages, double factor, double tol_stage) {
  if (!s || stages < 0 || stages > 30 || !(factor > 0.0 && factor < 1.0) || !(tol_stage > 0.0)) {
    finom::set_error("finom_server_set_eps_scaling: need 0 <= stages <= 30, 0 < factor < 1, tol_stage > 0");
    return FINOM_EINVAL;
  }
  s->sc_stages = stages;
  s->sc_factor = factor;
  s->sc_tol = tol_stage;
  return FINOM_OK;
}

finom_status finom_server_submit_1d(finom_server_t s, const double* x, int64_t N, const double* y, int64_t M,
                                    const double* u, const double* v, double eps, double tol, int64_t maxit,
                                    int64_t* id) {
  if (!s || !x || !y || !u || !v || N < 1 || M < 1 || N > INT32_MAX || M > INT32_MAX - N || !(eps > 0.0) ||
      !(tol >= 0.0) || maxit < 0) {
    finom::set_error("finom_server_submit_1d: bad argument");
    return FINOM_EINVAL;
  }
  Req* r = new (std::nothrow) Req();
  if (!r) return FINOM_ENOMEM;
  r->kind = 1;
  r->N = N;
  r->M = M;
  r->eps = eps;
  r->tol = tol;
  r->maxit = maxit;
  try {   // the host copies of the inputs (no C++ exception crosses the C ABI)
    r->in[0].assign(x, x + N);
    r->in[1].assign(y, y + M);
    r->in[2].assign(u, u + N);
    r->in[3].assign(v, v + M);
  } catch (const std::bad_alloc&) {
    delete r;
    finom::set_error("finom_server_submit_1d: out of host memory");
    return FINOM_ENOMEM;
  }
  return submit(s, r, id);
}

finom_status finom_server_submit_2d(finom_server_t s, const double* x1, const double* x2, int64_t N,
                                    const double* y1, const double* y2, int64_t M, const double* U,
                                    const double* V, double eps, double tol, int64_t maxit, int64_t* id) {
  if (!s || !x1 || !x2 || !y1 || !y2 || !U || !V || N < 1 || M < 1 || N > ((int64_t)1 << 31) / M ||
      !(eps > 0.0) || !(tol >= 0.0) || maxit < 0) {
    finom::set_error("finom_server_submit_2d: bad argument");
    return FINOM_EINVAL;
  }
  Req* r = new (std::nothrow) Req();
  if (!r) return FINOM_ENOMEM;
  r->kind = 2;
  r->N = N;
  r->M = M;
  r->eps = eps;
  r->tol = tol;
  r->maxit = maxit;
  try {   // the host copies of the inputs (no C++ exception crosses the C ABI)
    r->in[0].assign(x1, x1 + N);
    r->in[1].assign(x2, x2 + N);
    r->in[2].assign(y1, y1 + M);
    r->in[3].assign(y2, y2 + M);
    r->in[4].assign(U, U + N * M);
    r->in[5].assign(V, V + N * M);
  } catch (const std::bad_alloc&) {
    delete r;
    finom::set_error("finom_server_submit_2d: out of host memory");
    return FINOM_ENOMEM;
  }
  return submit(s, r, id);
}

finom_status finom_server_step(finom_server_t s, int32_t* n_pending, int32_t* n_active, int32_t* n_finished) {
  if (!s) {
    finom::set_error("finom_server_step: null server");
    return FINOM_EINVAL;
  }
  // the only host allocations of a round, before any state changes: every
  // request can move to the active list or its successor, and release up to
  // three plans (two of a request, one of an eps-scaling stage); a batch's
  // own bookkeeping is allocated at its admission, which falls back to a
  // solve alone when that fails
  std::vector<Req*> still;
  try {
    const size_t n = (size_t)s->max_active;   // every active solve or batch holds a slot
    s->active.reserve(n);
    still.reserve(n);
    s->graveyard.reserve(s->graveyard.size() + 3 * n);
    s->groups.reserve(n);
  } catch (const std::bad_alloc&) {
    finom::set_error("finom_server_step: out of host memory");
    return FINOM_ENOMEM;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != s->device) cudaSetDevice(s->device);
  // batches whose threads have finished and reapers that are done (their
  // slots and bytes serve this round's admissions)
  collect_reapers(s, false);
  for (size_t k = 0; k < s->groups.size();) {
    finom_server_s::Group* g = s->groups[k];
    if (!retire_group(s, g)) {
      ++k;
      continue;
    }
    s->groups[k] = s->groups.back();
    s->groups.pop_back();
    delete g;
  }
  // admissions, first come first served: an empty server always admits
  while (!s->pending.empty() && !s->free_slots.empty()) {
    // the next request: the queue head, or the smallest queued one
    auto pick = s->pending.begin();
    if (s->policy == FINOM_SERVE_SMALLEST_FIRST)
      for (auto it = s->pending.begin(); it != s->pending.end(); ++it)
        if ((*it)->footprint < (*pick)->footprint) pick = it;
    Req* r = *pick;
    const bool batch = batchable(s, r);
    if (batch && !r->valid) {   // refused before it can join a batch
      s->pending.erase(pick);
      finish_invalid(s, r);
      continue;
    }
    const int64_t need = batch ? group_bytes(r) : r->footprint;
    if (s->used + need > s->budget && !s->graveyard.empty()) flush_graveyard(s);
    if (!(s->active.empty() && s->groups.empty()) && s->used + need > s->budget) break;
    // a batch of it and the compatible queued requests; without host memory
    // or a thread for one, the request is served alone
    if (batch && admit_group(s, pick) == FINOM_OK) continue;
    s->pending.erase(pick);
    finom_status rc = admit(s, r);
    if (rc != FINOM_OK) fail(s, r, rc);
    else s->active.push_back(r);
  }
  // progress of the active solves whose launches have completed
  for (Req* r : s->active) {
    if (cudaEventQuery(r->ev) == cudaErrorNotReady) {
      still.push_back(r);
      continue;
    }
    cudaStream_t st = s->streams[r->slot];
    int32_t done = 0;
    int64_t its = 0;
    finom_status rc = finom_solve_poll(r->plan, &done, &its, st);
    if (rc == FINOM_OK && !done) {
      rc = finom_solve_step(r->plan, r->step, st);
      r->step = std::min<int64_t>(2 * r->step, 64);
      if (rc == FINOM_OK && cudaEventRecord(r->ev, st) != cudaSuccess) rc = FINOM_ECUDA;
      if (rc == FINOM_OK) {
        still.push_back(r);
        continue;
      }
    }
    bool more = false;
    if (rc == FINOM_OK) rc = finish(s, r, &more);
    if (rc != FINOM_OK) {
      fail(s, r, rc);
      continue;
    }
    if (more) {
      still.push_back(r);
      continue;
    }
    s->finished.push_back(r);
  }
  s->active.swap(still);
  if (s->graveyard.size() >= kGraveyard || (s->active.empty() && !s->graveyard.empty())) flush_graveyard(s);
  if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
  if (n_pending) *n_pending = (int32_t)s->pending.size();
  if (n_active) *n_active = (int32_t)(s->active.size() + s->groups.size());
  if (n_finished) *n_finished = (int32_t)s->finished.size();
  return FINOM_OK;
}

finom_status finom_server_result(finom_server_t s, int64_t id, finom_server_done* out, double* f, double* g) {
  if (!s || !out) {
    finom::set_error("finom_server_result: null argument");
    return FINOM_EINVAL;
  }
  auto it = find_finished(s, id);
  if (it == s->finished.end()) {
    finom::set_error("finom_server_result: request not finished (or unknown)");
    return FINOM_EPENDING;
  }
  Req* r = *it;
  out->id = r->id;
  out->kind = r->kind;
  out->status = r->status;
  out->result = r->res;
  out->latency_s = r->t_done - r->t_submit;
  out->queue_s = r->t_admit > 0.0 ? r->t_admit - r->t_submit : out->latency_s;
  if (f && !r->f.empty()) std::copy(r->f.begin(), r->f.end(), f);
  if (g && !r->g.empty()) std::copy(r->g.begin(), r->g.end(), g);
  *it = s->finished.back();
  s->finished.pop_back();
  delete r;
  return FINOM_OK;
}

finom_status finom_server_cancel(finom_server_t s, int64_t id) {
  if (!s) {
    finom::set_error("finom_server_cancel: null server");
    return FINOM_EINVAL;
  }
  if (find_finished(s, id) != s->finished.end()) return FINOM_OK;
  try {
    s->graveyard.reserve(s->graveyard.size() + 2);
  } catch (const std::bad_alloc&) {
    finom::set_error("finom_server_cancel: out of host memory");
    return FINOM_ENOMEM;
  }
  for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
    if ((*it)->id != id) continue;
    Req* r = *it;
    s->pending.erase(it);
    r->status = r->res.status = FINOM_ECANCELED;
    r->t_done = now_s();
    s->finished.push_back(r);
    return FINOM_OK;
  }
  for (finom_server_s::Group* g : s->groups) {   // a batched request: when its batch ends
    if (g->collected) continue;
    for (Req* q : g->members) {
      if (q->id != id) continue;
      q->cancelled = true;
      if (std::all_of(g->members.begin(), g->members.end(), [](const Req* m) { return m->cancelled; }))
        g->stop.store(1, std::memory_order_relaxed);
      return FINOM_OK;
    }
  }
  for (auto it = s->active.begin(); it != s->active.end(); ++it) {
    if ((*it)->id != id) continue;
    Req* r = *it;
    s->active.erase(it);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != s->device) cudaSetDevice(s->device);
    cudaStreamSynchronize(s->streams[r->slot]);
    fail(s, r, FINOM_ECANCELED);
    if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
    return FINOM_OK;
  }
  finom::set_error("finom_server_cancel: unknown request id");
  return FINOM_EINVAL;
}

finom_status finom_server_destroy(finom_server_t s) {
  if (!s) return FINOM_OK;
  for (finom_server_s::Group* g : s->groups) {
    g->stop.store(1, std::memory_order_relaxed);
    g->worker.join();
    if (!g->collected)
      for (Req* q : g->members) delete q;
    delete g;
  }
  for (Req* r : s->active) {
    cudaStreamSynchronize(s->streams[r->slot]);
    release(s, r);
    delete r;
  }
  for (Req* r : s->pending) delete r;
  for (Req* r : s->finished) delete r;
  flush_graveyard(s, true);
  collect_reapers(s, true);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  delete s;
  return FINOM_OK;
}

}  // extern "C"
