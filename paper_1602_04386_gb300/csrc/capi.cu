// capi.cu -- host driver of the C-ABI declared in include/fiedler.h.
//
// A solve is three kernel launches on the plan's stream and no host round trip
// in between: the cooperative grid-wide engine builds the large levels of the
// hierarchy, the one-block engine builds and solves the small levels (setup
// below tail_max_n, the coarsest solve and their refinement), and the
// cooperative engine refines the large levels and computes the Rayleigh
// quotient.  The device-resident State carries the hierarchy between them.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fiedler.h"
#include "fz_state.h"
#include "kernels.h"

using fz::State;

namespace {

struct Ticket {
  uint64_t id;
  int64_t n, nnz;
  int32_t *rowptr = nullptr, *col = nullptr;
  void *w = nullptr;
  int w_dtype = 0;
  double *x = nullptr;  // device result vector
  fiedler_result res{};
  fiedler_status st = FIEDLER_EAGAIN;
  bool done = false, canceled = false, running = false;
};

}  // namespace

struct fiedler_plan {
  fiedler_options opt;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0, sms = 0;
  fz::KernelSet ks[2];      // [0] double, [1] float
  int grid_blocks[2][2];    // [type][setup/solve]
  State *d_state = nullptr;
  State *h_state = nullptr; // pinned mirror
  fz::IRed *d_ipart = nullptr;
  double *d_dpart = nullptr;
  char *d_arena = nullptr;
  size_t arena_cap = 0;
  char *d_scratch = nullptr;
  size_t scratch_cap = 0;
  void *d_stage[3] = {nullptr, nullptr, nullptr};
  size_t stage_cap[3] = {0, 0, 0};
  double *d_xout = nullptr;
  size_t xout_cap = 0;
  cudaEvent_t ev[8];
  int profiling = 0;
  int last_type = 1;
  bool have_result = false;
  fiedler_profile prof;
  // batch form
  std::mutex exec_mu;       // one solve on the device state at a time
  std::mutex q_mu;
  std::condition_variable q_cv;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Ticket *> tickets;
  uint64_t next_ticket = 1;
  std::thread worker;
  bool stop = false;
};

namespace {

fiedler_status map_cuda(cudaError_t e) {
  if (e == cudaSuccess) return FIEDLER_OK;
  if (e == cudaErrorMemoryAllocation) return FIEDLER_ENOMEM;
  return FIEDLER_ECUDA;
}

#define CK(x)                                \
  do {                                       \
    cudaError_t e_ = (x);                    \
    if (e_ != cudaSuccess) return map_cuda(e_); \
  } while (0)

fiedler_status ensure(fiedler_plan *p, void **ptr, size_t *cap, size_t bytes) {
  if (*cap >= bytes && *ptr) return FIEDLER_OK;
  if (*ptr) {
    CK(cudaFreeAsync(*ptr, p->stream));
    *ptr = nullptr;
    *cap = 0;
  }
  size_t b = bytes < 256 ? 256 : bytes;
  CK(cudaMallocAsync(ptr, b, p->stream));
  *cap = b;
  return FIEDLER_OK;
}

size_t arena_estimate(int64_t n, int64_t nnz, size_t tsz, bool wf64) {
  // fine level: optional self-loop-free copy, degree, matching, aggregates,
  // colours, permutations, colour-order copy, iterates
  double l0 = 4.0 * (n + 1) + (4.0 + (wf64 ? 8.0 : 4.0)) * nnz + 8.0 * n + 4.0 * n * 3 + 8.0 * n +
              4.0 * (fz::kMaxColors + 1) + 4.0 * (n + 1) + (4.0 + tsz) * nnz + (2.0 * tsz + 4.0) * n;
  // coarse levels together: assume at most 2n vertices and 2nnz entries
  double lc = 2.0 * (4.0 * n + 16.0 * nnz + 8.0 * n + 4.0 * n * 3 + 8.0 * n + 4.0 * n + (4.0 + tsz) * nnz +
                     (2.0 * tsz + 4.0) * n) +
              fz::kMaxLevels * 4.0 * (fz::kMaxColors + 1);
  double slack = fz::kMaxLevels * 24.0 * 256.0 + (1 << 20);
  return (size_t)(l0 + lc + slack);
}

size_t scratch_estimate(int64_t n, int64_t nnz, int nblocks) {
  // one level's scratch, all live at once: colouring (cround + 3 worklists),
  // matching (cand + 3 worklists), Galerkin (9 per-vertex / per-aggregate
  // arrays, (J, slot) keys + FP64 weights per cross entry), colour histogram
  double b = 16.0 * n + 16.0 * n + 4.0 * (n + 1) * 9 + 16.0 * nnz + 4.0 * fz::kMaxColors * nblocks +
             64.0 * 256.0 + (1 << 20);
  return (size_t)b;
}

fiedler_status map_status(int st) {
  switch (st) {
    case fz::ST_OK: return FIEDLER_OK;
    case fz::ST_EINVAL: return FIEDLER_EINVAL;
    case fz::ST_ENOMEM: return FIEDLER_ENOMEM;
    case fz::ST_EDISC: return FIEDLER_EDISCONNECTED;
    case fz::ST_ENOTCONV: return FIEDLER_ENOTCONVERGED;
    case fz::ST_ETIMEOUT: return FIEDLER_ETIMEOUT;
    case fz::ST_EDEGEN: return FIEDLER_EDEGENERATE;
    case fz::ST_ENOTSUP: return FIEDLER_ENOTSUP;
    default: return FIEDLER_ECUDA;
  }
}

const char *kPhaseNames[fz::PH_COUNT] = {"ingest", "colour", "reorder", "match", "aggregate", "galerkin",
                                         "coarsest", "prolong", "gauss_seidel", "power_iter", "final"};

fiedler_status launch(fiedler_plan *p, const void *fn, int grid, int block, bool coop, int slot) {
  void *args[] = {(void *)&p->d_state};
  if (p->profiling) CK(cudaEventRecord(p->ev[2 + 2 * slot], p->stream));
  if (coop) CK(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, 0, p->stream));
  else CK(cudaLaunchKernel(fn, dim3(grid), dim3(block), args, 0, p->stream));
  if (p->profiling) CK(cudaEventRecord(p->ev[3 + 2 * slot], p->stream));
  p->prof.kernel_launches_by[slot]++;
  p->prof.kernel_launches++;
  return FIEDLER_OK;
}

// one solve on device-resident input; x_dev may be NULL
fiedler_status run_solve(fiedler_plan *p, int64_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col,
                         const void *w, int w_f64, double *x_dev, fiedler_result *res) {
  const int type = p->opt.precision == FIEDLER_FP64 ? 0 : 1;
  const size_t tsz = type == 0 ? 8 : 4;
  const fz::KernelSet &K = p->ks[type];
  const int gmax = p->grid_blocks[type][0] > p->grid_blocks[type][1] ? p->grid_blocks[type][0]
                                                                       : p->grid_blocks[type][1];
  size_t abytes = arena_estimate(n, nnz, tsz, w_f64 != 0);
  size_t sbytes = scratch_estimate(n, nnz, gmax);
  fiedler_status st = FIEDLER_OK;
  for (int attempt = 0; attempt < 4; attempt++) {
    if ((st = ensure(p, (void **)&p->d_arena, &p->arena_cap, abytes)) != FIEDLER_OK) return st;
    if ((st = ensure(p, (void **)&p->d_scratch, &p->scratch_cap, sbytes)) != FIEDLER_OK) return st;
    State *h = p->h_state;
    memset(h, 0, sizeof(State));
    fz::Opts &o = h->opt;
    o.precision = p->opt.precision;
    o.coarse_max_n = p->opt.coarse_max_n;
    o.max_levels = p->opt.max_levels;
    o.gs_sweeps = p->opt.gs_sweeps;
    o.pi_max_iters = p->opt.pi_max_iters;
    o.pi_max_iters_coarsest = p->opt.pi_max_iters_coarsest;
    o.tie_rule = p->opt.tie_rule;
    o.validate = p->opt.validate;
    o.tail_max_n = p->opt.tail_max_n;
    o.fault_inject = p->opt.fault_inject;
    o.stall_ratio = p->opt.stall_ratio;
    o.pi_cos_tol = p->opt.pi_cos_tol;
    o.resid_tol = p->opt.resid_tol;
    // annihilation guard on the deflated norm of a unit vector: above the
    // rounding noise of the fused variance sum x^2 - (sum x)^2 / n
    o.guard = type == 0 ? ldexp(1.0, -20) : ldexp(1.0, -16);
    o.seed = p->opt.seed;
    o.barrier_timeout_ns = (unsigned long long)p->opt.barrier_timeout_ms * 1000000ull;
    h->bad_index = LLONG_MAX;
    h->n0 = (int)n;
    h->nnz0 = (int)nnz;
    h->in_rowptr = rowptr;
    h->in_col = col;
    h->in_w = w;
    h->in_w_f64 = w_f64;
    h->arena = p->d_arena;
    h->arena_size = p->arena_cap;
    h->scratch = p->d_scratch;
    h->scratch_size = p->scratch_cap;
    h->xout = x_dev;
    h->ipart = p->d_ipart;
    h->dpart = p->d_dpart;
    memset(&p->prof, 0, sizeof(p->prof));
    CK(cudaMemcpyAsync(p->d_state, h, sizeof(State), cudaMemcpyHostToDevice, p->stream));
    CK(cudaEventRecord(p->ev[0], p->stream));
    const bool big = n > p->opt.tail_max_n;
    if (big && (st = launch(p, K.grid_setup, p->grid_blocks[type][0], fz::kGridThreads, true, 0)) != FIEDLER_OK)
      return st;
    if ((st = launch(p, K.cta, 1, fz::kCtaThreads, false, 1)) != FIEDLER_OK) return st;
    if (big && (st = launch(p, K.grid_solve, p->grid_blocks[type][1], fz::kGridThreads, true, 2)) != FIEDLER_OK)
      return st;
    CK(cudaEventRecord(p->ev[1], p->stream));
    CK(cudaMemcpyAsync(h, p->d_state, sizeof(State), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    p->have_result = true;
    p->last_type = type;
    if (h->status == fz::ST_ARENA) {
      abytes = abytes * 2;
      continue;
    }
    if (h->status == fz::ST_SCRATCH) {
      sbytes = sbytes * 2;
      continue;
    }
    break;
  }
  State *h = p->h_state;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, p->ev[0], p->ev[1]);
  // profile bookkeeping
  fiedler_profile &pr = p->prof;
  pr.n_kernels = 3;
  for (int k = 0; k < 3; k++) {
    pr.kernel_name[k] = K.names[k];
    if (p->profiling && pr.kernel_launches_by[k] > 0) {
      float km = 0.f;
      cudaEventElapsedTime(&km, p->ev[2 + 2 * k], p->ev[3 + 2 * k]);
      pr.kernel_ms[k] = km;
    }
  }
  pr.n_phases = fz::PH_COUNT;
  for (int ph = 0; ph < fz::PH_COUNT; ph++) {
    pr.phase_name[ph] = kPhaseNames[ph];
    for (int kd = 0; kd < 2; kd++) {
      pr.phase_ms[kd][ph] = h->phase_ns[kd][ph] * 1e-6;
      pr.phase_bytes[kd][ph] = h->phase_bytes[kd][ph];
    }
  }
  for (int ph = 0; ph < fz::PH_COUNT; ph++) {
    const int k = ph <= fz::PH_GALERKIN ? 0 : 2;
    pr.kernel_bytes[k] += h->phase_bytes[0][ph];
    pr.kernel_bytes[1] += h->phase_bytes[1][ph];
  }
  fiedler_status out = map_status(h->status);
  if (out == FIEDLER_OK && !h->finalized) out = FIEDLER_ECUDA;
  if (out == FIEDLER_OK && h->capped) out = FIEDLER_ENOTCONVERGED;
  if (res) {
    res->ms = ms;
    res->levels = h->nlevels;
    res->coarsest_n = h->nlevels > 0 ? h->lv[h->coarsest].n : 0;
    res->bad_index = h->bad_index == LLONG_MAX ? -1 : h->bad_index;
    if (out == FIEDLER_OK || out == FIEDLER_ENOTCONVERGED) {
      res->lambda2 = h->lambda;
      res->residual = h->residual;
      res->ortho = h->ortho;
      res->pi_iters_total = h->pi_total;
      res->gs_sweeps_total = h->gs_total;
    }
    res->status = out;
  }
  return out;
}

fiedler_status check_graph(const fiedler_graph *g, fiedler_result *res) {
  if (!g) return FIEDLER_EINVAL;
  bool bad = g->n < 2 || g->n >= INT_MAX || g->nnz < 0 || g->nnz >= INT_MAX || !g->rowptr ||
             (g->nnz > 0 && (!g->col || !g->w)) || (g->w_dtype != FIEDLER_W_F32 && g->w_dtype != FIEDLER_W_F64);
  if (bad) {
    if (res) {
      res->bad_index = 0;
      res->status = (g->nnz >= INT_MAX || g->n >= INT_MAX) ? FIEDLER_ENOTSUP : FIEDLER_EINVAL;
    }
    return (g->nnz >= INT_MAX || g->n >= INT_MAX) ? FIEDLER_ENOTSUP : FIEDLER_EINVAL;
  }
  return FIEDLER_OK;
}

fiedler_status solve_locked(fiedler_plan *p, const fiedler_graph *g, fiedler_result *res) {
  fiedler_status st = check_graph(g, res);
  if (st != FIEDLER_OK) return st;
  const int64_t n = g->n, nnz = g->nnz;
  const size_t wsz = g->w_dtype == FIEDLER_W_F64 ? 8 : 4;
  const int32_t *rp = g->rowptr, *ci = g->col;
  const void *w = g->w;
  if (!g->on_device) {
    if ((st = ensure(p, &p->d_stage[0], &p->stage_cap[0], 4 * (size_t)(n + 1))) != FIEDLER_OK) return st;
    if ((st = ensure(p, &p->d_stage[1], &p->stage_cap[1], 4 * (size_t)(nnz > 0 ? nnz : 1))) != FIEDLER_OK) return st;
    if ((st = ensure(p, &p->d_stage[2], &p->stage_cap[2], wsz * (size_t)(nnz > 0 ? nnz : 1))) != FIEDLER_OK)
      return st;
    CK(cudaMemcpyAsync(p->d_stage[0], rp, 4 * (size_t)(n + 1), cudaMemcpyHostToDevice, p->stream));
    if (nnz > 0) {
      CK(cudaMemcpyAsync(p->d_stage[1], ci, 4 * (size_t)nnz, cudaMemcpyHostToDevice, p->stream));
      CK(cudaMemcpyAsync(p->d_stage[2], w, wsz * (size_t)nnz, cudaMemcpyHostToDevice, p->stream));
    }
    rp = (const int32_t *)p->d_stage[0];
    ci = (const int32_t *)p->d_stage[1];
    w = p->d_stage[2];
  }
  double *xd = nullptr;
  bool host_x = false;
  if (res && res->x) {
    if (res->x_on_device) {
      xd = res->x;
    } else {
      if ((st = ensure(p, (void **)&p->d_xout, &p->xout_cap, 8 * (size_t)n)) != FIEDLER_OK) return st;
      xd = p->d_xout;
      host_x = true;
    }
  }
  st = run_solve(p, n, nnz, rp, ci, w, g->w_dtype == FIEDLER_W_F64, xd, res);
  if (host_x && (st == FIEDLER_OK || st == FIEDLER_ENOTCONVERGED)) {
    CK(cudaMemcpyAsync(res->x, xd, 8 * (size_t)n, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
  }
  return st;
}

// ---- batch form: a worker thread drains the ticket queue -------------------
void worker_main(fiedler_plan *p) {
  cudaSetDevice(p->device);
  for (;;) {
    Ticket *t = nullptr;
    {
      std::unique_lock<std::mutex> lk(p->q_mu);
      p->q_cv.wait(lk, [&] { return p->stop || !p->queue.empty(); });
      if (p->stop) return;
      uint64_t id = p->queue.front();
      p->queue.pop_front();
      auto it = p->tickets.find(id);
      if (it == p->tickets.end()) continue;
      t = it->second;
      if (t->canceled) {
        t->st = FIEDLER_ECANCELED;
        t->done = true;
        p->q_cv.notify_all();
        continue;
      }
      t->running = true;
    }
    fiedler_graph g{t->n, t->nnz, t->rowptr, t->col, t->w, t->w_dtype, 1};
    fiedler_result r{};
    r.x = t->x;
    r.x_on_device = 1;
    fiedler_status st;
    {
      std::lock_guard<std::mutex> ex(p->exec_mu);
      st = solve_locked(p, &g, &r);
    }
    std::lock_guard<std::mutex> lk(p->q_mu);
    t->res = r;
    t->st = st;
    t->done = true;
    t->running = false;
    p->q_cv.notify_all();
  }
}

void free_ticket(fiedler_plan *p, Ticket *t) {
  cudaFree(t->rowptr);
  cudaFree(t->col);
  cudaFree(t->w);
  cudaFree(t->x);
  delete t;
}

}  // namespace

extern "C" {

void fiedler_options_default(fiedler_options *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = FIEDLER_FP32_FP64RED;
  o->coarse_max_n = 25;
  o->max_levels = 30;
  o->stall_ratio = 0.9;
  o->gs_sweeps = 2;
  o->pi_max_iters = 10000;
  o->pi_max_iters_coarsest = 100000;
  o->pi_cos_tol = 1e-6;
  o->resid_tol = 0.0;
  o->tie_rule = FIEDLER_TIE_HASHED;
  o->seed = 20160214ull;
  o->validate = 1;
  o->tail_max_n = 4096;
  o->barrier_timeout_ms = 5000;
  o->fault_inject = 0;
}

fiedler_status fiedler_plan_create(const fiedler_options *opts, void *cuda_stream, fiedler_plan **out) {
  if (!out) return FIEDLER_EINVAL;
  *out = nullptr;
  fiedler_options o;
  if (opts) o = *opts;
  else fiedler_options_default(&o);
  if ((o.precision != FIEDLER_FP64 && o.precision != FIEDLER_FP32_FP64RED) || o.coarse_max_n < 1 ||
      o.max_levels < 1 || o.max_levels > fz::kMaxLevels || !(o.stall_ratio > 0.0 && o.stall_ratio <= 1.0) ||
      o.gs_sweeps < 0 || o.pi_max_iters < 0 || o.pi_max_iters_coarsest < 0 || !(o.pi_cos_tol >= 0.0) ||
      !(o.resid_tol >= 0.0) || (o.tie_rule != 0 && o.tie_rule != 1) || o.tail_max_n < 1 ||
      o.barrier_timeout_ms < 1)
    return FIEDLER_EINVAL;
  fiedler_plan *p = new (std::nothrow) fiedler_plan();
  if (!p) return FIEDLER_ENOMEM;
  p->opt = o;
  fiedler_status st = FIEDLER_OK;
  auto fail = [&](fiedler_status s) {
    fiedler_plan_destroy(p);
    return s;
  };
  if (cudaGetDevice(&p->device) != cudaSuccess) return fail(FIEDLER_ECUDA);
  if (cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess)
    return fail(FIEDLER_ECUDA);
  if (cuda_stream) {
    p->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(FIEDLER_ECUDA);
    p->own_stream = true;
  }
  fz::kernels_f64(&p->ks[0]);
  fz::kernels_f32(&p->ks[1]);
  for (int t = 0; t < 2; t++) {
    const void *fns[2] = {p->ks[t].grid_setup, p->ks[t].grid_solve};
    for (int k = 0; k < 2; k++) {
      int bps = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fns[k], fz::kGridThreads, 0) != cudaSuccess || bps < 1)
        return fail(FIEDLER_ECUDA);
      int g = bps * p->sms;
      p->grid_blocks[t][k] = g > fz::kMaxBlocks ? fz::kMaxBlocks : g;
    }
  }
  if (cudaMalloc(&p->d_state, sizeof(State)) != cudaSuccess) return fail(FIEDLER_ENOMEM);
  if (cudaMalloc(&p->d_ipart, sizeof(fz::IRed) * 2 * fz::kMaxBlocks) != cudaSuccess) return fail(FIEDLER_ENOMEM);
  if (cudaMalloc(&p->d_dpart, sizeof(double) * 2 * fz::kMaxBlocks * fz::kDSum) != cudaSuccess)
    return fail(FIEDLER_ENOMEM);
  if (cudaMallocHost(&p->h_state, sizeof(State)) != cudaSuccess) return fail(FIEDLER_ENOMEM);
  for (int i = 0; i < 8; i++)
    if (cudaEventCreate(&p->ev[i]) != cudaSuccess) return fail(FIEDLER_ECUDA);
  p->worker = std::thread(worker_main, p);
  *out = p;
  (void)st;
  return FIEDLER_OK;
}

fiedler_status fiedler_solve(fiedler_plan *p, const fiedler_graph *g, fiedler_result *res) {
  if (!p) return FIEDLER_EINVAL;
  std::lock_guard<std::mutex> ex(p->exec_mu);
  fiedler_status st = solve_locked(p, g, res);
  if (res) res->status = st;
  return st;
}

fiedler_status fiedler_batch_submit(fiedler_plan *p, const fiedler_graph *g, uint64_t *ticket) {
  if (!p || !ticket) return FIEDLER_EINVAL;
  fiedler_status st = check_graph(g, nullptr);
  if (st != FIEDLER_OK) return st;
  Ticket *t = new (std::nothrow) Ticket();
  if (!t) return FIEDLER_ENOMEM;
  t->n = g->n;
  t->nnz = g->nnz;
  t->w_dtype = g->w_dtype;
  const size_t wsz = g->w_dtype == FIEDLER_W_F64 ? 8 : 4;
  const size_t m = (size_t)(g->nnz > 0 ? g->nnz : 1);
  cudaError_t e = cudaMalloc(&t->rowptr, 4 * (size_t)(g->n + 1));
  if (e == cudaSuccess) e = cudaMalloc(&t->col, 4 * m);
  if (e == cudaSuccess) e = cudaMalloc(&t->w, wsz * m);
  if (e == cudaSuccess) e = cudaMalloc(&t->x, 8 * (size_t)g->n);
  const cudaMemcpyKind kind = g->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (e == cudaSuccess) e = cudaMemcpy(t->rowptr, g->rowptr, 4 * (size_t)(g->n + 1), kind);
  if (e == cudaSuccess && g->nnz > 0) e = cudaMemcpy(t->col, g->col, 4 * (size_t)g->nnz, kind);
  if (e == cudaSuccess && g->nnz > 0) e = cudaMemcpy(t->w, g->w, wsz * (size_t)g->nnz, kind);
  if (e != cudaSuccess) {
    free_ticket(p, t);
    return map_cuda(e);
  }
  std::lock_guard<std::mutex> lk(p->q_mu);
  t->id = p->next_ticket++;
  p->tickets[t->id] = t;
  p->queue.push_back(t->id);
  *ticket = t->id;
  p->q_cv.notify_all();
  return FIEDLER_OK;
}

fiedler_status fiedler_poll(fiedler_plan *p, uint64_t ticket, int timeout_ms, fiedler_result *res) {
  if (!p) return FIEDLER_EINVAL;
  std::unique_lock<std::mutex> lk(p->q_mu);
  auto it = p->tickets.find(ticket);
  if (it == p->tickets.end()) return FIEDLER_EINVAL;
  Ticket *t = it->second;
  if (!t->done) {
    if (timeout_ms == 0) return FIEDLER_EAGAIN;
    if (timeout_ms < 0) p->q_cv.wait(lk, [&] { return t->done; });
    else if (!p->q_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return t->done; }))
      return FIEDLER_EAGAIN;
  }
  fiedler_status st = t->st;
  if (res) {
    double *x = res->x;
    int xod = res->x_on_device;
    *res = t->res;
    res->x = x;
    res->x_on_device = xod;
    res->status = st;
    if (x && (st == FIEDLER_OK || st == FIEDLER_ENOTCONVERGED)) {
      cudaError_t e = cudaMemcpy(x, t->x, 8 * (size_t)t->n, xod ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) st = map_cuda(e);
    }
  }
  p->tickets.erase(it);
  free_ticket(p, t);
  return st;
}

fiedler_status fiedler_cancel(fiedler_plan *p, uint64_t ticket) {
  if (!p) return FIEDLER_EINVAL;
  std::lock_guard<std::mutex> lk(p->q_mu);
  auto it = p->tickets.find(ticket);
  if (it == p->tickets.end()) return FIEDLER_EINVAL;
  Ticket *t = it->second;
  if (!t->done && !t->running) t->canceled = true;
  return FIEDLER_OK;
}

void fiedler_plan_destroy(fiedler_plan *p) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lk(p->q_mu);
    p->stop = true;
    p->q_cv.notify_all();
  }
  if (p->worker.joinable()) p->worker.join();
  for (auto &kv : p->tickets) free_ticket(p, kv.second);
  p->tickets.clear();
  if (p->stream) cudaStreamSynchronize(p->stream);
  if (p->d_arena) cudaFreeAsync(p->d_arena, p->stream);
  if (p->d_scratch) cudaFreeAsync(p->d_scratch, p->stream);
  for (int i = 0; i < 3; i++)
    if (p->d_stage[i]) cudaFreeAsync(p->d_stage[i], p->stream);
  if (p->d_xout) cudaFreeAsync(p->d_xout, p->stream);
  if (p->stream) cudaStreamSynchronize(p->stream);
  if (p->d_state) cudaFree(p->d_state);
  if (p->d_ipart) cudaFree(p->d_ipart);
  if (p->d_dpart) cudaFree(p->d_dpart);
  if (p->h_state) cudaFreeHost(p->h_state);
  for (int i = 0; i < 8; i++)
    if (p->ev[i]) cudaEventDestroy(p->ev[i]);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

const char *fiedler_status_str(fiedler_status s) {
  switch (s) {
    case FIEDLER_OK: return "ok";
    case FIEDLER_EAGAIN: return "still in flight";
    case FIEDLER_EINVAL: return "invalid argument or malformed graph";
    case FIEDLER_ENOMEM: return "out of device memory";
    case FIEDLER_EDISCONNECTED: return "graph is not connected";
    case FIEDLER_ENOTCONVERGED: return "power iteration hit its cap (result returned)";
    case FIEDLER_ETIMEOUT: return "bounded device wait timed out";
    case FIEDLER_ECUDA: return "CUDA runtime error";
    case FIEDLER_ECANCELED: return "canceled";
    case FIEDLER_EDEGENERATE: return "iterate vanished after deflation";
    case FIEDLER_ENOTSUP: return "size limit exceeded";
  }
  return "unknown status";
}

int fiedler_plan_num_levels(const fiedler_plan *p) {
  if (!p || !p->have_result) return 0;
  return p->h_state->nlevels;
}

fiedler_status fiedler_plan_level_info(const fiedler_plan *p, int l, fiedler_level_info *info) {
  if (!p || !info || !p->have_result || l < 0 || l >= p->h_state->nlevels) return FIEDLER_EINVAL;
  const fz::Level &L = p->h_state->lv[l];
  info->n = L.n;
  info->nnz = L.nnz;
  info->nc = L.agg ? L.nc : 0;
  info->ncolors = L.ncolors;
  info->match_rounds = L.match_rounds;
  info->color_rounds = L.color_rounds;
  info->gs_sweeps = L.gs_sweeps;
  info->pi_iters = L.pi_iters;
  info->sigma = L.sigma;
  info->last_cos = L.last_cos;
  for (int i = 0; i < 16; i++) info->phase_ms[i] = i < fz::PH_COUNT ? (float)(p->h_state->level_ns[l][i] * 1e-6) : 0.f;
  return FIEDLER_OK;
}

fiedler_status fiedler_plan_copy_level(const fiedler_plan *cp, int l, int32_t *rowptr, int32_t *col, double *w,
                                       double *d, int32_t *agg, int32_t *mate, int32_t *color) {
  fiedler_plan *p = const_cast<fiedler_plan *>(cp);
  if (!p || !p->have_result || l < 0 || l >= p->h_state->nlevels) return FIEDLER_EINVAL;
  std::lock_guard<std::mutex> ex(p->exec_mu);
  const fz::Level &L = p->h_state->lv[l];
  const size_t n = (size_t)L.n, m = (size_t)L.nnz;
  if (rowptr) CK(cudaMemcpy(rowptr, L.rowptr, 4 * (n + 1), cudaMemcpyDeviceToHost));
  if (col && m) CK(cudaMemcpy(col, L.col, 4 * m, cudaMemcpyDeviceToHost));
  if (w && m) {
    if (L.w64) {
      CK(cudaMemcpy(w, L.w64, 8 * m, cudaMemcpyDeviceToHost));
    } else {
      std::vector<float> tmp(m);
      CK(cudaMemcpy(tmp.data(), L.w32, 4 * m, cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < m; i++) w[i] = tmp[i];
    }
  }
  if (d) CK(cudaMemcpy(d, L.d, 8 * n, cudaMemcpyDeviceToHost));
  if (agg && L.agg && l + 1 < p->h_state->nlevels) CK(cudaMemcpy(agg, L.agg, 4 * n, cudaMemcpyDeviceToHost));
  if (mate && L.mate) CK(cudaMemcpy(mate, L.mate, 4 * n, cudaMemcpyDeviceToHost));
  if (color && L.color) CK(cudaMemcpy(color, L.color, 4 * n, cudaMemcpyDeviceToHost));
  return FIEDLER_OK;
}

fiedler_status fiedler_plan_set_profiling(fiedler_plan *p, int on) {
  if (!p) return FIEDLER_EINVAL;
  p->profiling = on ? 1 : 0;
  return FIEDLER_OK;
}

fiedler_status fiedler_plan_get_profile(const fiedler_plan *p, fiedler_profile *out) {
  if (!p || !out) return FIEDLER_EINVAL;
  *out = p->prof;
  return FIEDLER_OK;
}

}  // extern "C"
