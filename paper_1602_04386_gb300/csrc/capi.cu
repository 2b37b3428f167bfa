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

#include <algorithm>
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
  size_t footprint = 0;  // device bytes while in flight (admission)
  std::chrono::steady_clock::time_point t_submit;
  fiedler_result res{};
  fiedler_status st = FIEDLER_EAGAIN;
  bool done = false, canceled = false, running = false;
};

// One graph of a batched launch.
struct BatchItem {
  int64_t n, nnz;
  const int32_t *rp, *ci;
  const void *w;
  int wf64;
  bool host_in;          // inputs are host pointers: packed into the staging region
  double *user_x;        // caller's output (may be NULL)
  int user_x_dev;
  size_t arena_b, scratch_b;
  size_t in_off, x_off;  // offsets in the input / output staging regions
  fiedler_result *res;   // where the result goes (solve_batch) or NULL (ticket)
  Ticket *ticket;
  int st;                // internal status after the run
};

// A batched launch in preparation or in flight: own stream, device buffer,
// pinned staging, completion event.
struct BatchCtx {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t done = nullptr;
  char *d_buf = nullptr;
  size_t d_cap = 0;
  char *h_buf = nullptr;  // pinned
  size_t h_cap = 0;
  std::vector<BatchItem> items;
  size_t footprint = 0;
  bool busy = false;
  int type = 1;
  // layout (offsets in d_buf / h_buf)
  size_t d_states, d_counter, d_scratch, slot_bytes, d_arena, d_in, d_x, d_total;
  size_t h_states, h_in, h_x, h_total, in_bytes, x_bytes;
  int nslots = 0;
};

}  // namespace

struct fiedler_plan {
  fiedler_options opt;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0, sms = 0;
  fz::KernelSet ks[2];      // [0] double, [1] float
  int grid_blocks[2][2];    // [type][setup/solve]
  int batch_slots[2];       // resident blocks of the batched kernel
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
  cudaEvent_t ev[10];         // [0,1] solve, [2..7] its kernels, [8,9] batched kernel
  int profiling = 0;
  int last_type = 1;
  bool have_result = false;
  fiedler_profile prof;
  BatchCtx bsync;           // fiedler_solve_batch (plan stream)
  BatchCtx bserve[4];       // serving launches (own streams)
  // serving form
  std::mutex exec_mu;       // one solve on the device state at a time
  std::mutex q_mu;
  std::condition_variable q_cv;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Ticket *> tickets;
  uint64_t next_ticket = 1;
  std::thread worker;
  bool stop = false;
  size_t inflight_bytes = 0, peak_inflight = 0;
  uint64_t n_submitted = 0, n_completed = 0, n_batches = 0, n_batched_tickets = 0;
  std::vector<float> latencies_ms;
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

void fill_opts(fz::Opts &o, const fiedler_options &u, int type) {
  o.precision = u.precision;
  o.coarse_max_n = u.coarse_max_n;
  o.max_levels = u.max_levels;
  o.gs_sweeps = u.gs_sweeps;
  o.pi_max_iters = u.pi_max_iters;
  o.pi_max_iters_coarsest = u.pi_max_iters_coarsest;
  o.tie_rule = u.tie_rule;
  o.validate = u.validate;
  o.tail_max_n = u.tail_max_n;
  o.tail_max_nnz = u.tail_max_nnz;
  o.fault_inject = u.fault_inject;
  o.stall_ratio = u.stall_ratio;
  o.pi_cos_tol = u.pi_cos_tol;
  o.resid_tol = u.resid_tol;
  // annihilation guard on the deflated norm of a unit vector: above the
  // rounding noise of the fused variance sum x^2 - (sum x)^2 / n
  o.guard = type == 0 ? ldexp(1.0, -20) : ldexp(1.0, -16);
  o.seed = u.seed;
  o.barrier_timeout_ns = (unsigned long long)u.barrier_timeout_ms * 1000000ull;
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
    fill_opts(h->opt, p->opt, type);
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
    // the engine's rule for the fine level (it may still hand the level to the
    // one-block kernel after ingest drops self-loops; a launch with nothing
    // eligible returns at once)
    const bool tiny = n <= fz::kTinyN && nnz <= fz::kTinyNnz;
    const bool big = !tiny && (n > p->opt.tail_max_n || nnz > p->opt.tail_max_nnz);
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

// ---- batched form --------------------------------------------------------
size_t r256(size_t b) { return (b + 255u) & ~(size_t)255u; }

fiedler_status ctx_reserve(BatchCtx &c, size_t dbytes, size_t hbytes) {
  if (c.d_cap < dbytes) {
    if (c.d_buf) CK(cudaFreeAsync(c.d_buf, c.stream));
    c.d_buf = nullptr;
    c.d_cap = 0;
    CK(cudaMallocAsync((void **)&c.d_buf, dbytes, c.stream));
    c.d_cap = dbytes;
  }
  if (c.h_cap < hbytes) {
    if (c.h_buf) {
      CK(cudaStreamSynchronize(c.stream));
      cudaFreeHost(c.h_buf);
    }
    c.h_buf = nullptr;
    c.h_cap = 0;
    CK(cudaMallocHost((void **)&c.h_buf, hbytes));
    c.h_cap = hbytes;
  }
  return FIEDLER_OK;
}

// device bytes one graph holds while its batch is in flight (admission)
size_t item_footprint(int64_t n, int64_t nnz, size_t tsz, bool wf64) {
  return r256(sizeof(State)) + r256(arena_estimate(n, nnz, tsz, wf64)) + r256(scratch_estimate(n, nnz, 1));
}

// Lays out and queues one batched launch of c.items on c.stream (asynchronous).
// The items are ordered by decreasing size so the largest graphs start first.
fiedler_status batch_launch(fiedler_plan *p, BatchCtx &c, double arena_scale) {
  const int type = c.type;
  const size_t tsz = type == 0 ? 8 : 4;
  std::stable_sort(c.items.begin(), c.items.end(),
                   [](const BatchItem &a, const BatchItem &b) { return a.nnz + a.n > b.nnz + b.n; });
  const int count = (int)c.items.size();
  const int nslots = std::min(count, p->batch_slots[type]);
  size_t slot = 0, arenas = 0, in_b = 0, x_b = 0;
  for (auto &it : c.items) {
    it.arena_b = r256((size_t)(arena_estimate(it.n, it.nnz, tsz, it.wf64) * arena_scale));
    it.scratch_b = r256((size_t)(scratch_estimate(it.n, it.nnz, 1) * arena_scale));
    slot = std::max(slot, it.scratch_b);
    arenas += it.arena_b;
    if (it.host_in) {
      it.in_off = in_b;
      in_b += r256(4 * (size_t)(it.n + 1)) + r256(4 * (size_t)std::max<int64_t>(it.nnz, 1)) +
              r256((it.wf64 ? 8 : 4) * (size_t)std::max<int64_t>(it.nnz, 1));
    }
    if (it.user_x && !it.user_x_dev) {
      it.x_off = x_b;
      x_b += r256(8 * (size_t)it.n);
    }
  }
  const size_t states_b = r256(sizeof(State) * (size_t)count);
  c.nslots = nslots;
  c.slot_bytes = slot;
  c.d_states = 0;
  c.d_counter = states_b;
  c.d_scratch = c.d_counter + 256;
  c.d_arena = c.d_scratch + slot * (size_t)nslots;
  c.d_in = c.d_arena + arenas;
  c.d_x = c.d_in + in_b;
  c.d_total = c.d_x + x_b;
  c.h_states = 0;
  c.h_in = states_b;
  c.h_x = c.h_in + in_b;
  c.h_total = c.h_x + x_b;
  c.in_bytes = in_b;
  c.x_bytes = x_b;
  fiedler_status st = ctx_reserve(c, c.d_total, c.h_total);
  if (st != FIEDLER_OK) return st;
  // host-side state of every graph, packed inputs
  State *hs = (State *)(c.h_buf + c.h_states);
  size_t aoff = c.d_arena;
  for (int i = 0; i < count; i++) {
    BatchItem &it = c.items[i];
    State *h = hs + i;
    memset(h, 0, sizeof(State));
    fill_opts(h->opt, p->opt, type);
    h->opt.tail_max_n = INT_MAX;  // every level in the one-block engine
    h->opt.tail_max_nnz = INT_MAX;
    h->opt.fault_inject = 0;
    h->bad_index = LLONG_MAX;
    h->n0 = (int)it.n;
    h->nnz0 = (int)it.nnz;
    if (it.host_in) {
      char *hin = c.h_buf + c.h_in + it.in_off;
      char *din = c.d_buf + c.d_in + it.in_off;
      const size_t rb = r256(4 * (size_t)(it.n + 1)), cb = r256(4 * (size_t)std::max<int64_t>(it.nnz, 1));
      memcpy(hin, it.rp, 4 * (size_t)(it.n + 1));
      if (it.nnz > 0) {
        memcpy(hin + rb, it.ci, 4 * (size_t)it.nnz);
        memcpy(hin + rb + cb, it.w, (it.wf64 ? 8 : 4) * (size_t)it.nnz);
      }
      h->in_rowptr = (const int *)din;
      h->in_col = (const int *)(din + rb);
      h->in_w = din + rb + cb;
    } else {
      h->in_rowptr = it.rp;
      h->in_col = it.ci;
      h->in_w = it.w;
    }
    h->in_w_f64 = it.wf64;
    h->arena = c.d_buf + aoff;
    h->arena_size = it.arena_b;
    aoff += it.arena_b;
    h->xout = it.user_x ? (it.user_x_dev ? it.user_x : (double *)(c.d_buf + c.d_x + it.x_off)) : nullptr;
  }
  if (in_b) CK(cudaMemcpyAsync(c.d_buf + c.d_in, c.h_buf + c.h_in, in_b, cudaMemcpyHostToDevice, c.stream));
  CK(cudaMemcpyAsync(c.d_buf + c.d_states, hs, sizeof(State) * (size_t)count, cudaMemcpyHostToDevice, c.stream));
  CK(cudaMemsetAsync(c.d_buf + c.d_counter, 0, 4, c.stream));
  State *d_states = (State *)(c.d_buf + c.d_states);
  int *d_counter = (int *)(c.d_buf + c.d_counter);
  char *d_scratch = c.d_buf + c.d_scratch;
  unsigned long long slot_bytes = c.slot_bytes;
  void *args[] = {(void *)&d_states, (void *)&count, (void *)&d_counter, (void *)&d_scratch, (void *)&slot_bytes};
  const bool prof = p->profiling && &c == &p->bsync;
  if (prof) CK(cudaEventRecord(p->ev[8], c.stream));
  CK(cudaLaunchKernel(p->ks[type].batch, dim3(nslots), dim3(fz::kCtaThreads), args, 0, c.stream));
  if (prof) CK(cudaEventRecord(p->ev[9], c.stream));
  CK(cudaMemcpyAsync(hs, c.d_buf + c.d_states, sizeof(State) * (size_t)count, cudaMemcpyDeviceToHost, c.stream));
  if (x_b) CK(cudaMemcpyAsync(c.h_buf + c.h_x, c.d_buf + c.d_x, x_b, cudaMemcpyDeviceToHost, c.stream));
  CK(cudaEventRecord(c.done, c.stream));
  return FIEDLER_OK;
}

// Reads back one finished launch; results of items whose hierarchy outgrew
// its arena are left with st = ST_ARENA / ST_SCRATCH for a rerun.
void batch_collect(BatchCtx &c) {
  State *hs = (State *)(c.h_buf + c.h_states);
  for (size_t i = 0; i < c.items.size(); i++) {
    BatchItem &it = c.items[i];
    const State *h = hs + i;
    it.st = h->status;
    fiedler_result r{};
    fiedler_status out = map_status(h->status);
    if (out == FIEDLER_OK && !h->finalized) out = FIEDLER_ECUDA;
    if (out == FIEDLER_OK && h->capped) out = FIEDLER_ENOTCONVERGED;
    r.levels = h->nlevels;
    r.coarsest_n = h->nlevels > 0 ? h->lv[h->coarsest].n : 0;
    r.bad_index = h->bad_index == LLONG_MAX ? -1 : h->bad_index;
    if (out == FIEDLER_OK || out == FIEDLER_ENOTCONVERGED) {
      r.lambda2 = h->lambda;
      r.residual = h->residual;
      r.ortho = h->ortho;
      r.pi_iters_total = h->pi_total;
      r.gs_sweeps_total = h->gs_total;
      if (it.user_x && !it.user_x_dev) memcpy(it.user_x, c.h_buf + c.h_x + it.x_off, 8 * (size_t)it.n);
    }
    r.x = it.user_x;
    r.x_on_device = it.user_x_dev;
    r.status = out;
    if (it.res) *it.res = r;
    if (it.ticket) {
      it.ticket->res = r;
      it.ticket->st = out;
    }
  }
}

bool needs_rerun(int st) { return st == fz::ST_ARENA || st == fz::ST_SCRATCH; }

// Profile of a finished synchronous batched launch (profiling on): the
// kernel's CUDA-event time, and per phase the device time summed over the
// graphs (block-time, not wall time) with the algorithmic bytes.
void batch_profile(fiedler_plan *p, BatchCtx &c) {
  fiedler_profile &pr = p->prof;
  const fz::KernelSet &K = p->ks[c.type];
  pr.n_kernels = 4;
  for (int k = 0; k < 4; k++) pr.kernel_name[k] = K.names[k];
  float km = 0.f;
  cudaEventElapsedTime(&km, p->ev[8], p->ev[9]);
  pr.kernel_ms[3] += km;
  pr.kernel_launches_by[3]++;
  pr.kernel_launches++;
  pr.n_phases = fz::PH_COUNT;
  const State *hs = (const State *)(c.h_buf + c.h_states);
  for (size_t i = 0; i < c.items.size(); i++)
    for (int ph = 0; ph < fz::PH_COUNT; ph++) {
      pr.phase_ms[1][ph] += hs[i].phase_ns[1][ph] * 1e-6;
      pr.phase_bytes[1][ph] += hs[i].phase_bytes[1][ph];
      pr.kernel_bytes[3] += hs[i].phase_bytes[1][ph];
    }
  for (int ph = 0; ph < fz::PH_COUNT; ph++) pr.phase_name[ph] = kPhaseNames[ph];
}

// Runs c.items to completion on c.stream, growing arenas for graphs whose
// hierarchy outgrew the first estimate (their rerun uses the same engine).
fiedler_status batch_run_sync(fiedler_plan *p, BatchCtx &c) {
  double scale = 1.0;
  std::vector<BatchItem> all = c.items;
  std::vector<BatchItem> todo = c.items;
  const bool prof = p->profiling && &c == &p->bsync;
  if (prof) memset(&p->prof, 0, sizeof(p->prof));
  for (int attempt = 0; attempt < 4 && !todo.empty(); attempt++) {
    c.items = todo;
    fiedler_status st = batch_launch(p, c, scale);
    if (st != FIEDLER_OK) return st;
    CK(cudaEventSynchronize(c.done));
    batch_collect(c);
    if (prof) batch_profile(p, c);
    todo.clear();
    for (auto &it : c.items)
      if (needs_rerun(it.st)) todo.push_back(it);
    scale *= 2.0;
  }
  for (auto &it : todo) {
    if (it.res) it.res->status = FIEDLER_ENOMEM;
    if (it.ticket) it.ticket->st = FIEDLER_ENOMEM;
  }
  c.items = all;
  return FIEDLER_OK;
}

void free_ticket(Ticket *t) {
  cudaFree(t->rowptr);
  cudaFree(t->col);
  cudaFree(t->w);
  cudaFree(t->x);
  delete t;
}

// ---- serving form: continuous batching -----------------------------------
// The scheduler admits queued tickets into a batched launch while the device
// memory of in-flight tickets stays within the budget (a launch always takes
// at least one ticket when nothing else is in flight), keeps up to
// max_inflight launches running on their own streams, and completes tickets
// as their launch's event fires.
void complete_ctx(fiedler_plan *p, BatchCtx &c) {
  batch_collect(c);
  std::vector<BatchItem> rerun;
  for (auto &it : c.items)
    if (needs_rerun(it.st)) rerun.push_back(it);
  if (!rerun.empty()) {  // rare: regrow and run those again, synchronously
    std::vector<BatchItem> keep = c.items;
    c.items = rerun;
    double scale = 2.0;
    for (int attempt = 0; attempt < 3 && !c.items.empty(); attempt++, scale *= 2.0) {
      if (batch_launch(p, c, scale) != FIEDLER_OK || cudaEventSynchronize(c.done) != cudaSuccess) break;
      batch_collect(c);
      std::vector<BatchItem> again;
      for (auto &it : c.items)
        if (needs_rerun(it.st)) again.push_back(it);
      c.items = again;
    }
    for (auto &it : c.items) it.ticket->st = FIEDLER_ENOMEM;
    c.items = keep;
  }
  const auto now = std::chrono::steady_clock::now();
  std::lock_guard<std::mutex> lk(p->q_mu);
  for (auto &it : c.items) {
    Ticket *t = it.ticket;
    t->done = true;
    t->running = false;
    p->inflight_bytes -= t->footprint;
    p->n_completed++;
    p->latencies_ms.push_back(std::chrono::duration<float, std::milli>(now - t->t_submit).count());
  }
  c.items.clear();
  c.busy = false;
  p->q_cv.notify_all();
}

void worker_main(fiedler_plan *p) {
  cudaSetDevice(p->device);
  const int type = p->opt.precision == FIEDLER_FP64 ? 0 : 1;
  const int nctx = std::max(1, std::min(4, p->opt.max_inflight));
  const size_t budget = p->opt.hbm_budget_bytes ? p->opt.hbm_budget_bytes : (size_t)16 << 30;
  const int max_batch = std::max(1, p->opt.max_batch);
  for (;;) {
    bool progressed = false;
    // finished launches
    for (int k = 0; k < nctx; k++) {
      BatchCtx &c = p->bserve[k];
      if (c.busy && cudaEventQuery(c.done) == cudaSuccess) {
        complete_ctx(p, c);
        progressed = true;
      }
    }
    // admit a new launch
    BatchCtx *free_ctx = nullptr;
    for (int k = 0; k < nctx && !free_ctx; k++)
      if (!p->bserve[k].busy) free_ctx = &p->bserve[k];
    {
      std::unique_lock<std::mutex> lk(p->q_mu);
      if (p->stop) return;
      if (free_ctx && !p->queue.empty()) {
        BatchCtx &c = *free_ctx;
        c.items.clear();
        c.type = type;
        bool any_inflight = p->inflight_bytes > 0;
        while (!p->queue.empty() && (int)c.items.size() < max_batch) {
          auto itk = p->tickets.find(p->queue.front());
          if (itk == p->tickets.end()) {
            p->queue.pop_front();
            continue;
          }
          Ticket *t = itk->second;
          if (t->canceled) {
            p->queue.pop_front();
            t->st = FIEDLER_ECANCELED;
            t->done = true;
            p->q_cv.notify_all();
            continue;
          }
          const bool fits = p->inflight_bytes + t->footprint <= budget;
          if (!fits && (any_inflight || !c.items.empty())) break;  // wait for memory to free up
          p->queue.pop_front();
          t->running = true;
          p->inflight_bytes += t->footprint;
          p->peak_inflight = std::max(p->peak_inflight, p->inflight_bytes);
          BatchItem it{};
          it.n = t->n;
          it.nnz = t->nnz;
          it.rp = t->rowptr;
          it.ci = t->col;
          it.w = t->w;
          it.wf64 = t->w_dtype == FIEDLER_W_F64;
          it.host_in = false;
          it.user_x = t->x;
          it.user_x_dev = 1;
          it.ticket = t;
          c.items.push_back(it);
        }
        if (!c.items.empty()) {
          p->n_batches++;
          p->n_batched_tickets += c.items.size();
          c.busy = true;
          lk.unlock();
          if (batch_launch(p, c, 1.0) != FIEDLER_OK) {
            std::lock_guard<std::mutex> lk2(p->q_mu);
            for (auto &it : c.items) {
              it.ticket->st = FIEDLER_ECUDA;
              it.ticket->done = true;
              it.ticket->running = false;
              p->inflight_bytes -= it.ticket->footprint;
            }
            c.items.clear();
            c.busy = false;
            p->q_cv.notify_all();
          }
          progressed = true;
          continue;
        }
      }
      bool any_busy = false;
      for (int k = 0; k < nctx; k++) any_busy |= p->bserve[k].busy;
      if (!progressed) {
        if (any_busy) p->q_cv.wait_for(lk, std::chrono::microseconds(50));
        else p->q_cv.wait(lk, [&] { return p->stop || !p->queue.empty(); });
      }
    }
  }
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
  o->tail_max_nnz = 32768;
  o->barrier_timeout_ms = 5000;
  o->fault_inject = 0;
  o->hbm_budget_bytes = 0;
  o->max_batch = 1024;
  o->max_inflight = 2;
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
      !(o.resid_tol >= 0.0) || (o.tie_rule != 0 && o.tie_rule != 1) || o.tail_max_n < 1 || o.tail_max_nnz < 1 ||
      o.barrier_timeout_ms < 1 || o.max_batch < 1 || o.max_inflight < 1 || o.max_inflight > 4)
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
  for (int t = 0; t < 2; t++) {
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, p->ks[t].batch, fz::kCtaThreads, 0) != cudaSuccess ||
        bps < 1)
      return fail(FIEDLER_ECUDA);
    p->batch_slots[t] = bps * p->sms;
  }
  p->bsync.stream = p->stream;
  if (cudaEventCreateWithFlags(&p->bsync.done, cudaEventDisableTiming) != cudaSuccess) return fail(FIEDLER_ECUDA);
  for (int k = 0; k < 4; k++) {
    BatchCtx &c = p->bserve[k];
    if (cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess) return fail(FIEDLER_ECUDA);
    c.own_stream = true;
    if (cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming) != cudaSuccess) return fail(FIEDLER_ECUDA);
  }
  if (cudaMalloc(&p->d_state, sizeof(State)) != cudaSuccess) return fail(FIEDLER_ENOMEM);
  if (cudaMalloc(&p->d_ipart, sizeof(fz::IRed) * 2 * fz::kMaxBlocks) != cudaSuccess) return fail(FIEDLER_ENOMEM);
  if (cudaMalloc(&p->d_dpart, sizeof(double) * 2 * fz::kMaxBlocks * fz::kDSum) != cudaSuccess)
    return fail(FIEDLER_ENOMEM);
  if (cudaMallocHost(&p->h_state, sizeof(State)) != cudaSuccess) return fail(FIEDLER_ENOMEM);
  for (int i = 0; i < 10; i++)
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
    free_ticket(t);
    return map_cuda(e);
  }
  t->footprint = item_footprint(g->n, g->nnz, p->opt.precision == FIEDLER_FP64 ? 8 : 4, g->w_dtype == FIEDLER_W_F64);
  t->t_submit = std::chrono::steady_clock::now();
  std::lock_guard<std::mutex> lk(p->q_mu);
  t->id = p->next_ticket++;
  p->tickets[t->id] = t;
  p->queue.push_back(t->id);
  p->n_submitted++;
  *ticket = t->id;
  p->q_cv.notify_all();
  return FIEDLER_OK;
}

fiedler_status fiedler_solve_batch(fiedler_plan *p, const fiedler_graph *graphs, int count, fiedler_result *results) {
  if (!p || count < 0 || (count > 0 && (!graphs || !results))) return FIEDLER_EINVAL;
  std::lock_guard<std::mutex> ex(p->exec_mu);
  BatchCtx &c = p->bsync;
  c.items.clear();
  c.type = p->opt.precision == FIEDLER_FP64 ? 0 : 1;
  for (int i = 0; i < count; i++) {
    const fiedler_graph &g = graphs[i];
    fiedler_result &r = results[i];
    double *ux = r.x;
    const int uxd = r.x_on_device;
    fiedler_status st = check_graph(&g, &r);
    if (st != FIEDLER_OK) {
      r.status = st;
      continue;
    }
    BatchItem it{};
    it.n = g.n;
    it.nnz = g.nnz;
    it.rp = g.rowptr;
    it.ci = g.col;
    it.w = g.w;
    it.wf64 = g.w_dtype == FIEDLER_W_F64;
    it.host_in = !g.on_device;
    it.user_x = ux;
    it.user_x_dev = uxd;
    it.res = &r;
    c.items.push_back(it);
  }
  if (c.items.empty()) return FIEDLER_OK;
  return batch_run_sync(p, c);
}

fiedler_status fiedler_plan_serving_stats(const fiedler_plan *cp, fiedler_serving_stats *out) {
  if (!cp || !out) return FIEDLER_EINVAL;
  fiedler_plan *p = const_cast<fiedler_plan *>(cp);
  std::lock_guard<std::mutex> lk(p->q_mu);
  memset(out, 0, sizeof(*out));
  out->submitted = p->n_submitted;
  out->completed = p->n_completed;
  out->batches = p->n_batches;
  out->mean_batch = p->n_batches ? (double)p->n_batched_tickets / (double)p->n_batches : 0.0;
  out->peak_inflight_bytes = p->peak_inflight;
  if (!p->latencies_ms.empty()) {
    std::vector<float> v = p->latencies_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) { return (double)v[std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double sum = 0.0;
    for (float x : v) sum += x;
    out->mean_ms = sum / (double)v.size();
  }
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
  free_ticket(t);
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
  for (int k = 0; k < 4; k++)
    if (p->bserve[k].stream) cudaStreamSynchronize(p->bserve[k].stream);
  for (auto &kv : p->tickets) free_ticket(kv.second);
  p->tickets.clear();
  BatchCtx *ctxs[5] = {&p->bsync, &p->bserve[0], &p->bserve[1], &p->bserve[2], &p->bserve[3]};
  for (BatchCtx *c : ctxs) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->d_buf) cudaFree(c->d_buf);
    if (c->h_buf) cudaFreeHost(c->h_buf);
    if (c->done) cudaEventDestroy(c->done);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  }
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
  for (int i = 0; i < 10; i++)
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
