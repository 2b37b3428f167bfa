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
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
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
#include "host_opts.h"
#include "kernels.h"
#include "partition.h"

using fz::State;

namespace {

struct Ticket {
  uint64_t id;
  int64_t n, nnz;
  char *buf = nullptr;  // one pool allocation: rowptr | col | w | x
  size_t bytes = 0;     // its size (charged to the queue budget until polled)
  int32_t *rowptr = nullptr, *col = nullptr;
  void *w = nullptr;
  int w_dtype = 0;
  double *x = nullptr;  // device result vector
  size_t footprint = 0;  // device bytes while in flight (admission)
  double scale = 1.0;     // arena / scratch estimate factor (doubled on a rerun)
  double learn = 1.0;     // the plan's learned arena factor when it was admitted
  size_t arena_b = 0, scratch_b = 0;  // its allocation at admission
  char *dwork = nullptr;  // in flight: state | arena | scratch (pool allocation)
  unsigned long long k = 0;  // position in the serving ring
  std::chrono::steady_clock::time_point t_submit;
  fiedler_result res{};
  fiedler_status st = FIEDLER_EAGAIN;
  bool done = false, canceled = false, running = false;
  bool lane = false;      // solved by the large-graph lane, not the serving ring
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
  int reserve_sms = 0;  // SMs whose block slots the launch leaves free (the large-graph lane)
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
  int batch_slots[2][3];    // resident blocks of each batched kernel variant
  int serve_slots[2][3];    // and of each serving kernel variant
  int batch_var = 0;        // variant used by batched and served launches (kBatchThreads)
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
  // ticket inputs and outputs: a stream-ordered pool on a stream of their own,
  // so that submit and poll never wait for the device as a whole
  cudaStream_t io_stream = nullptr;
  cudaStream_t sub_stream = nullptr;  // fiedler_batch_submit's copies (waits only for its own)
  cudaMemPool_t pool = nullptr;
  // serving form: a persistent kernel fed through a ring in device memory
  fz::ServeRing *d_ring = nullptr;
  fz::ServeDone *done = nullptr;      // host view of the completion flags (pinned, mapped)
  fz::ServeDone *done_dev = nullptr;  // device view of the same memory
  unsigned long long *h_pub = nullptr;  // pinned staging: item pointers of a round, then the tail
  unsigned long long published = 0;
  static constexpr unsigned long long kIdleNs = 20000000ull;  // a serving block idle this long leaves
  static constexpr int kReserveSms = 2;  // SMs whose block slots serving launches leave free
  static constexpr int kLaneFreeSms = 16;  // SMs a lane (lane_sms) leaves to the one-block kernels at least
  struct ServeLaunch {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    bool running = false;
    unsigned long long base = 0;  // number of its first block
    int nb = 0;
  };
  std::vector<ServeLaunch> serve;    // launch records (own streams), reused once finished
  unsigned long long block_next = 0;
  State *h_stage = nullptr;           // pinned staging of ticket states (max_batch of them)
  int stage_n = 0;
  std::deque<Ticket *> live;          // published, not yet finished (ring order)
  // large-graph lane: admitted large tickets of the serving form wait in q and
  // run through the cooperative grid-wide kernels, lane_slots of them at once,
  // each slot on its own stream with its own reduction partials on
  // slot_blocks blocks (lane_sms / lane_slots SMs); the batched form spreads
  // its large graphs over the same slots
  struct LaneSlot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    fz::IRed *ipart = nullptr;
    double *dpart = nullptr;
    void **h_part = nullptr;  // pinned {ipart, dpart}: copied into a ticket's state before its launch
    Ticket *cur = nullptr;
  };
  struct Lane {
    cudaStream_t stream = nullptr;  // slot 0's stream (null: no lane)
    fz::IRed *ipart = nullptr;      // slot 0's partials
    double *dpart = nullptr;
    int slot_blocks[2] = {0, 0};  // [type] blocks of one lane launch
    std::vector<LaneSlot> slots;
    std::deque<Ticket *> q;
    uint64_t solves = 0;
    bool busy() const {
      for (const LaneSlot &s : slots)
        if (s.cur) return true;
      return false;
    }
  } lane;
  uint64_t n_launches = 0;
  // serving form
  std::mutex exec_mu;       // one solve on the device state at a time
  std::mutex q_mu;
  std::condition_variable q_cv;
  std::deque<uint64_t> queue;
  std::deque<uint64_t> finished;  // tickets done since they were last listed by fiedler_poll_any
  std::unordered_map<uint64_t, Ticket *> tickets;
  uint64_t next_ticket = 1;
  std::thread worker;
  bool stop = false;
  size_t inflight_bytes = 0, peak_inflight = 0;
  size_t queued_bytes = 0;  // pool bytes of submitted, not yet polled tickets
  uint64_t n_submitted = 0, n_completed = 0, n_batches = 0, n_batched_tickets = 0;
  std::vector<float> latencies_ms;
  double block_seconds = 0.0, live_sum = 0.0, alive_sum = 0.0;
  // serving admission learns how much of the arena estimate tickets use: the
  // largest (arena used / estimate) seen, times 1.25, bounds later estimates
  double arena_ratio = 0.0;
  double arena_factor() const {
    return arena_ratio <= 0.0 ? 1.0 : std::min(1.0, std::max(0.25, 1.25 * arena_ratio));
  }
  uint64_t live_rounds = 0;
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

size_t arena_estimate(int64_t n, int64_t nnz, size_t tsz, bool wf64, const fiedler_options &o) {
  // fine level: optional self-loop-free copy, degree, matching, aggregates,
  // colours, permutations, colour-order copy, iterates
  double l0 = 4.0 * (n + 1) + (4.0 + (wf64 ? 8.0 : 4.0)) * nnz + 8.0 * n + 4.0 * n * 3 + 8.0 * n +
              4.0 * (fz::kMaxColors + 1) + 4.0 * (n + 1) + (4.0 + tsz) * nnz + (2.0 * tsz + 4.0) * n;
  // coarse levels together: assume at most 2n vertices and 2nnz entries
  double lc = 2.0 * (4.0 * n + 16.0 * nnz + 8.0 * n + 4.0 * n * 3 + 8.0 * n + 4.0 * n + (4.0 + tsz) * nnz +
                     (2.0 * tsz + 4.0) * n) +
              fz::kMaxLevels * 4.0 * (fz::kMaxColors + 1);
  double slack = fz::kMaxLevels * 24.0 * 256.0 + (1 << 20);
  return (size_t)(l0 + lc + slack) + fz::refine_bytes(n, tsz, o.refine, o.lanczos_basis, o.refine_precond);
}

size_t scratch_estimate(int64_t n, int64_t nnz, int nblocks, const fiedler_options &o) {
  // one level's scratch, all live at once: colouring (cround + 3 worklists +
  // heavy list + resume positions), matching (two 8-byte pick buffers + 3
  // worklists + heavy list), Galerkin (9 per-vertex / per-aggregate arrays,
  // (J, slot) keys + FP64 weights per cross entry), colour histogram
  double b = 24.0 * n + 32.0 * n + 4.0 * (n + 1) * 9 + 16.0 * nnz + 4.0 * fz::kMaxColors * nblocks +
             64.0 * 256.0 + (1 << 20);
  // Alg. 1's random-order greedy (hec_mode PAPER) keeps more per-vertex state
  // than the matching: heaviest neighbour, turn state, first claimant (key and
  // vertex), labels, founder ids and the founders' buckets
  if (o.hec_mode == FIEDLER_HEC_PAPER) b += 44.0 * n + 8.0 * 256.0;
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

}  // namespace

namespace fz {

bool options_valid(const fiedler_options &o) {
  return !((o.precision != FIEDLER_FP64 && o.precision != FIEDLER_FP32_FP64RED) || o.coarse_max_n < 1 ||
           o.max_levels < 1 || o.max_levels > fz::kMaxLevels || !(o.stall_ratio > 0.0 && o.stall_ratio <= 1.0) ||
           o.gs_sweeps < 0 || o.pi_max_iters < 0 || o.pi_max_iters_coarsest < 0 || !(o.pi_cos_tol >= 0.0) ||
           !(o.resid_tol >= 0.0) || (o.tie_rule != 0 && o.tie_rule != 1) || o.tail_max_n < 1 ||
           o.tail_max_nnz < 1 || o.barrier_timeout_ms < 1 || o.max_batch < 1 ||
           (o.batch_threads != 0 && o.batch_threads != 512 && o.batch_threads != 256 && o.batch_threads != 128) ||
           (o.refine != FIEDLER_REFINE_NONE && o.refine != FIEDLER_REFINE_LOBPCG &&
            o.refine != FIEDLER_REFINE_LANCZOS) ||
           o.refine_max_iters < 0 || !(o.refine_tol > 0.0 && o.refine_tol < 1.0) || o.lanczos_basis < 4 ||
           o.lanczos_basis > fz::kMaxBasis || (o.hec_mode != FIEDLER_HEC_DOMINANT && o.hec_mode != FIEDLER_HEC_PAPER) ||
           (o.refine_precond != FIEDLER_PRECOND_DEGREE && o.refine_precond != FIEDLER_PRECOND_VCYCLE) ||
           o.lane_sms < 0 || o.lane_min_n < 2 || o.lane_slots < 1 || (o.lane_sms > 0 && o.lane_slots > o.lane_sms));
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
  o.refine = u.refine;
  o.refine_max_iters = u.refine_max_iters;
  o.lanczos_basis = u.lanczos_basis;
  o.hec_mode = u.hec_mode;
  o.refine_precond = u.refine_precond;
  o.refine_tol = u.refine_tol;
}

}  // namespace fz

namespace {

using fz::fill_opts;

const char *kPhaseNames[fz::PH_COUNT] = {"ingest", "colour", "reorder", "match", "aggregate", "galerkin",
                                         "coarsest", "prolong", "gauss_seidel", "power_iter", "final", "refine"};

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
  size_t abytes = arena_estimate(n, nnz, tsz, w_f64 != 0, p->opt);
  size_t sbytes = scratch_estimate(n, nnz, gmax, p->opt);
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
      res->refine_iters = h->refine_total;
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
  // grow by half again at least, so that a stream of growing batches
  // reallocates (and frees pinned host memory) rarely
  if (c.d_cap < dbytes) dbytes = std::max(dbytes, c.d_cap + c.d_cap / 2);
  if (c.h_cap < hbytes) hbytes = std::max(hbytes, c.h_cap + c.h_cap / 2);
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
size_t item_footprint(int64_t n, int64_t nnz, size_t tsz, bool wf64, const fiedler_options &o) {
  return r256(sizeof(State)) + r256(arena_estimate(n, nnz, tsz, wf64, o)) + r256(scratch_estimate(n, nnz, 1, o));
}

// Lays out and queues one batched launch of c.items on c.stream (asynchronous).
// The items are ordered by decreasing size so the largest graphs start first.
fiedler_status batch_launch(fiedler_plan *p, BatchCtx &c, double arena_scale) {
  const int type = c.type;
  const size_t tsz = type == 0 ? 8 : 4;
  std::stable_sort(c.items.begin(), c.items.end(),
                   [](const BatchItem &a, const BatchItem &b) { return a.nnz + a.n > b.nnz + b.n; });
  const int count = (int)c.items.size();
  const int var = p->batch_var;
  const int per_sm = std::max(1, p->batch_slots[type][var] / p->sms);
  const int nslots = std::min(count, std::max(per_sm, p->batch_slots[type][var] - per_sm * c.reserve_sms));
  size_t slot = 0, arenas = 0, in_b = 0, x_b = 0;
  for (auto &it : c.items) {
    it.arena_b = r256((size_t)(arena_estimate(it.n, it.nnz, tsz, it.wf64, p->opt) * arena_scale));
    it.scratch_b = r256((size_t)(scratch_estimate(it.n, it.nnz, 1, p->opt) * arena_scale));
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
  CK(cudaLaunchKernel(p->ks[type].batch_v[var], dim3(nslots), dim3(fz::kBatchThreads[var]), args, 0, c.stream));
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
    double ns = 0.0;  // the graph's own device time (its block, device timer)
    for (int ph = 0; ph < fz::PH_COUNT; ph++) ns += h->phase_ns[1][ph];
    r.ms = (float)(ns * 1e-6);
    if (out == FIEDLER_OK || out == FIEDLER_ENOTCONVERGED) {
      r.lambda2 = h->lambda;
      r.residual = h->residual;
      r.ortho = h->ortho;
      r.pi_iters_total = h->pi_total;
      r.gs_sweeps_total = h->gs_total;
      r.refine_iters = h->refine_total;
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
  for (int k = 0; k < 3; k++) pr.kernel_name[k] = K.names[k];
  pr.kernel_name[3] = K.batch_names[p->batch_var];
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

// caller holds q_mu (or is the only thread left)
void free_ticket(fiedler_plan *p, Ticket *t) {
  if (t->buf) cudaFreeAsync(t->buf, p->io_stream);  // the ticket's launch has finished
  p->queued_bytes -= t->bytes;
  delete t;
}

// ---- serving form: continuous batching -----------------------------------
// A scheduler thread admits queued tickets while the device memory of the
// tickets in flight stays within the budget (a ticket is always admitted when
// nothing else is in flight): each admitted ticket gets one pool allocation
// holding its solve state, hierarchy arena and scratch, its state header is
// copied in, and it is published in the serving ring.  The serving kernel's
// resident blocks (one graph each, as in the batched form) claim published
// tickets in order and flag each as soon as it is done; the scheduler reads
// the flags, copies the finished state back and completes the ticket, which
// returns its memory to the budget at once.  A long solve therefore holds one
// block, not a launch.  The kernel's blocks leave after an idle spell; when
// unfinished tickets outnumber the blocks still alive, the scheduler launches
// the missing ones (never into the last kReserveSms SMs' block slots).

// fills the device-side state header of a ticket (host copy in *h)
void fill_ticket_state(fiedler_plan *p, Ticket *t, State *h, int type, size_t arena_b, size_t scratch_b) {
  memset(h, 0, sizeof(State));
  fill_opts(h->opt, p->opt, type);
  h->opt.tail_max_n = INT_MAX;  // every level in the one-block engine
  h->opt.tail_max_nnz = INT_MAX;
  h->opt.fault_inject = 0;
  h->bad_index = LLONG_MAX;
  h->n0 = (int)t->n;
  h->nnz0 = (int)t->nnz;
  h->in_rowptr = t->rowptr;
  h->in_col = t->col;
  h->in_w = t->w;
  h->in_w_f64 = t->w_dtype == FIEDLER_W_F64;
  h->arena = t->dwork + r256(sizeof(State));
  h->arena_size = arena_b;
  h->scratch = h->arena + arena_b;
  h->scratch_size = scratch_b;
  h->xout = t->x;
}

void ticket_result(const State *h, Ticket *t) {
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
    r.refine_iters = h->refine_total;
  }
  r.x = t->x;
  r.x_on_device = 1;
  r.status = out;
  t->res = r;
  t->st = out;
}

// Marks a ticket finished (q_mu held) and lists it for fiedler_poll_any.  Ids
// of tickets already collected by fiedler_poll are dropped from the list when
// it outgrows the live tickets, so a caller that never lists stays bounded.
void mark_done(fiedler_plan *p, Ticket *t) {
  t->done = true;
  p->finished.push_back(t->id);
  if (p->finished.size() > 2 * p->tickets.size() + 1024) {
    std::deque<uint64_t> keep;
    for (uint64_t id : p->finished)
      if (p->tickets.count(id)) keep.push_back(id);
    p->finished.swap(keep);
  }
}

void worker_main(fiedler_plan *p) {
  cudaSetDevice(p->device);
  const int type = p->opt.precision == FIEDLER_FP64 ? 0 : 1;
  const size_t tsz = type == 0 ? 8 : 4;
  const size_t budget = p->opt.hbm_budget_bytes ? p->opt.hbm_budget_bytes : (size_t)16 << 30;
  const int max_batch = std::max(1, std::min(p->opt.max_batch, p->stage_n));
  volatile fz::ServeDone *vd = p->done;
  std::vector<Ticket *> adm;
  for (;;) {
    bool progressed = false;
    // 1. finished tickets (any order): copy their states back, complete them
    std::vector<Ticket *> fin;
    for (auto it = p->live.begin(); it != p->live.end();) {
      Ticket *t = *it;
      if (vd->done[t->k % fz::kRing] == t->k + 1ull) {
        fin.push_back(t);
        it = p->live.erase(it);
      } else {
        ++it;
      }
    }
    if (!fin.empty()) {
      progressed = true;
      const size_t nf = std::min(fin.size(), (size_t)p->stage_n);
      for (size_t i = 0; i < fin.size(); i += nf) {
        const size_t m = std::min(nf, fin.size() - i);
        bool ok = true;
        for (size_t j = 0; j < m; j++)
          ok = ok && cudaMemcpyAsync(p->h_stage + j, fin[i + j]->dwork, sizeof(State), cudaMemcpyDeviceToHost,
                                     p->io_stream) == cudaSuccess;
        ok = ok && cudaStreamSynchronize(p->io_stream) == cudaSuccess;
        const auto now = std::chrono::steady_clock::now();
        std::lock_guard<std::mutex> lk(p->q_mu);
        for (size_t j = 0; j < m; j++) {
          Ticket *t = fin[i + j];
          const State *h = p->h_stage + j;
          cudaFreeAsync(t->dwork, p->io_stream);
          t->dwork = nullptr;
          p->inflight_bytes -= t->footprint;
          if (ok && h->status == fz::ST_ARENA) p->arena_ratio = std::max(p->arena_ratio, 2.0 * t->learn);
          if (ok && (h->status == fz::ST_ARENA || h->status == fz::ST_SCRATCH) && t->scale < 8.0) {
            t->scale *= 2.0;  // the hierarchy outgrew its estimate: run it again with more room
            t->running = false;
            p->queue.push_front(t->id);
            continue;
          }
          if (ok && h->status == fz::ST_OK)
            p->arena_ratio = std::max(p->arena_ratio, (double)h->arena_off / (double)arena_estimate(
                                                          t->n, t->nnz, tsz, t->w_dtype == FIEDLER_W_F64, p->opt));
          if (ok) ticket_result(h, t);
          else t->st = FIEDLER_ECUDA;
          if (ok)
            for (int ph = 0; ph < fz::PH_COUNT; ph++) p->block_seconds += h->phase_ns[1][ph] * 1e-9;
          if (ok && (h->status == fz::ST_ARENA || h->status == fz::ST_SCRATCH)) t->st = FIEDLER_ENOMEM;
          mark_done(p, t);
          t->running = false;
          p->n_completed++;
          p->latencies_ms.push_back(std::chrono::duration<float, std::milli>(now - t->t_submit).count());
        }
        p->q_cv.notify_all();
      }
    }
    // 1b. the large-graph lane: each slot's finished ticket, then its next one
    for (fiedler_plan::LaneSlot &sl : p->lane.slots) {
      if (sl.cur && cudaEventQuery(sl.ev) == cudaSuccess) {
        progressed = true;
        Ticket *t = sl.cur;
        sl.cur = nullptr;
        State *hs = p->h_stage;  // read back and synchronised before the next slot's
        const bool ok = cudaMemcpyAsync(hs, t->dwork, sizeof(State), cudaMemcpyDeviceToHost, sl.stream) ==
                            cudaSuccess &&
                        cudaStreamSynchronize(sl.stream) == cudaSuccess;
        const State *h = hs;
        const auto now = std::chrono::steady_clock::now();
        std::lock_guard<std::mutex> lk(p->q_mu);
        cudaFreeAsync(t->dwork, sl.stream);
        t->dwork = nullptr;
        p->inflight_bytes -= t->footprint;
        if (ok && (h->status == fz::ST_ARENA || h->status == fz::ST_SCRATCH) && t->scale < 8.0) {
          t->scale *= 2.0;  // the hierarchy outgrew its estimate: run it again with more room
          t->running = false;
          p->queue.push_front(t->id);
        } else {
          if (ok) ticket_result(h, t);
          else t->st = FIEDLER_ECUDA;
          if (ok && (h->status == fz::ST_ARENA || h->status == fz::ST_SCRATCH)) t->st = FIEDLER_ENOMEM;
          mark_done(p, t);
          t->running = false;
          p->n_completed++;
          p->lane.solves++;
          p->latencies_ms.push_back(std::chrono::duration<float, std::milli>(now - t->t_submit).count());
        }
        p->q_cv.notify_all();
      }
      if (!sl.cur && !p->lane.q.empty()) {
        progressed = true;
        Ticket *t = p->lane.q.front();
        p->lane.q.pop_front();
        const fz::KernelSet &K = p->ks[type];
        const int nbl = p->lane.slot_blocks[type];
        void *args[] = {(void *)&t->dwork};
        // the slot's reduction partials into the ticket's state, in stream order
        // before its kernels (ipart and dpart are adjacent in State)
        const bool ok =
            cudaMemcpyAsync((char *)t->dwork + offsetof(State, ipart), sl.h_part, 2 * sizeof(void *),
                            cudaMemcpyHostToDevice, sl.stream) == cudaSuccess &&
            cudaLaunchCooperativeKernel(K.grid_setup, dim3(nbl), dim3(fz::kGridThreads), args, 0, sl.stream) ==
                cudaSuccess &&
            cudaLaunchKernel(K.cta, dim3(1), dim3(fz::kCtaThreads), args, 0, sl.stream) == cudaSuccess &&
            cudaLaunchCooperativeKernel(K.grid_solve, dim3(nbl), dim3(fz::kGridThreads), args, 0, sl.stream) ==
                cudaSuccess &&
            cudaEventRecord(sl.ev, sl.stream) == cudaSuccess;
        if (ok) {
          sl.cur = t;
          p->n_launches += 3;
        } else {
          std::lock_guard<std::mutex> lk(p->q_mu);
          cudaFreeAsync(t->dwork, sl.stream);
          t->dwork = nullptr;
          p->inflight_bytes -= t->footprint;
          t->st = FIEDLER_ECUDA;
          mark_done(p, t);
          t->running = false;
          p->q_cv.notify_all();
        }
      }
    }
    // 2. admissions
    adm.clear();
    {
      std::unique_lock<std::mutex> lk(p->q_mu);
      if (p->stop) break;
      while (!p->queue.empty() && (int)adm.size() < max_batch && p->live.size() + adm.size() < fz::kRing - 1) {
        auto itk = p->tickets.find(p->queue.front());
        if (itk == p->tickets.end()) {
          p->queue.pop_front();
          continue;
        }
        Ticket *t = itk->second;
        if (t->canceled) {
          p->queue.pop_front();
          t->st = FIEDLER_ECANCELED;
          mark_done(p, t);
          p->q_cv.notify_all();
          continue;
        }
        // footprint with the learned arena factor (a rerun doubles t->scale)
        t->lane = p->lane.stream && t->n >= p->opt.lane_min_n;
        t->learn = p->arena_factor();
        t->arena_b = r256((size_t)(arena_estimate(t->n, t->nnz, tsz, t->w_dtype == FIEDLER_W_F64, p->opt) * t->scale * t->learn));
        t->scratch_b = r256((size_t)(scratch_estimate(t->n, t->nnz, t->lane ? p->lane.slot_blocks[type] : 1, p->opt) *
                                     t->scale));
        t->footprint = r256(sizeof(State)) + t->arena_b + t->scratch_b;
        const bool empty = p->inflight_bytes == 0 && adm.empty();
        if (!empty && p->inflight_bytes + t->footprint > budget) break;  // wait for memory to free up
        p->queue.pop_front();
        t->running = true;
        p->inflight_bytes += t->footprint;
        p->peak_inflight = std::max(p->peak_inflight, p->inflight_bytes);
        adm.push_back(t);
      }
    }
    if (!adm.empty()) {
      progressed = true;
      int staged = 0;
      std::vector<Ticket *> ok_t;
      for (Ticket *t : adm) {
        const size_t ab = t->arena_b, sb = t->scratch_b;
        const size_t bytes = r256(sizeof(State)) + ab + sb;
        if (cudaMallocFromPoolAsync((void **)&t->dwork, bytes, p->pool, p->io_stream) != cudaSuccess) {
          t->dwork = nullptr;
          std::lock_guard<std::mutex> lk(p->q_mu);
          p->inflight_bytes -= t->footprint;
          t->st = FIEDLER_ENOMEM;
          mark_done(p, t);
          t->running = false;
          p->q_cv.notify_all();
          continue;
        }
        State *h = p->h_stage + staged++;
        fill_ticket_state(p, t, h, type, ab, sb);
        if (t->lane) {  // the grid-wide engine on the large levels; the partials
                        // are those of the slot that launches it (written then)
          h->opt.tail_max_n = p->opt.tail_max_n;
          h->opt.tail_max_nnz = p->opt.tail_max_nnz;
          h->ipart = p->lane.ipart;
          h->dpart = p->lane.dpart;
        }
        cudaMemcpyAsync(t->dwork, h, sizeof(State), cudaMemcpyHostToDevice, p->io_stream);
        if (t->lane) p->lane.q.push_back(t);
        else ok_t.push_back(t);
      }
      // item pointers, then the new tail, in stream order after the states
      const unsigned long long first = p->published;
      const size_t m = ok_t.size();
      for (size_t j = 0; j < m; j++) {
        Ticket *t = ok_t[j];
        t->k = first + j;
        p->h_pub[j] = (unsigned long long)(uintptr_t)t->dwork;
        p->live.push_back(t);
      }
      p->published = first + m;
      p->h_pub[m] = p->published;
      if (m > 0) {
        const size_t pos = first % fz::kRing, part = std::min(m, (size_t)fz::kRing - pos);
        cudaMemcpyAsync(p->d_ring->item + pos, p->h_pub, 8 * part, cudaMemcpyHostToDevice, p->io_stream);
        if (part < m)
          cudaMemcpyAsync(p->d_ring->item, p->h_pub + part, 8 * (m - part), cudaMemcpyHostToDevice, p->io_stream);
        cudaMemcpyAsync(&p->d_ring->tail, p->h_pub + m, 8, cudaMemcpyHostToDevice, p->io_stream);
      }
      cudaStreamSynchronize(p->io_stream);
      std::lock_guard<std::mutex> lk(p->q_mu);
      p->n_batches++;
      p->n_batched_tickets += ok_t.size();

    }
    // 3. blocks for the published work: every unfinished ticket needs one;
    // blocks that find nothing to do leave after a short wait, so the alive
    // count is read from their exit flags and topped up with a new launch of
    // the blocks still missing.  Launching only those, and never into the
    // block slots of the last kReserveSms SMs, leaves room for other work on
    // the device: a device-to-device copy (fiedler_batch_submit's) or another
    // kernel would otherwise wait for resident serving blocks to leave.
    if (!p->live.empty()) {
      int alive = 0, freei = -1;
      unsigned long long oldest = p->block_next;
      for (int i = 0; i < (int)p->serve.size(); i++) {
        fiedler_plan::ServeLaunch &L = p->serve[i];
        if (L.running && cudaEventQuery(L.ev) == cudaSuccess) L.running = false;
        if (!L.running) {
          if (freei < 0) freei = i;
          continue;
        }
        int gone = 0;
        for (int b = 0; b < L.nb; b++) {
          const unsigned long long g = L.base + (unsigned long long)b;
          gone += vd->exited[g % fz::kExitRing] == g + 1ull;
        }
        alive += L.nb - gone;
        oldest = std::min(oldest, L.base);
      }
      int unfinished = 0;
      for (Ticket *t : p->live) unfinished += vd->done[t->k % fz::kRing] != t->k + 1ull;
      const int var = p->batch_var;
      const int slots = p->serve_slots[type][var], per_sm = slots / p->sms;
      const int room =
          std::max(per_sm, slots - per_sm * (fiedler_plan::kReserveSms + (p->lane.stream ? p->opt.lane_sms : 0))) -
          alive;
      p->live_sum += (double)unfinished;
      p->alive_sum += (double)alive;
      p->live_rounds++;
      const int want = std::min(unfinished - alive, room);
      // block numbers stay within the exit-flag ring of every running launch
      const bool fits = p->block_next + fz::kServeSlots - oldest < (unsigned long long)fz::kExitRing;
      if (want > 0 && fits && (freei >= 0 || p->serve.size() < 4096)) {
        if (freei < 0) {
          fiedler_plan::ServeLaunch L;
          if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming) == cudaSuccess) {
            p->serve.push_back(L);
            freei = (int)p->serve.size() - 1;
          } else {
            if (L.stream) cudaStreamDestroy(L.stream);
          }
        }
        if (freei >= 0) {
          fiedler_plan::ServeLaunch &L = p->serve[freei];
          const int nb = std::min(want, fz::kServeSlots);
          unsigned long long base = p->block_next;
          void *args[] = {(void *)&p->d_ring, (void *)&p->done_dev, (void *)&base};
          if (cudaLaunchKernel(p->ks[type].serve_v[var], dim3(nb), dim3(fz::kBatchThreads[var]), args, 0, L.stream) ==
                  cudaSuccess &&
              cudaEventRecord(L.ev, L.stream) == cudaSuccess) {
            L.running = true;
            L.base = base;
            L.nb = nb;
            p->block_next += (unsigned long long)nb;
            p->n_launches++;
          }
        }
      }
    }
    if (!progressed) {
      std::unique_lock<std::mutex> lk(p->q_mu);
      if (p->stop) break;
      if (p->live.empty() && p->queue.empty() && !p->lane.busy() && p->lane.q.empty())
        p->q_cv.wait(lk, [&] { return p->stop || !p->queue.empty(); });
      else p->q_cv.wait_for(lk, std::chrono::microseconds(50));
    }
  }
  // leaving: let the kernel's blocks go, wait for them, release what is in flight
  {
    const unsigned long long one = 1;
    cudaMemcpyAsync(&p->d_ring->stop, &one, 8, cudaMemcpyHostToDevice, p->io_stream);
    cudaStreamSynchronize(p->io_stream);
  }
  for (auto &L : p->serve) {
    if (L.running) cudaEventSynchronize(L.ev);
    L.running = false;
  }
  for (fiedler_plan::LaneSlot &sl : p->lane.slots)
    if (sl.cur) {
      cudaEventSynchronize(sl.ev);
      p->live.push_back(sl.cur);  // released below
      sl.cur = nullptr;
    }
  for (Ticket *t : p->lane.q) p->live.push_back(t);
  p->lane.q.clear();
  for (Ticket *t : p->live) {
    if (t->dwork) cudaFreeAsync(t->dwork, p->io_stream);
    t->dwork = nullptr;
  }
  p->live.clear();
}

}  // namespace

namespace {

// Recursive spectral bisection on the plan (the plan's exec lock held): the
// largest part with at least two vertices (lowest id on ties) is split by the
// sign of the Fiedler vector of its induced subgraph, or along its connected
// components when that subgraph is disconnected, until `parts` parts exist.
fiedler_status partition_locked(fiedler_plan *p, const fiedler_graph *g, int parts, int32_t *labels, int lab_dev,
                                fiedler_partition_info *info) {
  const int64_t n = g->n, nnz = g->nnz;
  const size_t wsz = g->w_dtype == FIEDLER_W_F64 ? 8 : 4;
  cudaStream_t st = p->stream;
  // device copies of the input (if on the host), the labels, the subgraph
  // buffers and the scratch: one allocation
  const size_t in_b = g->on_device ? 0 : r256(4 * (size_t)(n + 1)) + r256(4 * (size_t)std::max<int64_t>(nnz, 1)) +
                                          r256(wsz * (size_t)std::max<int64_t>(nnz, 1));
  const size_t sub_b = r256(4 * (size_t)(n + 1)) + r256(4 * (size_t)std::max<int64_t>(nnz, 1)) +
                       r256(wsz * (size_t)std::max<int64_t>(nnz, 1)) + r256(4 * (size_t)n) + r256(8 * (size_t)n) +
                       r256(4 * (size_t)n) + r256(4 * fz::part_scratch_ints(n)) + r256(4 * (size_t)n);
  char *buf = nullptr;
  CK(cudaMallocAsync((void **)&buf, in_b + sub_b, st));
  int *h = nullptr;
  cudaError_t he = cudaMallocHost((void **)&h, 4 * sizeof(int));
  if (he != cudaSuccess) {
    cudaFreeAsync(buf, st);
    return map_cuda(he);
  }
  auto cleanup = [&](fiedler_status rs) {
    cudaFreeAsync(buf, st);
    cudaStreamSynchronize(st);
    cudaFreeHost(h);
    return rs;
  };
  char *q = buf;
  auto take = [&](size_t b) {
    char *r = q;
    q += r256(b);
    return r;
  };
  const int32_t *rp = g->rowptr, *ci = g->col;
  const void *w = g->w;
  if (!g->on_device) {
    int32_t *drp = (int32_t *)take(4 * (size_t)(n + 1));
    int32_t *dci = (int32_t *)take(4 * (size_t)std::max<int64_t>(nnz, 1));
    void *dw = take(wsz * (size_t)std::max<int64_t>(nnz, 1));
    if (cudaMemcpyAsync(drp, rp, 4 * (size_t)(n + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        (nnz > 0 && (cudaMemcpyAsync(dci, ci, 4 * (size_t)nnz, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                     cudaMemcpyAsync(dw, w, wsz * (size_t)nnz, cudaMemcpyHostToDevice, st) != cudaSuccess)))
      return cleanup(FIEDLER_ECUDA);
    rp = drp;
    ci = dci;
    w = dw;
  }
  int32_t *srp = (int32_t *)take(4 * (size_t)(n + 1));
  int32_t *sci = (int32_t *)take(4 * (size_t)std::max<int64_t>(nnz, 1));
  void *sw = take(wsz * (size_t)std::max<int64_t>(nnz, 1));
  int32_t *map = (int32_t *)take(4 * (size_t)n);
  double *x = (double *)take(8 * (size_t)n);
  int32_t *comp = (int32_t *)take(4 * (size_t)n);
  int *sc = (int *)take(4 * fz::part_scratch_ints(n));
  int32_t *lab = (int32_t *)take(4 * (size_t)n);
  fz::PartScratch ps;
  ps.keep = sc;
  ps.cnt = sc + (n + 1);
  ps.bsum = sc + 2 * (n + 1);
  ps.flag = sc + fz::part_scratch_ints(n) - 2;
  if (cudaMemsetAsync(lab, 0, 4 * (size_t)n, st) != cudaSuccess) return cleanup(FIEDLER_ECUDA);
  std::vector<int64_t> size(1, n);
  std::vector<char> stuck(1, 0);
  int solves = 0, comp_splits = 0;
  const auto t0 = std::chrono::steady_clock::now();
  fiedler_status out = FIEDLER_OK;
  while ((int)size.size() < parts) {
    int pick = -1;
    for (int k = 0; k < (int)size.size(); k++)
      if (!stuck[k] && size[k] >= 2 && (pick < 0 || size[k] > size[pick])) pick = k;
    if (pick < 0) break;  // every part is a single vertex or cannot be split
    const int newp = (int)size.size();
    if (fz::part_extract(rp, ci, w, wsz == 8, n, lab, pick, srp, sci, sw, map, ps, h, st) != cudaSuccess)
      return cleanup(FIEDLER_ECUDA);
    const int64_t m = h[0], mnz = h[1];
    fiedler_result res{};
    fiedler_status sst = run_solve(p, m, mnz, srp, sci, sw, wsz == 8, x, &res);
    solves++;
    cudaError_t ce;
    if (sst == FIEDLER_OK || sst == FIEDLER_ENOTCONVERGED) {
      ce = fz::part_split_sign(x, m, map, lab, newp, ps, &h[2], st);
    } else if (sst == FIEDLER_EDISCONNECTED) {
      ce = fz::part_split_components(srp, sci, m, map, lab, newp, comp, ps, &h[2], st);
      comp_splits++;
    } else {
      out = sst;
      break;
    }
    if (ce != cudaSuccess) return cleanup(FIEDLER_ECUDA);
    const int64_t moved = h[2];
    if (moved <= 0 || moved >= size[pick]) {  // nothing to split off (cannot happen for x orthogonal to 1)
      stuck[pick] = 1;
      continue;
    }
    size[pick] -= moved;
    size.push_back(moved);
    stuck.push_back(0);
  }
  if (out == FIEDLER_OK) {
    if (cudaMemcpyAsync(labels, lab, 4 * (size_t)n, lab_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        st) != cudaSuccess)
      return cleanup(FIEDLER_ECUDA);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return cleanup(FIEDLER_ECUDA);
  if (info) {
    info->parts = (int)size.size();
    info->solves = solves;
    info->component_splits = comp_splits;
    info->ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return cleanup(out);
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
  o->queue_budget_bytes = 0;
  o->batch_threads = 0;
  o->refine = FIEDLER_REFINE_NONE;
  o->refine_max_iters = 5000;
  o->refine_tol = 1e-4;
  o->lanczos_basis = 24;
  o->hec_mode = FIEDLER_HEC_DOMINANT;
  o->refine_precond = FIEDLER_PRECOND_VCYCLE;
  o->lane_sms = 0;
  o->lane_min_n = 200000;
  o->lane_slots = 1;
}

fiedler_status fiedler_plan_create(const fiedler_options *opts, void *cuda_stream, fiedler_plan **out) {
  if (!out) return FIEDLER_EINVAL;
  *out = nullptr;
  fiedler_options o;
  if (opts) o = *opts;
  else fiedler_options_default(&o);
  if (!fz::options_valid(o)) return FIEDLER_EINVAL;
  fiedler_plan *p = new (std::nothrow) fiedler_plan();
  if (!p) return FIEDLER_ENOMEM;
  p->opt = o;
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
  for (int t = 0; t < 2; t++)
    for (int v = 0; v < 3; v++) {
      int bps = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, p->ks[t].batch_v[v], fz::kBatchThreads[v], 0) !=
              cudaSuccess ||
          bps < 1)
        return fail(FIEDLER_ECUDA);
      p->batch_slots[t][v] = bps * p->sms;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, p->ks[t].serve_v[v], fz::kBatchThreads[v], 0) !=
              cudaSuccess ||
          bps < 1)
        return fail(FIEDLER_ECUDA);
      p->serve_slots[t][v] = bps * p->sms;
    }
  p->batch_var = o.batch_threads == 256 ? 1 : o.batch_threads == 128 ? 2 : 0;
  if (o.lane_sms > 0) {
    // the one-block kernels keep the block slots of at least kLaneFreeSms SMs
    if (o.lane_sms > p->sms - fiedler_plan::kLaneFreeSms) return fail(FIEDLER_EINVAL);
    const int per_slot = o.lane_sms / o.lane_slots;
    for (int t = 0; t < 2; t++) {
      const int bps = std::max(1, std::min(p->grid_blocks[t][0], p->grid_blocks[t][1]) / p->sms);
      p->lane.slot_blocks[t] = bps * per_slot;
    }
    p->lane.slots.resize(o.lane_slots);
    for (fiedler_plan::LaneSlot &sl : p->lane.slots) {
      if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) return fail(FIEDLER_ECUDA);
      if (cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) return fail(FIEDLER_ECUDA);
      if (cudaMalloc(&sl.ipart, sizeof(fz::IRed) * 2 * fz::kMaxBlocks) != cudaSuccess) return fail(FIEDLER_ENOMEM);
      if (cudaMalloc(&sl.dpart, sizeof(double) * 2 * fz::kMaxBlocks * fz::kDSum) != cudaSuccess)
        return fail(FIEDLER_ENOMEM);
      if (cudaHostAlloc((void **)&sl.h_part, 2 * sizeof(void *), cudaHostAllocDefault) != cudaSuccess)
        return fail(FIEDLER_ENOMEM);
      sl.h_part[0] = sl.ipart;
      sl.h_part[1] = sl.dpart;
    }
    p->lane.stream = p->lane.slots[0].stream;
    p->lane.ipart = p->lane.slots[0].ipart;
    p->lane.dpart = p->lane.slots[0].dpart;
  }
  p->bsync.stream = p->stream;
  if (cudaEventCreateWithFlags(&p->bsync.done, cudaEventDisableTiming) != cudaSuccess) return fail(FIEDLER_ECUDA);
  if (cudaHostAlloc((void **)&p->done, sizeof(fz::ServeDone), cudaHostAllocMapped) != cudaSuccess)
    return fail(FIEDLER_ENOMEM);
  memset(p->done, 0, sizeof(fz::ServeDone));
  if (cudaHostGetDevicePointer((void **)&p->done_dev, p->done, 0) != cudaSuccess) return fail(FIEDLER_ECUDA);
  if (cudaMalloc(&p->d_ring, sizeof(fz::ServeRing)) != cudaSuccess) return fail(FIEDLER_ENOMEM);
  if (cudaMemset(p->d_ring, 0, sizeof(fz::ServeRing)) != cudaSuccess) return fail(FIEDLER_ECUDA);
  {
    const unsigned long long idle = fiedler_plan::kIdleNs;
    if (cudaMemcpy(&p->d_ring->idle_ns, &idle, 8, cudaMemcpyHostToDevice) != cudaSuccess) return fail(FIEDLER_ECUDA);
  }
  p->stage_n = std::max(1, std::min(o.max_batch, 256));
  if (cudaMallocHost((void **)&p->h_pub, 8 * (size_t)(p->stage_n + 1)) != cudaSuccess) return fail(FIEDLER_ENOMEM);
  if (cudaMallocHost((void **)&p->h_stage, sizeof(State) * (size_t)p->stage_n) != cudaSuccess)
    return fail(FIEDLER_ENOMEM);
  if (cudaStreamCreateWithFlags(&p->io_stream, cudaStreamNonBlocking) != cudaSuccess) return fail(FIEDLER_ECUDA);
  if (cudaStreamCreateWithFlags(&p->sub_stream, cudaStreamNonBlocking) != cudaSuccess) return fail(FIEDLER_ECUDA);
  {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = p->device;
    if (cudaMemPoolCreate(&p->pool, &props) != cudaSuccess) return fail(FIEDLER_ECUDA);
    uint64_t keep = UINT64_MAX;  // freed blocks stay in the pool for the next tickets
    if (cudaMemPoolSetAttribute(p->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess)
      return fail(FIEDLER_ECUDA);
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
  return FIEDLER_OK;
}

fiedler_status fiedler_partition(fiedler_plan *p, const fiedler_graph *g, int parts, int32_t *labels,
                                 int labels_on_device, fiedler_partition_info *info) {
  if (!p || !labels || parts < 1) return FIEDLER_EINVAL;
  fiedler_status st = check_graph(g, nullptr);
  if (st != FIEDLER_OK) return st;
  std::lock_guard<std::mutex> ex(p->exec_mu);
  return partition_locked(p, g, parts, labels, labels_on_device, info);
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
  const size_t rb = r256(4 * (size_t)(g->n + 1)), cb = r256(4 * m), wb = r256(wsz * m);
  t->bytes = rb + cb + wb + 8 * (size_t)g->n;
  {
    // back-pressure: one ticket always fits into an empty queue
    const size_t qb = p->opt.queue_budget_bytes ? p->opt.queue_budget_bytes : (size_t)8 << 30;
    std::lock_guard<std::mutex> lk(p->q_mu);
    if (p->queued_bytes > 0 && p->queued_bytes + t->bytes > qb) {
      delete t;
      return FIEDLER_EAGAIN;
    }
    p->queued_bytes += t->bytes;
  }
  cudaError_t e = cudaMallocFromPoolAsync((void **)&t->buf, t->bytes, p->pool, p->sub_stream);
  if (e == cudaSuccess) {
    t->rowptr = (int32_t *)t->buf;
    t->col = (int32_t *)(t->buf + rb);
    t->w = t->buf + rb + cb;
    t->x = (double *)(t->buf + rb + cb + wb);
  } else {
    t->buf = nullptr;
  }
  const cudaMemcpyKind kind = g->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaStream_t io = p->sub_stream;
  if (e == cudaSuccess) e = cudaMemcpyAsync(t->rowptr, g->rowptr, 4 * (size_t)(g->n + 1), kind, io);
  if (e == cudaSuccess && g->nnz > 0) e = cudaMemcpyAsync(t->col, g->col, 4 * (size_t)g->nnz, kind, io);
  if (e == cudaSuccess && g->nnz > 0) e = cudaMemcpyAsync(t->w, g->w, wsz * (size_t)g->nnz, kind, io);
  if (e == cudaSuccess) e = cudaStreamSynchronize(io);  // the copies only: the input may be freed on return
  if (e != cudaSuccess) {
    std::lock_guard<std::mutex> lk(p->q_mu);
    // the pool is full while other tickets hold memory: that frees up as they
    // complete and are polled, so the caller retries (back-pressure)
    const bool busy = e == cudaErrorMemoryAllocation && (p->queued_bytes > t->bytes || p->inflight_bytes > 0);
    if (busy) (void)cudaGetLastError();
    free_ticket(p, t);
    return busy ? FIEDLER_EAGAIN : map_cuda(e);
  }
  t->footprint = item_footprint(g->n, g->nnz, p->opt.precision == FIEDLER_FP64 ? 8 : 4, g->w_dtype == FIEDLER_W_F64,
                                p->opt);
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

namespace {

// The large graphs of a batched call, solved by the cooperative grid-wide
// kernels on the lane's slots (graph i on slot i mod lane_slots, one after
// another within a slot, each slot on lane_sms / lane_slots SMs with its own
// stream and reduction partials) while the batched kernel, launched with the
// lane's SMs left free, runs the others.  lane_queue queues them (their device
// memory stays allocated until lane_finish), lane_finish waits, fills the
// results and reruns any graph whose hierarchy outgrew its arena or scratch.
struct LaneBatch {
  std::vector<BatchItem> items;
  State *hs = nullptr;  // pinned: the state copies must not block the host
  char *d = nullptr;
  double scale = 1.0;
  ~LaneBatch() {
    if (hs) cudaFreeHost(hs);
  }
};

fiedler_status lane_queue(fiedler_plan *p, LaneBatch &lb, int type) {
  const size_t tsz = type == 0 ? 8 : 4;
  const int nbl = p->lane.slot_blocks[type];
  const size_t nsl = p->lane.slots.size();
  std::vector<size_t> off(lb.items.size());
  size_t total = 0;
  for (size_t i = 0; i < lb.items.size(); i++) {
    BatchItem &it = lb.items[i];
    it.arena_b = r256((size_t)(arena_estimate(it.n, it.nnz, tsz, it.wf64, p->opt) * lb.scale));
    it.scratch_b = r256((size_t)(scratch_estimate(it.n, it.nnz, nbl, p->opt) * lb.scale));
    off[i] = total;
    total += r256(sizeof(State)) + it.arena_b + it.scratch_b;
    if (it.host_in)
      total += r256(4 * (size_t)(it.n + 1)) + r256(4 * (size_t)std::max<int64_t>(it.nnz, 1)) +
               r256((it.wf64 ? 8 : 4) * (size_t)std::max<int64_t>(it.nnz, 1));
    if (it.user_x && !it.user_x_dev) total += r256(8 * (size_t)it.n);
  }
  CK(cudaMallocAsync((void **)&lb.d, std::max<size_t>(total, 256), p->lane.stream));
  if (nsl > 1) {  // the other slots start after the allocation
    cudaEvent_t e = nullptr;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaEventRecord(e, p->lane.stream));
    for (size_t k = 1; k < nsl; k++) CK(cudaStreamWaitEvent(p->lane.slots[k].stream, e, 0));
    cudaEventDestroy(e);
  }
  if (lb.hs) cudaFreeHost(lb.hs);
  lb.hs = nullptr;
  CK(cudaMallocHost((void **)&lb.hs, sizeof(State) * lb.items.size()));
  const fz::KernelSet &K = p->ks[type];
  for (size_t i = 0; i < lb.items.size(); i++) {
    BatchItem &it = lb.items[i];
    const fiedler_plan::LaneSlot &sl = p->lane.slots[i % nsl];
    char *base = lb.d + off[i];
    State *h = &lb.hs[i];
    memset(h, 0, sizeof(State));
    fill_opts(h->opt, p->opt, type);
    h->opt.fault_inject = 0;
    h->bad_index = LLONG_MAX;
    h->n0 = (int)it.n;
    h->nnz0 = (int)it.nnz;
    h->arena = base + r256(sizeof(State));
    h->arena_size = it.arena_b;
    h->scratch = h->arena + it.arena_b;
    h->scratch_size = it.scratch_b;
    char *q = h->scratch + it.scratch_b;
    h->in_rowptr = it.rp;
    h->in_col = it.ci;
    h->in_w = it.w;
    h->in_w_f64 = it.wf64;
    if (it.host_in) {
      const size_t rb = r256(4 * (size_t)(it.n + 1)), cb = r256(4 * (size_t)std::max<int64_t>(it.nnz, 1));
      CK(cudaMemcpyAsync(q, it.rp, 4 * (size_t)(it.n + 1), cudaMemcpyHostToDevice, sl.stream));
      if (it.nnz > 0) {
        CK(cudaMemcpyAsync(q + rb, it.ci, 4 * (size_t)it.nnz, cudaMemcpyHostToDevice, sl.stream));
        CK(cudaMemcpyAsync(q + rb + cb, it.w, (it.wf64 ? 8 : 4) * (size_t)it.nnz, cudaMemcpyHostToDevice,
                           sl.stream));
      }
      h->in_rowptr = (const int *)q;
      h->in_col = (const int *)(q + rb);
      h->in_w = q + rb + cb;
      q += rb + cb + r256((it.wf64 ? 8 : 4) * (size_t)std::max<int64_t>(it.nnz, 1));
    }
    h->xout = it.user_x ? (it.user_x_dev ? it.user_x : (double *)q) : nullptr;
    it.x_off = (size_t)(q - lb.d);
    h->ipart = sl.ipart;
    h->dpart = sl.dpart;
    CK(cudaMemcpyAsync(base, h, sizeof(State), cudaMemcpyHostToDevice, sl.stream));
    void *args[] = {(void *)&base};
    CK(cudaLaunchCooperativeKernel(K.grid_setup, dim3(nbl), dim3(fz::kGridThreads), args, 0, sl.stream));
    CK(cudaLaunchKernel(K.cta, dim3(1), dim3(fz::kCtaThreads), args, 0, sl.stream));
    CK(cudaLaunchCooperativeKernel(K.grid_solve, dim3(nbl), dim3(fz::kGridThreads), args, 0, sl.stream));
    CK(cudaMemcpyAsync(h, base, sizeof(State), cudaMemcpyDeviceToHost, sl.stream));
    it.in_off = off[i];
  }
  return FIEDLER_OK;
}

fiedler_status lane_finish(fiedler_plan *p, LaneBatch &lb, int type) {
  for (int attempt = 0;; attempt++) {
    for (const fiedler_plan::LaneSlot &sl : p->lane.slots) CK(cudaStreamSynchronize(sl.stream));
    std::vector<BatchItem> again;
    for (size_t i = 0; i < lb.items.size(); i++) {
      BatchItem &it = lb.items[i];
      const State *h = &lb.hs[i];
      it.st = h->status;
      if (needs_rerun(h->status) && attempt < 3) {
        again.push_back(it);
        continue;
      }
      fiedler_result r{};
      fiedler_status out = map_status(h->status);
      if (out == FIEDLER_OK && !h->finalized) out = FIEDLER_ECUDA;
      if (out == FIEDLER_OK && h->capped) out = FIEDLER_ENOTCONVERGED;
      if (needs_rerun(h->status)) out = FIEDLER_ENOMEM;
      r.levels = h->nlevels;
      r.coarsest_n = h->nlevels > 0 ? h->lv[h->coarsest].n : 0;
      r.bad_index = h->bad_index == LLONG_MAX ? -1 : h->bad_index;
      double ns = 0.0;
      for (int k = 0; k < 2; k++)
        for (int ph = 0; ph < fz::PH_COUNT; ph++) ns += h->phase_ns[k][ph];
      r.ms = (float)(ns * 1e-6);
      if (out == FIEDLER_OK || out == FIEDLER_ENOTCONVERGED) {
        r.lambda2 = h->lambda;
        r.residual = h->residual;
        r.ortho = h->ortho;
        r.pi_iters_total = h->pi_total;
        r.gs_sweeps_total = h->gs_total;
        r.refine_iters = h->refine_total;
        if (it.user_x && !it.user_x_dev)
          CK(cudaMemcpy(it.user_x, lb.d + it.x_off, 8 * (size_t)it.n, cudaMemcpyDeviceToHost));
      }
      r.x = it.user_x;
      r.x_on_device = it.user_x_dev;
      r.status = out;
      if (it.res) *it.res = r;
    }
    CK(cudaFreeAsync(lb.d, p->lane.stream));
    lb.d = nullptr;
    if (again.empty()) return FIEDLER_OK;
    lb.items = again;
    lb.scale *= 2.0;
    fiedler_status st = lane_queue(p, lb, type);
    if (st != FIEDLER_OK) return st;
  }
}

}  // namespace

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
  LaneBatch lb;
  c.reserve_sms = 0;
  if (p->lane.stream) {  // the large graphs to the lane, queued first so that both run at once
    std::vector<BatchItem> rest;
    for (auto &it : c.items) (it.n >= p->opt.lane_min_n ? lb.items : rest).push_back(it);
    if (!lb.items.empty()) {
      cudaEvent_t e = nullptr;
      CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      CK(cudaEventRecord(e, p->stream));  // inputs the caller queued on the plan's stream
      for (const fiedler_plan::LaneSlot &sl : p->lane.slots) CK(cudaStreamWaitEvent(sl.stream, e, 0));
      cudaEventDestroy(e);
      fiedler_status st = lane_queue(p, lb, c.type);
      if (st != FIEDLER_OK) return st;
      c.items = rest;
      c.reserve_sms = p->opt.lane_sms;
    }
  }
  fiedler_status st = c.items.empty() ? FIEDLER_OK : batch_run_sync(p, c);
  if (!lb.items.empty()) {
    fiedler_status ls = lane_finish(p, lb, c.type);
    if (st == FIEDLER_OK) st = ls;
  }
  c.reserve_sms = 0;
  return st;
}

fiedler_status fiedler_plan_autotune(fiedler_plan *p, const fiedler_graph *graphs, int count, fiedler_tuning *out) {
  if (!p || !graphs || count < 1 || p->opt.batch_threads != 0) return FIEDLER_EINVAL;
  std::lock_guard<std::mutex> ex(p->exec_mu);
  // throughput, not the latency of the largest graph: the sample is repeated
  // until every variant has at least two graphs per resident block, as far as
  // the repeated graphs' memory stays within the serving budget (else the
  // sample as it is, cut to that budget, at least one graph)
  const int type = p->opt.precision == FIEDLER_FP64 ? 0 : 1;
  const size_t tsz = type == 0 ? 8 : 4;
  const size_t budget = p->opt.hbm_budget_bytes ? p->opt.hbm_budget_bytes : (size_t)16 << 30;
  int want = count;
  for (int v = 0; v < 3; v++) want = std::max(want, 2 * p->batch_slots[type][v]);
  int total = 0;
  size_t bytes = 0;
  while (total < want) {
    const fiedler_graph &g = graphs[total % count];
    const size_t f = item_footprint(g.n, g.nnz, tsz, g.w_dtype == FIEDLER_W_F64, p->opt);
    if (total > 0 && bytes + f > budget) break;
    bytes += f;
    total++;
  }
  std::vector<fiedler_result> res((size_t)total);
  BatchCtx &c = p->bsync;
  auto run = [&](int var, float *ms) -> fiedler_status {
    p->batch_var = var;
    c.items.clear();
    c.type = type;
    for (int i = 0; i < total; i++) {
      const fiedler_graph &g = graphs[i % count];
      fiedler_status st = check_graph(&g, &res[i]);
      if (st != FIEDLER_OK) return st;
      BatchItem it{};
      it.n = g.n;
      it.nnz = g.nnz;
      it.rp = g.rowptr;
      it.ci = g.col;
      it.w = g.w;
      it.wf64 = g.w_dtype == FIEDLER_W_F64;
      it.host_in = !g.on_device;
      it.user_x = nullptr;
      it.res = &res[i];
      c.items.push_back(it);
    }
    CK(cudaEventRecord(p->ev[0], p->stream));
    fiedler_status st = batch_run_sync(p, c);
    CK(cudaEventRecord(p->ev[1], p->stream));
    CK(cudaEventSynchronize(p->ev[1]));
    if (ms) CK(cudaEventElapsedTime(ms, p->ev[0], p->ev[1]));
    return st;
  };
  fiedler_tuning t{};
  fiedler_status st = run(0, nullptr);  // sizes the buffers once
  int best = 0;
  for (int v = 0; v < 3 && st == FIEDLER_OK; v++) {
    st = run(v, &t.batch_ms[v]);
    if (st == FIEDLER_OK && t.batch_ms[v] < t.batch_ms[best]) best = v;
  }
  p->batch_var = st == FIEDLER_OK ? best : 0;
  t.batch_threads = fz::kBatchThreads[p->batch_var];
  if (out) *out = t;
  return st;
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
  out->launches = p->n_launches;
  out->block_seconds = p->block_seconds;
  out->mean_inflight = p->live_rounds ? p->live_sum / (double)p->live_rounds : 0.0;
  out->mean_blocks = p->live_rounds ? p->alive_sum / (double)p->live_rounds : 0.0;
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
      cudaError_t e = cudaMemcpyAsync(x, t->x, 8 * (size_t)t->n,
                                      xod ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->io_stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(p->io_stream);
      if (e != cudaSuccess) st = map_cuda(e);
    }
  }
  p->tickets.erase(it);
  free_ticket(p, t);
  return st;
}

fiedler_status fiedler_poll_any(fiedler_plan *p, uint64_t *tickets, int max, int timeout_ms, int *count) {
  if (!p || !tickets || max < 1 || !count) return FIEDLER_EINVAL;
  std::unique_lock<std::mutex> lk(p->q_mu);
  auto ready = [&] { return !p->finished.empty(); };
  if (!ready()) {
    if (timeout_ms < 0) p->q_cv.wait(lk, ready);
    else if (timeout_ms > 0) p->q_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  }
  int k = 0;
  while (k < max && !p->finished.empty()) {
    const uint64_t id = p->finished.front();
    p->finished.pop_front();
    if (p->tickets.count(id)) tickets[k++] = id;  // still held (not polled yet)
  }
  *count = k;
  return k > 0 ? FIEDLER_OK : FIEDLER_EAGAIN;
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
  if (p->io_stream) cudaStreamSynchronize(p->io_stream);
  if (p->sub_stream) cudaStreamSynchronize(p->sub_stream);
  std::vector<BatchCtx *> ctxs{&p->bsync};
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
  for (fiedler_plan::LaneSlot &sl : p->lane.slots) {
    if (sl.stream) {
      cudaStreamSynchronize(sl.stream);
      cudaStreamDestroy(sl.stream);
    }
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.ipart) cudaFree(sl.ipart);
    if (sl.dpart) cudaFree(sl.dpart);
    if (sl.h_part) cudaFreeHost(sl.h_part);
  }
  if (p->h_state) cudaFreeHost(p->h_state);
  for (int i = 0; i < 10; i++)
    if (p->ev[i]) cudaEventDestroy(p->ev[i]);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  for (auto &L : p->serve) {
    if (L.stream) cudaStreamDestroy(L.stream);
    if (L.ev) cudaEventDestroy(L.ev);
  }
  if (p->done) cudaFreeHost(p->done);
  if (p->d_ring) cudaFree(p->d_ring);
  if (p->h_pub) cudaFreeHost(p->h_pub);
  if (p->h_stage) cudaFreeHost(p->h_stage);
  if (p->io_stream) cudaStreamDestroy(p->io_stream);
  if (p->sub_stream) cudaStreamDestroy(p->sub_stream);
  if (p->pool) cudaMemPoolDestroy(p->pool);
  delete p;
}

const char *fiedler_status_str(fiedler_status s) {
  switch (s) {
    case FIEDLER_OK: return "ok";
    case FIEDLER_EAGAIN: return "still in flight (poll) or queue full (submit)";
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
  info->refine_iters = L.refine_iters;
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
