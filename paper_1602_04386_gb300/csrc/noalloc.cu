// noalloc.cu -- fiedler_solve_noalloc: a solve that allocates no memory.
//
// Some callers cannot call cudaMalloc: code running inside a memory-capped
// pool or arena owned by someone else, plug-ins that must not grow the
// process's device footprint after start-up, or hosts that forbid allocation
// on a latency-critical path.  For them this entry point runs the one-block
// level engine (every level of the hierarchy, small graphs only) on a
// file-scope device array instead of plan-owned arenas.  The caller passes
// device-resident inputs and a device output vector; nothing else is needed.
//
// The array holds, in order, the solve state, the hierarchy arena and the
// per-level scratch.  Every GPU that loads this library keeps it for the
// life of the process.  Each call overwrites it, so calls must not overlap
// on the GPU; the host side serialises callers of this process with a mutex
// and every call returns only after its work on the stream has finished.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>

#include "engine.cuh"
#include "fiedler.h"
#include "host_opts.h"

namespace {

// 16 MiB: enough for graphs up to roughly 80k vertices and 300k stored entries
constexpr size_t kNoAllocBytes = 16u << 20;
constexpr size_t kScratchSlack = 1u << 20;

static __device__ __align__(256) unsigned char g_noalloc[kNoAllocBytes];

__global__ void __launch_bounds__(fz::kCtaThreads, 1) fz_noalloc_f32(fz::State *S) {
  fz::engine_entry<float, false>(S, 1);
}
__global__ void __launch_bounds__(fz::kCtaThreads, 1) fz_noalloc_f64(fz::State *S) {
  fz::engine_entry<double, false>(S, 1);
}

constexpr int kMaxDevices = 64;
unsigned char *g_dev_base[kMaxDevices];  // device address of g_noalloc, per device
fz::State g_host_state;                  // host staging copy of the state (static)
std::mutex g_mu;

size_t round256(size_t b) { return (b + 255u) & ~(size_t)255u; }

// per-level scratch bound (every level is at most as large as the fine one)
size_t scratch_bytes(int64_t n, int64_t nnz, int hec_mode) {
  return round256((size_t)(56.0 * n + 4.0 * (n + 1) * 9 + 16.0 * nnz + 4.0 * fz::kMaxColors + 64.0 * 256.0 +
                           (hec_mode == FIEDLER_HEC_PAPER ? 44.0 * n + 8.0 * 256.0 : 0.0)));
}

// hierarchy bound: the fine level plus coarse levels of at most 2n vertices and
// 2 nnz entries in total (the same bound the plan-owned arena starts from)
size_t arena_bytes(int64_t n, int64_t nnz, size_t tsz, bool wf64, int refine, int basis, int precond) {
  double l0 = 4.0 * (n + 1) + (4.0 + (wf64 ? 8.0 : 4.0)) * nnz + 8.0 * n + 12.0 * n + 8.0 * n +
              4.0 * (fz::kMaxColors + 1) + 4.0 * (n + 1) + (4.0 + tsz) * nnz + (2.0 * tsz + 4.0) * n;
  double lc = 2.0 * (4.0 * n + 16.0 * nnz + 8.0 * n + 12.0 * n + 8.0 * n + 4.0 * n + (4.0 + tsz) * nnz +
                     (2.0 * tsz + 4.0) * n) +
              fz::kMaxLevels * 4.0 * (fz::kMaxColors + 1) + fz::kMaxLevels * 24.0 * 256.0;
  return round256((size_t)(l0 + lc + fz::refine_bytes(n, tsz, refine, basis, precond)));
}

fiedler_status status_of(int st) {
  switch (st) {
    case fz::ST_OK: return FIEDLER_OK;
    case fz::ST_EINVAL: return FIEDLER_EINVAL;
    case fz::ST_EDISC: return FIEDLER_EDISCONNECTED;
    case fz::ST_ETIMEOUT: return FIEDLER_ETIMEOUT;
    case fz::ST_EDEGEN: return FIEDLER_EDEGENERATE;
    case fz::ST_ENOTSUP: return FIEDLER_ENOTSUP;
    case fz::ST_ARENA:
    case fz::ST_SCRATCH: return FIEDLER_ENOTSUP;  // the hierarchy outgrew the fixed array
    default: return FIEDLER_ECUDA;
  }
}

// a refused call still reports its status (and no offending position) in *res
fiedler_status refuse(fiedler_result *res, fiedler_status st) {
  if (res) {
    res->status = st;
    res->bad_index = -1;
  }
  return st;
}

}  // namespace

extern "C" fiedler_status fiedler_solve_noalloc(const fiedler_options *opts, const fiedler_graph *g, double *x,
                                                void *cuda_stream, fiedler_result *res) {
  if (!g || g->n < 2 || g->nnz < 0 || !g->rowptr || (g->nnz > 0 && (!g->col || !g->w)) || !g->on_device ||
      (g->w_dtype != FIEDLER_W_F32 && g->w_dtype != FIEDLER_W_F64))
    return refuse(res, FIEDLER_EINVAL);
  if (g->n >= INT_MAX || g->nnz >= INT_MAX) return refuse(res, FIEDLER_ENOTSUP);
  fiedler_options o;
  if (opts) o = *opts;
  else fiedler_options_default(&o);
  // the checks of fiedler_plan_create: the same options give the same status
  if (!fz::options_valid(o)) return refuse(res, FIEDLER_EINVAL);
  const bool wf64 = g->w_dtype == FIEDLER_W_F64;
  const int type = o.precision == FIEDLER_FP64 ? 0 : 1;
  const size_t tsz = type == 0 ? 8 : 4;
  // fixed layout: state | arena | scratch; larger problems are refused up front
  const size_t state_b = round256(sizeof(fz::State));
  size_t scratch_b = scratch_bytes(g->n, g->nnz, o.hec_mode);
  const size_t need = state_b + arena_bytes(g->n, g->nnz, tsz, wf64, o.refine, o.lanczos_basis, o.refine_precond) + scratch_b;
  if (need > kNoAllocBytes) return refuse(res, FIEDLER_ENOTSUP);
  // the plan's scratch keeps 1 MiB of slack; give it here too when the array has room
  scratch_b += std::min(kScratchSlack, (kNoAllocBytes - need) & ~(size_t)255u);
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  {
    // every call ends in a stream synchronisation and reads pageable host
    // memory, neither of which a stream capture allows
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) return refuse(res, FIEDLER_ECUDA);
    if (cs != cudaStreamCaptureStatusNone) return refuse(res, FIEDLER_EINVAL);
  }
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return refuse(res, FIEDLER_ECUDA);
  if (!g_dev_base[dev]) {
    // set-up on the first call on this device (this device current): the
    // array's name is a host-side stand-in, the kernel needs its device address
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc) != cudaSuccess || !p) return refuse(res, FIEDLER_ECUDA);
    g_dev_base[dev] = (unsigned char *)p;
  }
  unsigned char *base = g_dev_base[dev];
  fz::State *h = &g_host_state;
  memset(h, 0, sizeof(fz::State));
  fz::fill_opts(h->opt, o, type);
  h->opt.tail_max_n = INT_MAX;  // every level in the one-block engine
  h->opt.tail_max_nnz = INT_MAX;
  h->opt.fault_inject = 0;
  h->bad_index = LLONG_MAX;
  h->n0 = (int)g->n;
  h->nnz0 = (int)g->nnz;
  h->in_rowptr = g->rowptr;
  h->in_col = g->col;
  h->in_w = g->w;
  h->in_w_f64 = wf64;
  h->arena = (char *)base + state_b;
  h->arena_size = kNoAllocBytes - state_b - scratch_b;
  h->scratch = (char *)base + (kNoAllocBytes - scratch_b);
  h->scratch_size = scratch_b;
  h->xout = x;
  h->ipart = nullptr;  // grid-wide partials: unused by the one-block engine
  h->dpart = nullptr;
  const auto t0 = std::chrono::steady_clock::now();
  cudaError_t err = cudaMemcpyAsync(base, h, sizeof(fz::State), cudaMemcpyHostToDevice, stream);
  if (err == cudaSuccess) {
    void *args[] = {(void *)&base};
    const void *fn = tsz == 8 ? (const void *)fz_noalloc_f64 : (const void *)fz_noalloc_f32;
    err = cudaLaunchKernel(fn, dim3(1), dim3(fz::kCtaThreads), args, 0, stream);
    if (err == cudaSuccess) err = cudaMemcpyAsync(h, base, sizeof(fz::State), cudaMemcpyDeviceToHost, stream);
  }
  // whatever was queued finishes before the lock is released: the next caller
  // (perhaps on another stream) overwrites the same array
  const cudaError_t serr = cudaStreamSynchronize(stream);
  if (err == cudaSuccess) err = serr;
  const float ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (err != cudaSuccess) return refuse(res, err == cudaErrorMemoryAllocation ? FIEDLER_ENOMEM : FIEDLER_ECUDA);
  fiedler_status out = status_of(h->status);
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
    res->x = x;
    res->x_on_device = 1;
    res->status = out;
  }
  return out;
}
