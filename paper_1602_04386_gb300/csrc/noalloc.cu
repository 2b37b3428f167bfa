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

#include <chrono>
#include <mutex>

#include "engine.cuh"
#include "fiedler.h"

namespace {

// 16 MiB: enough for graphs up to roughly 80k vertices and 300k stored entries
constexpr size_t kNoAllocBytes = 16u << 20;

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
size_t scratch_bytes(int64_t n, int64_t nnz) {
  return round256((size_t)(44.0 * n + 4.0 * (n + 1) * 9 + 16.0 * nnz + 4.0 * fz::kMaxColors + 64.0 * 256.0));
}

// hierarchy bound: the fine level plus coarse levels of at most 2n vertices and
// 2 nnz entries in total (the same bound the plan-owned arena starts from)
size_t arena_bytes(int64_t n, int64_t nnz, size_t tsz, bool wf64) {
  double l0 = 4.0 * (n + 1) + (4.0 + (wf64 ? 8.0 : 4.0)) * nnz + 8.0 * n + 12.0 * n + 8.0 * n +
              4.0 * (fz::kMaxColors + 1) + 4.0 * (n + 1) + (4.0 + tsz) * nnz + (2.0 * tsz + 4.0) * n;
  double lc = 2.0 * (4.0 * n + 16.0 * nnz + 8.0 * n + 12.0 * n + 8.0 * n + 4.0 * n + (4.0 + tsz) * nnz +
                     (2.0 * tsz + 4.0) * n) +
              fz::kMaxLevels * 4.0 * (fz::kMaxColors + 1) + fz::kMaxLevels * 24.0 * 256.0;
  return round256((size_t)(l0 + lc));
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

}  // namespace

extern "C" fiedler_status fiedler_solve_noalloc(const fiedler_options *opts, const fiedler_graph *g, double *x,
                                                void *cuda_stream, fiedler_result *res) {
  if (!g || g->n < 2 || g->nnz < 0 || !g->rowptr || (g->nnz > 0 && (!g->col || !g->w)) || !g->on_device ||
      (g->w_dtype != FIEDLER_W_F32 && g->w_dtype != FIEDLER_W_F64))
    return FIEDLER_EINVAL;
  if (g->n >= INT_MAX || g->nnz >= INT_MAX) return FIEDLER_ENOTSUP;
  fiedler_options o;
  if (opts) o = *opts;
  else fiedler_options_default(&o);
  if ((o.precision != FIEDLER_FP64 && o.precision != FIEDLER_FP32_FP64RED) || o.max_levels < 1 ||
      o.max_levels > fz::kMaxLevels || o.gs_sweeps < 0 || o.pi_max_iters < 0 || o.pi_max_iters_coarsest < 0 ||
      !(o.stall_ratio > 0.0 && o.stall_ratio <= 1.0) || o.coarse_max_n < 1 || o.barrier_timeout_ms < 1)
    return FIEDLER_EINVAL;
  const bool wf64 = g->w_dtype == FIEDLER_W_F64;
  const size_t tsz = o.precision == FIEDLER_FP64 ? 8 : 4;
  // fixed layout: state | arena | scratch; larger problems are refused up front
  const size_t state_b = round256(sizeof(fz::State));
  const size_t scratch_b = scratch_bytes(g->n, g->nnz);
  const size_t need = state_b + arena_bytes(g->n, g->nnz, tsz, wf64) + scratch_b;
  if (need > kNoAllocBytes) {
    if (res) {
      res->status = FIEDLER_ENOTSUP;
      res->bad_index = -1;
    }
    return FIEDLER_ENOTSUP;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FIEDLER_ECUDA;
  if (!g_dev_base[dev]) {
    // set-up on the first call on this device (this device current): the
    // array's name is a host-side stand-in, the kernel needs its device address
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc) != cudaSuccess || !p) return FIEDLER_ECUDA;
    g_dev_base[dev] = (unsigned char *)p;
  }
  unsigned char *base = g_dev_base[dev];
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  fz::State *h = &g_host_state;
  memset(h, 0, sizeof(fz::State));
  fz::Opts &so = h->opt;
  so.precision = o.precision;
  so.coarse_max_n = o.coarse_max_n;
  so.max_levels = o.max_levels;
  so.gs_sweeps = o.gs_sweeps;
  so.pi_max_iters = o.pi_max_iters;
  so.pi_max_iters_coarsest = o.pi_max_iters_coarsest;
  so.tie_rule = o.tie_rule;
  so.validate = o.validate;
  so.tail_max_n = INT_MAX;  // every level in the one-block engine
  so.tail_max_nnz = INT_MAX;
  so.fault_inject = 0;
  so.stall_ratio = o.stall_ratio;
  so.pi_cos_tol = o.pi_cos_tol;
  so.resid_tol = o.resid_tol;
  so.guard = tsz == 8 ? ldexp(1.0, -20) : ldexp(1.0, -16);
  so.seed = o.seed;
  so.barrier_timeout_ns = (unsigned long long)o.barrier_timeout_ms * 1000000ull;
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
  if (cudaMemcpyAsync(base, h, sizeof(fz::State), cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return FIEDLER_ECUDA;
  void *args[] = {(void *)&base};
  const void *fn = tsz == 8 ? (const void *)fz_noalloc_f64 : (const void *)fz_noalloc_f32;
  cudaError_t err = cudaLaunchKernel(fn, dim3(1), dim3(fz::kCtaThreads), args, 0, stream);
  if (err == cudaSuccess) err = cudaMemcpyAsync(h, base, sizeof(fz::State), cudaMemcpyDeviceToHost, stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
  const float ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (err != cudaSuccess) return err == cudaErrorMemoryAllocation ? FIEDLER_ENOMEM : FIEDLER_ECUDA;
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
    }
    res->x = x;
    res->x_on_device = 1;
    res->status = out;
  }
  return out;
}
