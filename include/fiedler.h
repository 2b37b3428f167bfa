/*
 * fiedler.h -- C-ABI of the GB300 cascadic multigrid Fiedler-vector solver.
 *
 * The library computes the second smallest eigenpair (lambda_2, phi_2) of a
 * weighted graph Laplacian (Def 2.1 and Def 2.2 of S. Gandhi, "Improvement of
 * the Cascadic Multigrid Algorithm with a Gauss Seidel Smoother to Efficiently
 * Compute the Fiedler Vector of a Graph Laplacian", 2015) with the method of
 * its Alg. 3: heavy edge coarsening (Alg. 1) into a Galerkin hierarchy
 * L^{i+1} = I L^i I^T, a coarsest-level solve, and cascadic refinement
 * y^j = I^T y^{j+1} followed by Gauss-Seidel sweeps (Alg. 2), power iteration
 * on the shifted matrix sigma I - L with deflation of the constant vector, and
 * a final Rayleigh quotient (Sec. 2), stopped by (u^k, u^{k-1}) > 1 - tol
 * (Sec. 3).  Every step runs in hand-written sm_103a CUDA kernels.
 *
 * Conventions shared by every entry point:
 *  - No exceptions or aborts cross this ABI; every call returns a status.
 *  - Graphs are symmetric adjacency matrices in CSR form: rowptr[n+1] (int32,
 *    rowptr[0] = 0, non-decreasing, rowptr[n] = nnz), col[nnz] (int32, strictly
 *    ascending within a row), w[nnz] (float or double, finite, > 0 off the
 *    diagonal, w_ij == w_ji bit for bit).  Diagonal entries (self-loops) are
 *    accepted and dropped.  The Laplacian is L = D - W with d_i = sum_j w_ij.
 *  - Inputs are borrowed for the duration of the call only.  Device pointers
 *    must be on the plan's device; host pointers may be pageable or pinned.
 *  - A plan is not thread-safe: one solve at a time per plan.  Plans on the
 *    same device may be used from different threads.
 *  - All device memory the library needs beyond the caller's inputs and
 *    outputs is owned by the plan (device-side bump arenas, grown on demand
 *    and kept between solves) and released by fiedler_plan_destroy.
 */
#ifndef FIEDLER_H
#define FIEDLER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FIEDLER_OK = 0,
  FIEDLER_EAGAIN = 1,            /* fiedler_poll: the ticket is still in flight;
                                    fiedler_batch_submit: the queue budget is used up */
  FIEDLER_EINVAL = -1,           /* malformed arguments or CSR (see result.bad_index) */
  FIEDLER_ENOMEM = -2,           /* device memory could not be obtained */
  FIEDLER_EDISCONNECTED = -3,    /* the graph is not connected: lambda_2 = 0 is degenerate */
  FIEDLER_ENOTCONVERGED = -4,    /* a power-iteration cap was hit; the result is still returned */
  FIEDLER_ETIMEOUT = -5,         /* a bounded device-side wait gave up */
  FIEDLER_ECUDA = -6,            /* a CUDA runtime call failed */
  FIEDLER_ECANCELED = -7,        /* the ticket was cancelled */
  FIEDLER_EDEGENERATE = -8,      /* an iterate vanished after deflation (cannot be normalised) */
  FIEDLER_ENOTSUP = -9           /* a compiled-in size limit was exceeded */
} fiedler_status;

/* fiedler_options.precision */
enum { FIEDLER_FP64 = 0, FIEDLER_FP32_FP64RED = 1 };
/* fiedler_options.tie_rule: heavy-edge ties broken by a hash of the edge's
 * vertex indices (then the indices), or by the indices alone */
enum { FIEDLER_TIE_HASHED = 0, FIEDLER_TIE_INDEX = 1 };
/* fiedler_graph.w_dtype */
enum { FIEDLER_W_F32 = 0, FIEDLER_W_F64 = 1 };
/* fiedler_options.refine: what runs on the finest level after its Gauss-Seidel
 * sweeps.  NONE is the method as the paper states it (power iteration on
 * sigma I - L, stopped by the cosine test of Sec. 3).  The two Krylov
 * eigensolvers replace that power iteration on the finest level only and run
 * until the eigen-residual is below refine_tol (Sec. 4 proposes a Lanczos
 * smoother as future work; the cosine test stops power iteration long before
 * the residual is small on graphs with a wide spread of degrees):
 *  - LOBPCG: single-vector locally optimal preconditioned conjugate gradient
 *    (Knyazev, 2001) on 1-perp, preconditioned as refine_precond says;
 *  - LANCZOS: Lanczos with full reorthogonalisation on 1-perp, restarted from
 *    the Ritz vector every lanczos_basis steps. */
enum { FIEDLER_REFINE_NONE = 0, FIEDLER_REFINE_LOBPCG = 1, FIEDLER_REFINE_LANCZOS = 2 };
/* fiedler_options.hec_mode: heavy-edge coarsening rule (Alg. 1).  DOMINANT:
 * the deterministic locally dominant matching under the order of tie_rule
 * (default).  PAPER: Alg. 1 as printed, vertices visited in a seeded random
 * order, each unaggregated vertex pairing with its heaviest neighbour or
 * joining that neighbour's aggregate; the order on level l is the ascending
 * order of the keys splitmix64(seed + l, v) (ties by v). */
enum { FIEDLER_HEC_DOMINANT = 0, FIEDLER_HEC_PAPER = 1 };
/* fiedler_options.refine_precond: LOBPCG's preconditioner.  DEGREE: D^-1.
 * VCYCLE (default): one V-cycle of the cascade's own hierarchy on L e = r
 * (a project addition; the paper has no preconditioner): one forward
 * Gauss-Seidel sweep from e = 0 per level (colour classes ascending), the
 * residual summed over each aggregate as the next level's right-hand side,
 * 20 sweeps and the mean removed on the coarsest level, the correction added
 * to every member, one backward sweep (classes descending). */
enum { FIEDLER_PRECOND_DEGREE = 0, FIEDLER_PRECOND_VCYCLE = 1 };

typedef struct {
  int precision;             /* FIEDLER_FP64: values and arithmetic in double.
                                FIEDLER_FP32_FP64RED: Laplacian values, Gauss-Seidel and the
                                power-iteration matvec in float; deflation, normalisation,
                                dot products and the Rayleigh quotient in double. */
  int coarse_max_n;          /* coarsen while n > coarse_max_n (Alg. 3 uses 25) */
  int max_levels;            /* at most this many levels, fine level included (<= 32) */
  double stall_ratio;        /* a coarse level with more than stall_ratio * n vertices is not built */
  int gs_sweeps;             /* Gauss-Seidel sweeps per level (Alg. 2 with N = gs_sweeps) */
  int pi_max_iters;          /* power-iteration cap on every level but the coarsest */
  int pi_max_iters_coarsest; /* power-iteration cap on the coarsest level */
  double pi_cos_tol;         /* stop when (u^k, u^{k-1}) > 1 - pi_cos_tol (Sec. 3: 1e-6) */
  double resid_tol;          /* 0: paper stop rule only; > 0: also require ||L u - rho u|| <= resid_tol * sigma */
  int tie_rule;              /* FIEDLER_TIE_HASHED (default) or FIEDLER_TIE_INDEX */
  uint64_t seed;             /* random start vector on the coarsest level (splitmix64 stream) */
  int validate;              /* 1: check the CSR on the device (symmetry, order, weights) */
  int tail_max_n;            /* levels with n <= tail_max_n and nnz <= tail_max_nnz run in one
                                thread block; larger levels run in a cooperative grid-wide
                                kernel.  Levels with n <= 256 and nnz <= 4096 always run in
                                the thread block. */
  int tail_max_nnz;          /* see tail_max_n */
  int barrier_timeout_ms;    /* bound on every device-side wait (grid barriers) */
  int fault_inject;          /* testing only: 1 = one block skips the first grid barrier, so the
                                others' bounded wait runs out and the solve reports ETIMEOUT */
  size_t hbm_budget_bytes;   /* serving: device memory the in-flight tickets may hold (0 = 16 GiB) */
  int max_batch;             /* serving: most tickets admitted in one scheduling round */
  size_t queue_budget_bytes; /* serving: device memory the copied inputs of submitted, not yet
                                polled tickets may hold (0 = 8 GiB); beyond it fiedler_batch_submit
                                returns FIEDLER_EAGAIN */
  int batch_threads;         /* batched and serving forms: threads per graph's block, 512, 256 or
                                128 (1, 2 or 4 graphs per SM); 0 = 512 until fiedler_plan_autotune
                                picks one */
  int refine;                /* FIEDLER_REFINE_NONE (default), _LOBPCG or _LANCZOS (see above) */
  int refine_max_iters;      /* cap on the finest level's Krylov matvecs; reaching it gives
                                FIEDLER_ENOTCONVERGED with the result filled */
  double refine_tol;         /* Krylov stop: ||L x - theta x|| <= refine_tol * theta * ||x||,
                                theta = x^T L x / x^T x */
  int lanczos_basis;         /* FIEDLER_REFINE_LANCZOS: basis vectors per restart cycle, 4..64 */
  int hec_mode;              /* FIEDLER_HEC_DOMINANT (default) or FIEDLER_HEC_PAPER */
  int refine_precond;        /* FIEDLER_PRECOND_VCYCLE (default) or FIEDLER_PRECOND_DEGREE */
  int lane_sms;              /* serving and batched forms (a project addition): SMs whose block
                                slots the one-block kernels leave to a lane for large graphs,
                                solved with the cooperative grid-wide kernels (2 blocks per SM);
                                0 = no lane (default), at most the device's SMs minus 16 */
  int lane_min_n;            /* graphs with at least this many vertices take the lane (if any) */
  int lane_slots;            /* large graphs solved at once on the lane, each on
                                lane_sms / lane_slots SMs; 1..lane_sms, default 1 */
} fiedler_options;

typedef struct {
  int64_t n;                 /* vertices, n >= 2 */
  int64_t nnz;               /* stored entries, < 2^31 */
  const int32_t *rowptr;     /* [n + 1] */
  const int32_t *col;        /* [nnz] */
  const void *w;             /* [nnz] float or double per w_dtype */
  int w_dtype;               /* FIEDLER_W_F32 or FIEDLER_W_F64 */
  int on_device;             /* 1: the three arrays are device pointers; 0: host pointers */
} fiedler_graph;

typedef struct {
  double lambda2;            /* Rayleigh quotient x^T L x / x^T x of the returned vector */
  double residual;           /* ||L x - lambda2 x|| / ||x|| */
  double ortho;              /* |1^T x| / (sqrt(n) ||x||) */
  int levels;                /* hierarchy depth, fine level included */
  int coarsest_n;            /* vertices on the coarsest level */
  int pi_iters_total;        /* power iterations summed over levels */
  int gs_sweeps_total;       /* Gauss-Seidel sweeps summed over levels */
  double *x;                 /* caller-owned output, length n, double; NULL = not wanted.
                                Unit 2-norm, orthogonal to 1, and sign-normalised so that the
                                entry of largest |x_i| (lowest index on ties) is positive. */
  int x_on_device;           /* 1: x is a device pointer; 0: host pointer */
  float ms;                  /* device time of the solve: CUDA events (fiedler_solve), or the
                                graph's own block time on the device timer (batched form) */
  long long bad_index;       /* first offending position when status == FIEDLER_EINVAL, else -1 */
  fiedler_status status;     /* same value as returned */
  int refine_iters;          /* Krylov matvecs on the finest level (0 with FIEDLER_REFINE_NONE) */
} fiedler_result;

typedef struct fiedler_plan fiedler_plan;

/* Fills opts with the defaults: FP32_FP64RED, coarse_max_n 25, max_levels 30,
 * stall_ratio 0.9, gs_sweeps 2, pi_max_iters 10000, pi_max_iters_coarsest
 * 100000, pi_cos_tol 1e-6, resid_tol 0, hashed ties, seed 20160214,
 * validate 1, tail_max_n 4096, tail_max_nnz 32768, barrier_timeout_ms 5000, fault_inject 0,
 * hbm_budget_bytes 0 (16 GiB), max_batch 1024, queue_budget_bytes 0 (8 GiB),
 * batch_threads 0, refine NONE, refine_max_iters 5000, refine_tol 1e-4,
 * lanczos_basis 24, hec_mode DOMINANT, refine_precond VCYCLE, lane_sms 0,
 * lane_min_n 200000, lane_slots 1. */
void fiedler_options_default(fiedler_options *opts);

/* Creates a plan on the current CUDA device.  opts may be NULL (defaults);
 * cuda_stream is a cudaStream_t on which every solve is ordered, or NULL for a
 * stream the plan creates.  Errors: EINVAL (bad option), ECUDA, ENOMEM. */
fiedler_status fiedler_plan_create(const fiedler_options *opts, void *cuda_stream, fiedler_plan **out);

/* Blocking solve of one graph (Alg. 3 + power iteration + Rayleigh quotient).
 * On return the result fields are filled, and result->x (if non-NULL) holds the
 * Fiedler vector.  The hierarchy of the last solve stays readable through
 * fiedler_plan_level_info / fiedler_plan_copy_level until the next solve.
 * Errors: EINVAL (bad CSR, reported with bad_index), EDISCONNECTED, ENOMEM,
 * ENOTSUP (nnz >= 2^31, more colours than supported), ETIMEOUT, ECUDA,
 * EDEGENERATE; ENOTCONVERGED still fills the result. */
fiedler_status fiedler_solve(fiedler_plan *plan, const fiedler_graph *graph, fiedler_result *result);

/* Batched form (a project addition): solves `count` independent graphs in one
 * persistent launch (each graph by one thread block of batch_threads threads
 * running every level of its hierarchy; blocks take the next graph, largest
 * first, when they finish one).  results[i] is filled as by fiedler_solve
 * (results[i].x / x_on_device give the output buffer, may be NULL; ms is the
 * graph's own device time); a graph's result does not depend on the other
 * graphs of the batch.  Returns FIEDLER_OK if the batch ran (per-graph outcomes
 * in results[i].status), or the error that stopped it. */
fiedler_status fiedler_solve_batch(fiedler_plan *plan, const fiedler_graph *graphs, int count,
                                   fiedler_result *results);

/* Serving form (continuous batching; a project addition): fiedler_batch_submit
 * copies the graph (host or device) into plan-owned memory, queues it and
 * returns a ticket at once; it returns FIEDLER_EAGAIN without queueing when
 * the copies held by earlier tickets (until they are polled) would exceed
 * queue_budget_bytes, or when the device has no memory left for the copy
 * while earlier tickets hold some, so the caller can wait for completions and
 * submit again (back-pressure; ENOMEM only when no other ticket holds
 * memory).  A scheduler thread admits queued tickets while the device
 * memory of the tickets in flight (state, hierarchy arena, scratch) stays
 * within hbm_budget_bytes, at most max_batch per round, and publishes them to
 * a persistent kernel whose resident blocks (one graph each, as in the batched
 * form, batch_threads per block) take them in order and finish each one
 * independently: a ticket admitted while others are on the GPU starts as soon
 * as a block is free, and a finished ticket returns its memory at once.
 * Thread-safe against fiedler_poll / fiedler_cancel.  Serving launches add
 * only the blocks that unfinished tickets lack and leave the block slots of
 * two SMs free, so copies and small kernels of other streams keep running;
 * a plan's fiedler_solve (a cooperative launch over every SM) should still
 * not run at the same time on the same device. */
fiedler_status fiedler_batch_submit(fiedler_plan *plan, const fiedler_graph *graph, uint64_t *ticket);

/* Waits up to timeout_ms (0 = do not wait, < 0 = wait forever) for a ticket.
 * Returns EAGAIN while it is in flight; otherwise the solve's status with
 * result filled as by fiedler_solve (result->x must have room for n doubles,
 * host or device per x_on_device).  A finished ticket is forgotten after a
 * successful poll. */
fiedler_status fiedler_poll(fiedler_plan *plan, uint64_t ticket, int timeout_ms, fiedler_result *result);

/* Lists up to `max` tickets that finished since the last call (*count of them
 * written to tickets[]), waiting up to timeout_ms (0 = do not wait, < 0 = wait
 * forever) for at least one; EAGAIN if none.  Each is then collected with
 * fiedler_poll (timeout 0), in any order: a server answers requests as they
 * complete instead of waiting on the oldest. */
fiedler_status fiedler_poll_any(fiedler_plan *plan, uint64_t *tickets, int max, int timeout_ms, int *count);

/* Cancels a queued ticket (ECANCELED on its next poll); a ticket already on
 * the GPU completes normally.  EINVAL for unknown tickets. */
fiedler_status fiedler_cancel(fiedler_plan *plan, uint64_t ticket);

/* Releases the plan, its stream (if owned) and all its device memory. */
void fiedler_plan_destroy(fiedler_plan *plan);

/* Static English description of a status. */
const char *fiedler_status_str(fiedler_status status);

/* ---- spectral partitioning ---------------------------------------------- */

typedef struct {
  int parts;                 /* parts produced (fewer than asked only when every part left is a
                                single vertex) */
  int solves;                /* Fiedler solves run (one per split) */
  int component_splits;      /* splits made along connected components (disconnected parts) */
  float ms;                  /* wall time of the call */
} fiedler_partition_info;

/* Spectral partitioning by recursive Fiedler bisection, the application the
 * paper's Introduction names (partitioning a graph by its Fiedler vector; a
 * project addition in this form).  Every vertex starts in part 0; until
 * `parts` parts exist, the part with the most vertices (lowest part id on
 * ties) is split: its induced subgraph is extracted on the device and solved
 * with the plan's options, and its vertices with x_i < 0 (x sign-normalised as
 * fiedler_result.x) form the new part, numbered in order of creation.  A part
 * whose subgraph is disconnected is split along its components instead: the
 * component of its lowest vertex stays, the rest forms the new part.
 *  - graph: host or device CSR as for fiedler_solve.
 *  - labels: n int32 (host, or device if labels_on_device), the part of every
 *    vertex on return.  info may be NULL.
 * Errors: those of fiedler_solve for the first split that fails; EINVAL for
 * parts < 1.  The plan's last-solve introspection then describes the last
 * split's subgraph. */
fiedler_status fiedler_partition(fiedler_plan *plan, const fiedler_graph *graph, int parts, int32_t *labels,
                                 int labels_on_device, fiedler_partition_info *info);

/* ---- introspection of the last solve (tests, profiling) ---------------- */

typedef struct {
  int64_t n, nnz;            /* level size (setup operator, self-loops dropped) */
  int nc;                    /* vertices of the next level (0 on the coarsest) */
  int ncolors;               /* colour classes used by the multicolour Gauss-Seidel */
  int match_rounds;          /* handshake rounds of the heavy-edge matching */
  int color_rounds;          /* Jones-Plassmann rounds */
  int gs_sweeps;             /* Gauss-Seidel sweeps kept on this level */
  int pi_iters;              /* power iterations on this level */
  double sigma;              /* shift: 2 max_i d_i */
  double last_cos;           /* (u^k, u^{k-1}) of the last power iteration */
  float phase_ms[16];        /* device time spent on this level per phase, in the order of
                                fiedler_profile.phase_name (device timer) */
  int refine_iters;          /* Krylov matvecs on this level (finest level only) */
} fiedler_level_info;

/* Number of levels of the last solve (0 before any solve). */
int fiedler_plan_num_levels(const fiedler_plan *plan);

/* Sizes and counters of level l of the last solve.  EINVAL if l is out of range. */
fiedler_status fiedler_plan_level_info(const fiedler_plan *plan, int level, fiedler_level_info *info);

/* Copies level l of the last solve to HOST arrays in the graph's own vertex
 * numbering (any pointer may be NULL): the Laplacian's off-diagonal part as
 * CSR (rowptr[n+1], col[nnz], w[nnz] as double), its diagonal d[n], the
 * aggregate map agg[n] to level l+1 (left untouched on the coarsest level),
 * the matching mate[n] (-1 = unmatched) and the colour of every vertex. */
fiedler_status fiedler_plan_copy_level(const fiedler_plan *plan, int level, int32_t *rowptr, int32_t *col,
                                       double *w, double *d, int32_t *agg, int32_t *mate, int32_t *color);

typedef struct {
  uint64_t kernel_launches;  /* kernels launched by the last solve */
  int n_kernels;             /* entries used in the arrays below */
  const char *kernel_name[4];
  int kernel_launches_by[4]; /* launches of each kernel in the last solve */
  float kernel_ms[4];        /* CUDA-event time of each kernel in the last solve (profiling on) */
  double kernel_bytes[4];    /* algorithmic bytes moved by each kernel in the last solve */
  int n_phases;
  const char *phase_name[16];
  double phase_ms[2][16];    /* device-timer time per phase, [0] grid-wide kernel, [1] one-block kernel */
  double phase_bytes[2][16]; /* algorithmic bytes per phase, same split */
} fiedler_profile;

typedef struct {
  uint64_t submitted, completed, batches;  /* serving counters since plan creation */
  double p50_ms, p99_ms, mean_ms;           /* ticket latency, submit to completion */
  double mean_batch;                        /* tickets per batched launch */
  size_t peak_inflight_bytes;               /* most device memory held by in-flight tickets */
  uint64_t launches;                        /* serving kernel launches */
  double block_seconds;                     /* device time of the finished tickets' solves, summed */
  double mean_inflight;                     /* unfinished published tickets, averaged over scheduler rounds */
  double mean_blocks;                       /* serving blocks alive, averaged the same way */
} fiedler_serving_stats;

/* Counters of the serving form. */
fiedler_status fiedler_plan_serving_stats(const fiedler_plan *plan, fiedler_serving_stats *out);

typedef struct {
  int batch_threads;         /* block size chosen for this plan's batched and served launches */
  float batch_ms[3];         /* CUDA-event time of the (repeated) sample batch with 512, 256
                                and 128 threads per graph (0 = not run).  A batch's time is set
                                both by its total work and by its largest graphs, so the sample
                                should look like the batches to come (a share of one, say) */
} fiedler_tuning;

/* Autotuner of the batched form (a project addition; the paper has none):
 * solves the `count` sample graphs, repeated until every block size has at
 * least two graphs per resident block (or, for large graphs, until their
 * memory would pass hbm_budget_bytes), as one batch with each block size
 * (512, 256 and 128 threads per graph, i.e. 1, 2 and 4 graphs resident per
 * SM), keeps the fastest for every later fiedler_solve_batch and serving
 * launch of this plan, and reports the timings of the repeated sample.  Results depend on the block size only
 * through the rounding of block-wide sums, so a graph gives the same result in
 * any batch of a tuned plan; the sample results are discarded.  Returns EINVAL
 * for an empty sample or a plan created with a fixed batch_threads. */
fiedler_status fiedler_plan_autotune(fiedler_plan *plan, const fiedler_graph *graphs, int count,
                                     fiedler_tuning *out);

/* 1: record CUDA events around every kernel of the following solves. */
fiedler_status fiedler_plan_set_profiling(fiedler_plan *plan, int on);

/* Counters of the last solve. */
fiedler_status fiedler_plan_get_profile(const fiedler_plan *plan, fiedler_profile *out);

/* ---- solve without allocation ------------------------------------------ */

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory (code running inside a memory pool or
 * cap owned by someone else, plug-ins that must not grow the device
 * footprint after start-up, latency-critical paths where allocation is
 * forbidden).  It solves one graph like fiedler_solve, but all its working
 * memory (solve state, hierarchy, scratch) is one fixed 16 MiB device array
 * inside the library, which every GPU that loads the library holds until the
 * process exits.  It calls no cudaMalloc / cudaFree and no allocating library
 * routine, and needs no plan.
 *  - graph: device-resident inputs (on_device = 1), else EINVAL.
 *  - x: device output of n doubles (may be NULL).  opts may be NULL.
 *  - cuda_stream: stream the work is ordered on (NULL = legacy default stream);
 *    the call returns after that work has finished.
 *  - Size limit: graphs whose hierarchy cannot fit the array (roughly beyond
 *    80k vertices / 300k stored entries) are refused with FIEDLER_ENOTSUP
 *    before any work is queued; a hierarchy that still outgrows it at run time
 *    also returns FIEDLER_ENOTSUP.
 *  - Every call reuses the same array and overwrites the previous call's
 *    contents (the state is rewritten at the start of each call), so calls must
 *    not overlap on the GPU: the library serialises callers within a process.
 *  - Not for stream capture: every call reads host memory and ends in a
 *    synchronisation of cuda_stream, so a call on a stream that is capturing
 *    returns FIEDLER_EINVAL without queueing work.
 *  - The first call on each device looks up the array's device address with
 *    cudaGetSymbolAddress (with that device current).
 *  - Options are checked as fiedler_plan_create checks them; a refused call
 *    sets result->status (and bad_index = -1) when result is given.
 *  - Every level runs in the one-block engine, so results equal those of
 *    fiedler_solve with tail_max_n at least n and tail_max_nnz at least nnz. */
fiedler_status fiedler_solve_noalloc(const fiedler_options *opts, const fiedler_graph *graph, double *x,
                                     void *cuda_stream, fiedler_result *result);

#ifdef __cplusplus
}
#endif
#endif /* FIEDLER_H */
