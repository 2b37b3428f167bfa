// fz_state.h -- device-resident solve state shared by the host driver and the
// engine kernels.  One State lives in device memory per plan; the host writes
// its header before a solve and reads it back afterwards.  Level descriptors
// are filled on the device as the hierarchy is built (no host round trips).
#pragma once
#include <stdint.h>

namespace fz {

constexpr int kMaxLevels = 32;
constexpr int kMaxBlocks = 2048;   // grid-wide kernel blocks (partials buffer size)
constexpr int kMaxColors = 1024;   // colour classes per level supported by the reorder
constexpr int kCtaThreads = 512;   // one-block kernel
constexpr int kMaxThreads = 1024;  // largest block of any engine kernel (shared worklists)
constexpr int kGridThreads = 1024;  // grid-wide kernel block size (one block per SM)
// tiny levels (n <= kTinyN and nnz <= kTinyNnz): always in the one-block
// engine, smoothed by one warp, values in FP64 in both forms
constexpr int kTinyN = 256;
constexpr int kTinyNnz = 4096;
constexpr int kMaxBasis = 64;      // Lanczos basis vectors per restart cycle, at most

enum Phase {
  PH_INGEST = 0, PH_COLOR, PH_REORDER, PH_MATCH, PH_AGG, PH_GALERKIN,
  PH_COARSEST, PH_PROLONG, PH_GS, PH_PI, PH_FINAL, PH_REFINE, PH_COUNT
};

// internal status codes; the host maps them to fiedler_status
enum : int {
  ST_OK = 0, ST_EINVAL = -1, ST_ENOMEM = -2, ST_EDISC = -3, ST_ENOTCONV = -4, ST_ETIMEOUT = -5,
  ST_EDEGEN = -8, ST_ENOTSUP = -9, ST_ARENA = -100, ST_SCRATCH = -101
};

struct Opts {
  int precision;
  int coarse_max_n;
  int max_levels;
  int gs_sweeps;
  int pi_max_iters;
  int pi_max_iters_coarsest;
  int tie_rule;
  int validate;
  int tail_max_n;
  int tail_max_nnz;
  int fault_inject;
  int refine;                // 0: paper (power iteration); 1: LOBPCG; 2: Lanczos (finest level)
  int refine_max_iters;
  int lanczos_basis;
  int hec_mode;              // 0: locally dominant matching; 1: Alg. 1's random-order greedy
  int refine_precond;        // LOBPCG preconditioner: 0 D^-1, 1 V-cycle of the hierarchy
  int pad_opt;
  double refine_tol;
  double stall_ratio;
  double pi_cos_tol;
  double resid_tol;
  double guard;              // annihilation guard of the deflated norm
  unsigned long long seed;
  unsigned long long barrier_timeout_ns;
};

struct Level {
  // setup operator in the graph's own numbering (off-diagonal CSR, FP64 or
  // the caller's float weights on the fine level), diagonal and shift
  int n, nnz;
  int *rowptr, *col;
  double *w64;
  float *w32;
  double *d;
  double sigma;
  // heavy-edge matching and aggregate map to the next level
  int *mate, *agg;
  int nc;
  // colouring; perm[k] = vertex at solve position k, iperm its inverse
  int *color, *colstart, *perm, *iperm;
  int ncolors;
  // solve operator in colour order (value type float or double)
  int *srowptr, *scol;
  void *sw;
  int *sagg;  // solve position on this level -> solve position on the next
  // iterate: x (or y) with a lazy affine map xhat = (x - mu) * s
  void *x, *y;
  double mu, s;
  // V-cycle preconditioner: members of each aggregate (graph numbering,
  // ascending; kept from the Galerkin step) and the level's right-hand side,
  // correction and residual vectors (value type of the level)
  int *mptr, *mem;
  void *vb, *ve, *vt;
  // counters
  int match_rounds, color_rounds, gs_sweeps, pi_iters, capped;
  int refine_iters;
  double last_cos;
};

constexpr int kDSum = 72;  // doubles per block partial of a floating-point grid sum (>= kMaxBasis + 1)

struct IRed {              // per-block partials of an integer grid reduction
  long long a, b;          // sums (prefix over lower blocks available for both)
  long long mx;            // maximum (also used for non-negative doubles by bit pattern)
};

struct State {
  int status;
  int setup_done;
  long long bad_index;
  int nlevels;
  int coarsest;
  int coarsest_solved;
  int solved;              // lowest level index whose vector is final
  int finalized;
  int refined;             // the finest level's Krylov refinement is done
  int capped;
  Opts opt;
  // input graph
  int n0, nnz0;
  const int *in_rowptr, *in_col;
  const void *in_w;
  int in_w_f64;
  int pad1;
  // device arenas (bump allocation, offsets advanced identically by every block)
  char *arena;
  unsigned long long arena_size, arena_off;
  char *scratch;
  unsigned long long scratch_size;
  double *xout;            // device output (n0 doubles), original numbering
  IRed *ipart;             // [2][kMaxBlocks] integer partials
  double *dpart;           // [2][kMaxBlocks][kDSum] floating-point partials
  long long *amax;         // [2][kMaxBlocks] argmax partials: (|x| bits, index) packed by the final pass
  int wl_cnt[4];           // worklist counters of the matching (rotating)
  int jp_cnt[4];           // worklist counters of the colouring (rotating)
  int col_max;             // largest colour of the level being coloured
  // results
  double lambda, residual, ortho;
  int pi_total, gs_total, refine_total, pad3;
  // grid barrier: one word whose top bit flips when every block has arrived;
  // failword = (barriers passed by the failing block << 32) | status code
  unsigned bar_word;
  int pad2;
  unsigned long long failword;
  // device-timer profile: [0] grid-wide kernel, [1] one-block kernel
  unsigned long long t_last;
  double phase_ns[2][PH_COUNT];
  double phase_bytes[2][PH_COUNT];
  double level_ns[kMaxLevels][PH_COUNT];  // device time per level and phase
  Level lv[kMaxLevels];
};

// Serving ring.  The host publishes ticket states item[k % kRing] for
// k < tail (device memory, written by copies on one stream: items before the
// tail); resident blocks of the serving kernel claim items through the
// device counter head and, once item k is finished, write done[k % kRing] =
// k + 1 into host-mapped memory.  The host keeps fewer than kRing items
// unfinished.
constexpr int kRing = 4096;
struct ServeRing {               // device memory
  unsigned long long tail;       // items published
  unsigned long long head;       // items claimed
  unsigned long long stop;       // 1: the kernel's blocks leave as soon as they are idle
  unsigned long long idle_ns;    // a block with no work for this long leaves
  State *item[kRing];
};
constexpr int kServeSlots = 1024;    // blocks of one serving launch, at most
constexpr int kExitRing = 1 << 16;  // exit flags of the most recent serving blocks
struct ServeDone {                   // host-mapped pinned memory
  unsigned long long done[kRing];
  // serving blocks are numbered across launches; block g writes
  // exited[g % kExitRing] = g + 1 when it leaves
  unsigned long long exited[kExitRing];
};

}  // namespace fz
