/*
 * fiedler_oracle.c -- plain, sequential, FP64 CPU reference of the Gauss-Seidel
 * cascadic multigrid (GSCMG) Fiedler-vector method of S. Gandhi, "Improvement of
 * the Cascadic Multigrid Algorithm with a Gauss Seidel Smoother to Efficiently
 * Compute the Fiedler Vector of a Graph Laplacian" (2015).
 *
 * TEST INFRASTRUCTURE.  This file is the oracle that the CUDA path is checked
 * against.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load it.  It shares no code, header, table or constant
 * generator with the CUDA library; it is written from the paper's definitions:
 *
 *   Def 2.1  graph Laplacian L = D - W (weighted degree on the diagonal)
 *   Def 2.2  Fiedler vector = eigenvector of the second smallest eigenvalue
 *   Alg. 1   heavy edge coarsening (HEC), setup phase
 *   Alg. 2   Gauss-Seidel G-S(A, b, X0, tol, N)
 *   Alg. 3   GSCMG: setup (L^{i+1} = I L^i I^T while n_i > 25), coarsest solve,
 *            cascadic refinement y^j = I^T y^{j+1}, y^j <- GS(L^j, y^j)
 *   Sec. 2   power iteration on a shifted ("modified") matrix, Rayleigh quotient
 *   Sec. 3   stopping tolerance (u^k, u^{k-1}) > 1 - 1e-6
 *
 * Readings of points where the paper is silent or garbled (each is listed in
 * the design notes of the repository):
 *   R1  degree = weighted degree sum_j w_ij; self-loops are dropped.
 *   R2  HEC has three modes: the paper's random-order greedy (hec_mode 2), and
 *       a deterministic heavy-edge matching under the strict edge order
 *       K(e) = (w desc, h(min,max) asc, min asc, max asc) computed either by
 *       handshake rounds (hec_mode 0) or by a greedy scan of the globally sorted
 *       edges (hec_mode 1); both give the same matching (locally dominant
 *       matching under a strict total order).  tie_rule 1 drops h.
 *       Unmatched vertices with neighbours join the aggregate of their best
 *       neighbour under K (the "else q(p(i)) = q(m)" branch of Alg. 1);
 *       isolated vertices are singletons.  Aggregate ids are the ranks of the
 *       aggregate leaders (min of a matched pair, or the singleton itself).
 *   R3  coarse weights are FP64 sums over the contributing fine entries in
 *       ascending (fine row, fine column) order; the coarse diagonal is the sum
 *       of the coarse row's off-diagonal weights in ascending column order.
 *   R4  coarsening stops when n <= coarse_max_n, at max_levels levels, or when
 *       a coarse level would have fewer than 2 vertices or more than
 *       stall_ratio * n vertices (that coarse level is then not built).
 *   R5  Gauss-Seidel acts on L x = 0 (b = 0), one full forward sweep per
 *       iteration, a fixed number of sweeps; since L is singular the constant
 *       vector is deflated and the iterate normalised after every sweep.  Order:
 *       lexicographic (gs_order 0) or colour classes ascending, ascending index
 *       within a class (gs_order 1).  A sweep whose deflated result has norm
 *       <= guard (2^-20; the input is a unit vector) is discarded and ends the
 *       smoothing on that level.  The guard sits above the rounding noise of a
 *       deflated norm taken as sum x^2 - (sum x)^2 / n in double, so that an
 *       implementation fusing the deflation into its reductions takes the same
 *       decision; it only fires when a sweep maps the iterate onto the constant
 *       vector (K_2, stars swept centre first).
 *   R6  after the Gauss-Seidel sweeps every level runs power iteration on
 *       sigma I - L, sigma = 2 max_i d_i (Gershgorin), with deflation and
 *       normalisation, until (u^k, u^{k-1}) > 1 - pi_cos_tol and (if
 *       resid_tol > 0) ||L u^{k-1} - rho u^{k-1}|| <= resid_tol * sigma.  A step
 *       whose deflated result has norm <= guard * sigma ends the iteration and
 *       keeps the previous vector.
 *   R7  colouring: greedy in decreasing priority (h(v), v); equal to the
 *       Jones-Plassmann rounds with that priority.
 *   R8  random start: x_i = uniform draw i of the splitmix64 stream of `seed`.
 *   R9  output sign: the entry of largest |x_i| (lowest index on ties) is >= 0.
 *   R11 randperm of Alg. 1 (hec_mode 2): the visiting order of level l is the
 *       ascending order of the keys splitmix64(seed + l, v), ties by v (a
 *       uniformly random order when the keys are distinct).
 *   R12 Krylov refinement of the finest level (refine 1 or 2; Sec. 4 names a
 *       Lanczos smoother as future work): with it on, the finest level skips
 *       its power iteration and, after its Gauss-Seidel sweeps, runs
 *       (1) LOBPCG (Knyazev 2001), one vector, on 1-perp with preconditioner
 *           D^-1: w = D^-1 (L x - theta x) with its mean removed, Rayleigh-Ritz
 *           on span{x, w, p} (columns scaled to unit norm; w, then p, dropped
 *           when its Cholesky pivot of the scaled Gram matrix is <= 1e-10),
 *           x and p = the w, p part of the Ritz vector, both normalised;
 *       (2) Lanczos with full reorthogonalisation (classical Gram-Schmidt,
 *           twice) on 1-perp, restarted from the smallest Ritz vector every
 *           lanczos_basis steps;
 *       until ||L x - theta x|| <= refine_tol * theta * ||x|| (LOBPCG: tested
 *       before every step; Lanczos: the Ritz estimate beta_m |s_m| at the end
 *       of a cycle), or refine_max_iters matvecs.  In exact arithmetic each
 *       Rayleigh-Ritz step lowers the Rayleigh quotient; a step that brings no
 *       new lowest value (rounding) restarts LOBPCG without p, and eight such
 *       steps in a row end the iteration: the rounding floor of the arithmetic
 *       (in float the residual stalls near 1e-3 theta on graphs of small
 *       lambda_2 while lambda_2 itself is already exact to ~1e-8).
 *   R13 LOBPCG's preconditioner (refine_precond; not in the paper): D^-1, or
 *       one V-cycle of the cascade's own hierarchy on L e = r: on level l, one
 *       forward Gauss-Seidel sweep from e = 0 (colour classes ascending), the
 *       residual r - L e summed over each aggregate (members in ascending
 *       index) as the next level's right-hand side, the next level's
 *       correction added to every member, one backward sweep (classes
 *       descending); on the coarsest level 20 forward sweeps from e = 0 and
 *       the mean removed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_EDISCONNECTED (-3)
#define ORC_EDEGENERATE (-8)

#define ORC_MAX_LEVELS 64

/* ------------------------------------------------------------------------ */
/* splitmix64 (S. Vigna): state += 0x9E3779B97F4A7C15, then the mix function. */

static uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* output k (k >= 0) of the splitmix64 stream seeded with s */
uint64_t oracle_splitmix64(uint64_t s, uint64_t k) {
  return orc_mix64(s + (k + 1) * 0x9E3779B97F4A7C15ULL);
}

static double orc_uniform(uint64_t s, uint64_t k) {
  return (double)(oracle_splitmix64(s, k) >> 11) * (1.0 / 9007199254740992.0);
}

/* tie-break hash of an edge {a, b}: first output of the stream seeded with
 * (min << 32 | max) */
static uint64_t orc_edge_hash(int a, int b) {
  uint64_t lo = (uint64_t)(a < b ? a : b), hi = (uint64_t)(a < b ? b : a);
  return oracle_splitmix64((lo << 32) | hi, 0);
}

static uint64_t orc_vertex_hash(int v) { return oracle_splitmix64((uint64_t)(uint32_t)v, 0); }

/* ------------------------------------------------------------------------ */
/* options and run state */

typedef struct {
  int coarse_max_n;          /* 25 (Alg. 3: while n_i > 25) */
  int max_levels;            /* 30 */
  double stall_ratio;        /* 0.9 */
  int hec_mode;              /* 0 handshake, 1 sorted greedy, 2 paper random order */
  int tie_rule;              /* 0 hashed, 1 index */
  int gs_order;              /* 0 lexicographic, 1 colour classes */
  int gs_sweeps;             /* sweeps per level */
  int pi_max_iters;          /* power-iteration cap on non-coarsest levels */
  int pi_max_iters_coarsest; /* cap on the coarsest level */
  double pi_cos_tol;         /* 1e-6 (Sec. 3) */
  double resid_tol;          /* 0 = paper stop rule only */
  double guard;              /* annihilation guard, 2^-20 */
  uint64_t seed;             /* random start on the coarsest level */
  int coarsest_dense;        /* 1 = coarsest eigenvector by dense Jacobi */
  int refine;                /* 0 none (paper), 1 LOBPCG, 2 Lanczos on the finest level (R12) */
  int refine_max_iters;      /* matvec cap of the refinement */
  double refine_tol;         /* stop: ||L x - theta x|| <= refine_tol * theta * ||x|| */
  int lanczos_basis;         /* Lanczos steps per restart cycle */
  int refine_forced;         /* >= 0: run exactly this many matvecs (replay); -1: stop rule */
  int refine_precond;        /* LOBPCG preconditioner: 0 D^-1, 1 one V-cycle of the hierarchy (R13) */
} oracle_opts;

typedef struct {
  int n;
  long long nnz;
  int *rowptr, *col;
  double *w, *d;
} orc_lap;

typedef struct {
  orc_lap L;
  int *agg; /* to the next level; NULL on the coarsest */
  int nc;
  int *mate;
  int match_rounds;
  int *color;
  int ncolors;
  int color_rounds;
  double sigma;
  int gs_sweeps_done;
  int pi_iters;
  double last_cos;
  int refine_iters;
  int capped; /* a power-iteration or refinement cap was reached */
  double *x; /* level result after smoothing */
} orc_level;

typedef struct oracle_run {
  int status;
  int nlevels;
  orc_level lv[ORC_MAX_LEVELS];
  int n;
  double *x;
  double lambda, residual, ortho;
  long long bad_index;
} oracle_run;

static void lap_free(orc_lap *L) {
  free(L->rowptr);
  free(L->col);
  free(L->w);
  free(L->d);
  memset(L, 0, sizeof(*L));
}

static void level_free(orc_level *l) {
  lap_free(&l->L);
  free(l->agg);
  free(l->mate);
  free(l->color);
  free(l->x);
  memset(l, 0, sizeof(*l));
}

oracle_run *oracle_run_create(void) { return (oracle_run *)calloc(1, sizeof(oracle_run)); }

static void run_clear(oracle_run *r) {
  for (int i = 0; i < r->nlevels; i++) level_free(&r->lv[i]);
  free(r->x);
  memset(r, 0, sizeof(*r));
}

void oracle_run_destroy(oracle_run *r) {
  if (!r) return;
  run_clear(r);
  free(r);
}

void oracle_default_opts(oracle_opts *o) {
  o->coarse_max_n = 25;
  o->max_levels = 30;
  o->stall_ratio = 0.9;
  o->hec_mode = 0;
  o->tie_rule = 0;
  o->gs_order = 1;
  o->gs_sweeps = 2;
  o->pi_max_iters = 10000;
  o->pi_max_iters_coarsest = 100000;
  o->pi_cos_tol = 1e-6;
  o->resid_tol = 0.0;
  o->guard = 9.5367431640625e-07; /* 2^-20 */
  o->seed = 20160214ULL;
  o->coarsest_dense = 0;
  o->refine = 0;
  o->refine_max_iters = 5000;
  o->refine_tol = 1e-4;
  o->lanczos_basis = 24;
  o->refine_forced = -1;
  o->refine_precond = 1;
}

/* ------------------------------------------------------------------------ */
/* A1: Laplacian ingest (Def 2.1).  Input: symmetric adjacency CSR with column
 * indices strictly ascending in each row and positive finite off-diagonal
 * weights; self-loops (diagonal entries) are dropped.  d_i = sum_j w_ij
 * accumulated in ascending column order. */

static int lap_ingest(int n, long long nnz, const int *rowptr, const int *col, const double *w,
                      orc_lap *out, long long *bad) {
  *bad = -1;
  if (n < 2 || nnz < 0 || !rowptr) { *bad = 0; return ORC_EINVAL; }
  if (rowptr[0] != 0 || (long long)rowptr[n] != nnz) { *bad = 0; return ORC_EINVAL; }
  for (int i = 0; i < n; i++)
    if (rowptr[i + 1] < rowptr[i]) { *bad = i; return ORC_EINVAL; }
  for (int i = 0; i < n; i++) {
    for (int e = rowptr[i]; e < rowptr[i + 1]; e++) {
      int j = col[e];
      if (j < 0 || j >= n) { *bad = e; return ORC_EINVAL; }
      if (e > rowptr[i] && col[e - 1] >= j) { *bad = e; return ORC_EINVAL; }
      if (!isfinite(w[e])) { *bad = e; return ORC_EINVAL; }
      if (j == i) continue;
      if (!(w[e] > 0.0)) { *bad = e; return ORC_EINVAL; }
      /* symmetric partner (j, i) with the same weight */
      int lo = rowptr[j], hi = rowptr[j + 1] - 1, found = -1;
      while (lo <= hi) {
        int mid = lo + (hi - lo) / 2;
        if (col[mid] == i) { found = mid; break; }
        if (col[mid] < i) lo = mid + 1; else hi = mid - 1;
      }
      if (found < 0 || w[found] != w[e]) { *bad = e; return ORC_EINVAL; }
    }
  }
  long long m = 0;
  for (int i = 0; i < n; i++)
    for (int e = rowptr[i]; e < rowptr[i + 1]; e++) m += (col[e] != i);
  out->n = n;
  out->nnz = m;
  out->rowptr = (int *)malloc(sizeof(int) * (size_t)(n + 1));
  out->col = (int *)malloc(sizeof(int) * (size_t)(m ? m : 1));
  out->w = (double *)malloc(sizeof(double) * (size_t)(m ? m : 1));
  out->d = (double *)malloc(sizeof(double) * (size_t)n);
  if (!out->rowptr || !out->col || !out->w || !out->d) return ORC_ENOMEM;
  long long k = 0;
  out->rowptr[0] = 0;
  for (int i = 0; i < n; i++) {
    double di = 0.0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; e++) {
      if (col[e] == i) continue;
      out->col[k] = col[e];
      out->w[k] = w[e];
      di += w[e];
      k++;
    }
    out->rowptr[i + 1] = (int)k;
    out->d[i] = di;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Deterministic heavy-edge order K (reading R2): returns 1 if edge {a1,b1}
 * with weight w1 precedes edge {a2,b2} with weight w2. */

static int key_precedes(double w1, int a1, int b1, double w2, int a2, int b2, int tie_rule) {
  if (w1 != w2) return w1 > w2;
  int lo1 = a1 < b1 ? a1 : b1, hi1 = a1 < b1 ? b1 : a1;
  int lo2 = a2 < b2 ? a2 : b2, hi2 = a2 < b2 ? b2 : a2;
  if (tie_rule == 0) {
    uint64_t h1 = orc_edge_hash(lo1, hi1), h2 = orc_edge_hash(lo2, hi2);
    if (h1 != h2) return h1 < h2;
  }
  if (lo1 != lo2) return lo1 < lo2;
  return hi1 < hi2;
}

/* best neighbour of u under K among neighbours v with (only_free ? mate[v] < 0 : any) */
static int best_neighbour(const orc_lap *L, int u, const int *mate, int only_free, int tie_rule) {
  int best = -1;
  double bw = 0.0;
  for (int e = L->rowptr[u]; e < L->rowptr[u + 1]; e++) {
    int v = L->col[e];
    if (only_free && mate[v] >= 0) continue;
    if (best < 0 || key_precedes(L->w[e], u, v, bw, u, best, tie_rule)) {
      best = v;
      bw = L->w[e];
    }
  }
  return best;
}

/* Handshake rounds: every unmatched vertex points at its best unmatched
 * neighbour; mutual pointers become matched pairs; repeat until no unmatched
 * vertex has an unmatched neighbour. */
static int match_handshake(const orc_lap *L, int tie_rule, int *mate, int *rounds) {
  int n = L->n;
  int *cand = (int *)malloc(sizeof(int) * (size_t)n);
  if (!cand) return ORC_ENOMEM;
  for (int i = 0; i < n; i++) mate[i] = -1;
  int r = 0;
  for (;;) {
    int any = 0;
    for (int u = 0; u < n; u++) {
      cand[u] = -1;
      if (mate[u] >= 0) continue;
      cand[u] = best_neighbour(L, u, mate, 1, tie_rule);
      if (cand[u] >= 0) any = 1;
    }
    if (!any) break;
    r++;
    for (int u = 0; u < n; u++) {
      int v = cand[u];
      if (v >= 0 && cand[v] == u) mate[u] = v;
    }
  }
  free(cand);
  *rounds = r;
  return ORC_OK;
}

typedef struct {
  double w;
  int a, b;
  int tie_rule;
} orc_edge;

static int edge_cmp(const void *p, const void *q) {
  const orc_edge *x = (const orc_edge *)p, *y = (const orc_edge *)q;
  if (key_precedes(x->w, x->a, x->b, y->w, y->a, y->b, x->tie_rule)) return -1;
  if (key_precedes(y->w, y->a, y->b, x->w, x->a, x->b, x->tie_rule)) return 1;
  return 0;
}

/* Greedy scan of all edges sorted by K: take an edge when both ends are free. */
static int match_sorted_greedy(const orc_lap *L, int tie_rule, int *mate) {
  int n = L->n;
  long long m = L->nnz / 2;
  orc_edge *E = (orc_edge *)malloc(sizeof(orc_edge) * (size_t)(m ? m : 1));
  if (!E) return ORC_ENOMEM;
  long long k = 0;
  for (int i = 0; i < n; i++)
    for (int e = L->rowptr[i]; e < L->rowptr[i + 1]; e++)
      if (L->col[e] > i) {
        E[k].w = L->w[e];
        E[k].a = i;
        E[k].b = L->col[e];
        E[k].tie_rule = tie_rule;
        k++;
      }
  qsort(E, (size_t)k, sizeof(orc_edge), edge_cmp);
  for (int i = 0; i < n; i++) mate[i] = -1;
  for (long long t = 0; t < k; t++)
    if (mate[E[t].a] < 0 && mate[E[t].b] < 0) {
      mate[E[t].a] = E[t].b;
      mate[E[t].b] = E[t].a;
    }
  free(E);
  return ORC_OK;
}

/* Aggregates from a maximal matching (reading R2). Returns the number of
 * aggregates, or a negative status. */
static int aggregate_from_matching(const orc_lap *L, const int *mate, int tie_rule, int *agg) {
  int n = L->n;
  int *id = (int *)malloc(sizeof(int) * (size_t)n);
  if (!id) return ORC_ENOMEM;
  int nc = 0;
  for (int u = 0; u < n; u++) {
    int deg = L->rowptr[u + 1] - L->rowptr[u];
    int leader = (mate[u] >= 0) ? (u < mate[u]) : (deg == 0);
    id[u] = leader ? nc++ : -1;
  }
  for (int u = 0; u < n; u++) {
    if (mate[u] >= 0) {
      agg[u] = id[u < mate[u] ? u : mate[u]];
    } else if (L->rowptr[u + 1] == L->rowptr[u]) {
      agg[u] = id[u];
    } else {
      int v = best_neighbour(L, u, mate, 0, tie_rule);
      if (mate[v] < 0) { free(id); return ORC_EINVAL; } /* matching not maximal */
      agg[u] = id[v < mate[v] ? v : mate[v]];
    }
  }
  free(id);
  return nc;
}

/* Alg. 1 as printed: random order p; for each unaggregated p(i), m = argmin of
 * column p(i) of L (the heaviest neighbour, lowest index on ties); pair with m
 * if m is unaggregated, else join m's aggregate.  A vertex without neighbours
 * becomes a singleton. `perm` may be given; otherwise the vertices sorted by
 * the keys splitmix64(seed, v), ties by v (reading R11). */
typedef struct {
  uint64_t key;
  int v;
} orc_keyv;

static int keyv_cmp(const void *p, const void *q) {
  const orc_keyv *a = (const orc_keyv *)p, *b = (const orc_keyv *)q;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->v < b->v ? -1 : (a->v > b->v);
}

static int hec_paper(const orc_lap *L, uint64_t seed, const int *perm_in, int *agg) {
  int n = L->n;
  int *p = (int *)malloc(sizeof(int) * (size_t)n);
  int *q = (int *)malloc(sizeof(int) * (size_t)n);
  if (!p || !q) { free(p); free(q); return ORC_ENOMEM; }
  if (perm_in) {
    memcpy(p, perm_in, sizeof(int) * (size_t)n);
  } else {
    orc_keyv *kv = (orc_keyv *)malloc(sizeof(orc_keyv) * (size_t)n);
    if (!kv) { free(p); free(q); return ORC_ENOMEM; }
    for (int i = 0; i < n; i++) {
      kv[i].key = oracle_splitmix64(seed, (uint64_t)i);
      kv[i].v = i;
    }
    qsort(kv, (size_t)n, sizeof(orc_keyv), keyv_cmp);
    for (int i = 0; i < n; i++) p[i] = kv[i].v;
    free(kv);
  }
  for (int i = 0; i < n; i++) q[i] = 0;
  int c = 0;
  for (int i = 0; i < n; i++) {
    int u = p[i];
    if (q[u] != 0) continue;
    /* argmin over column u of L: off-diagonal entries are -w_vu */
    int m = -1;
    double best = 0.0;
    for (int e = L->rowptr[u]; e < L->rowptr[u + 1]; e++) {
      double val = -L->w[e];
      if (m < 0 || val < best) { best = val; m = L->col[e]; }
    }
    if (m < 0) { q[u] = ++c; continue; }
    if (q[m] == 0) { c++; q[m] = c; q[u] = c; }
    else q[u] = q[m];
  }
  for (int i = 0; i < n; i++) agg[i] = q[i] - 1;
  free(p);
  free(q);
  return c;
}

/* ------------------------------------------------------------------------ */
/* Galerkin coarse operator L^{i+1} = I L^i I^T (Alg. 3, setup), reading R3. */

typedef struct {
  int I, J;
  long long order;
  double w;
} orc_trip;

static int trip_cmp(const void *p, const void *q) {
  const orc_trip *x = (const orc_trip *)p, *y = (const orc_trip *)q;
  if (x->I != y->I) return x->I < y->I ? -1 : 1;
  if (x->J != y->J) return x->J < y->J ? -1 : 1;
  if (x->order != y->order) return x->order < y->order ? -1 : 1;
  return 0;
}

static int galerkin(const orc_lap *F, const int *agg, int nc, orc_lap *C) {
  long long m = 0;
  for (int i = 0; i < F->n; i++)
    for (int e = F->rowptr[i]; e < F->rowptr[i + 1]; e++) m += agg[F->col[e]] != agg[i];
  orc_trip *T = (orc_trip *)malloc(sizeof(orc_trip) * (size_t)(m ? m : 1));
  if (!T) return ORC_ENOMEM;
  long long k = 0;
  for (int i = 0; i < F->n; i++)
    for (int e = F->rowptr[i]; e < F->rowptr[i + 1]; e++) {
      int I = agg[i], J = agg[F->col[e]];
      if (I == J) continue;
      T[k].I = I; T[k].J = J; T[k].order = e; T[k].w = F->w[e];
      k++;
    }
  qsort(T, (size_t)k, sizeof(orc_trip), trip_cmp);
  long long groups = 0;
  for (long long t = 0; t < k; t++)
    if (t == 0 || T[t].I != T[t - 1].I || T[t].J != T[t - 1].J) groups++;
  C->n = nc;
  C->nnz = groups;
  C->rowptr = (int *)calloc((size_t)nc + 1, sizeof(int));
  C->col = (int *)malloc(sizeof(int) * (size_t)(groups ? groups : 1));
  C->w = (double *)malloc(sizeof(double) * (size_t)(groups ? groups : 1));
  C->d = (double *)calloc((size_t)nc, sizeof(double));
  if (!C->rowptr || !C->col || !C->w || !C->d) { free(T); return ORC_ENOMEM; }
  long long g = -1;
  for (long long t = 0; t < k; t++) {
    if (t == 0 || T[t].I != T[t - 1].I || T[t].J != T[t - 1].J) {
      g++;
      C->col[g] = T[t].J;
      C->w[g] = T[t].w;
      C->rowptr[T[t].I + 1]++;
    } else {
      C->w[g] += T[t].w;
    }
  }
  for (int I = 0; I < nc; I++) C->rowptr[I + 1] += C->rowptr[I];
  for (int I = 0; I < nc; I++) {
    double s = 0.0;
    for (int e = C->rowptr[I]; e < C->rowptr[I + 1]; e++) s += C->w[e];
    C->d[I] = s;
  }
  free(T);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Colouring (reading R7): priority of v is (h(v), v); higher goes first. */

static int prio_higher(int a, int b) {
  uint64_t ha = orc_vertex_hash(a), hb = orc_vertex_hash(b);
  if (ha != hb) return ha > hb;
  return a > b;
}

static int smallest_free_colour(const orc_lap *L, int v, const int *color, const int *stamp, int round,
                                unsigned char *used, int cap) {
  int deg = L->rowptr[v + 1] - L->rowptr[v];
  int lim = deg + 1 < cap ? deg + 1 : cap;
  memset(used, 0, (size_t)lim);
  for (int e = L->rowptr[v]; e < L->rowptr[v + 1]; e++) {
    int u = L->col[e];
    int coloured = stamp ? (stamp[u] < round) : (color[u] >= 0);
    if (coloured && color[u] < lim) used[color[u]] = 1;
  }
  int c = 0;
  while (c < lim && used[c]) c++;
  return c;
}

typedef struct {
  uint64_t h;
  int v;
} orc_prio;

static int prio_cmp_desc(const void *p, const void *q) {
  const orc_prio *x = (const orc_prio *)p, *y = (const orc_prio *)q;
  if (x->h != y->h) return x->h > y->h ? -1 : 1;
  return x->v > y->v ? -1 : (x->v < y->v ? 1 : 0);
}

/* greedy colouring in decreasing priority order; returns the colour count */
static int color_greedy(const orc_lap *L, int *color) {
  int n = L->n, maxdeg = 0;
  orc_prio *P = (orc_prio *)malloc(sizeof(orc_prio) * (size_t)n);
  if (!P) return ORC_ENOMEM;
  for (int v = 0; v < n; v++) {
    P[v].h = orc_vertex_hash(v);
    P[v].v = v;
    color[v] = -1;
    int deg = L->rowptr[v + 1] - L->rowptr[v];
    if (deg > maxdeg) maxdeg = deg;
  }
  qsort(P, (size_t)n, sizeof(orc_prio), prio_cmp_desc);
  unsigned char *used = (unsigned char *)malloc((size_t)maxdeg + 2);
  if (!used) { free(P); return ORC_ENOMEM; }
  int nc = 0;
  for (int t = 0; t < n; t++) {
    int v = P[t].v;
    color[v] = smallest_free_colour(L, v, color, NULL, 0, used, maxdeg + 2);
    if (color[v] + 1 > nc) nc = color[v] + 1;
  }
  free(used);
  free(P);
  return nc;
}

/* Jones-Plassmann rounds: an uncoloured vertex whose priority beats all
 * neighbours still uncoloured at the start of the round takes the smallest
 * colour unused by neighbours coloured in earlier rounds. */
static int color_jp(const orc_lap *L, int *color, int *rounds) {
  int n = L->n, maxdeg = 0;
  int *stamp = (int *)malloc(sizeof(int) * (size_t)n);
  if (!stamp) return ORC_ENOMEM;
  for (int v = 0; v < n; v++) {
    stamp[v] = 0x7fffffff;
    color[v] = -1;
    int deg = L->rowptr[v + 1] - L->rowptr[v];
    if (deg > maxdeg) maxdeg = deg;
  }
  unsigned char *used = (unsigned char *)malloc((size_t)maxdeg + 2);
  if (!used) { free(stamp); return ORC_ENOMEM; }
  int left = n, r = 0, nc = 0;
  while (left > 0) {
    for (int v = 0; v < n; v++) {
      if (stamp[v] < r) continue;
      int top = 1;
      for (int e = L->rowptr[v]; e < L->rowptr[v + 1] && top; e++) {
        int u = L->col[e];
        if (stamp[u] >= r && prio_higher(u, v)) top = 0;
      }
      if (!top) continue;
      color[v] = smallest_free_colour(L, v, color, stamp, r, used, maxdeg + 2);
      stamp[v] = r;
      if (color[v] + 1 > nc) nc = color[v] + 1;
      left--;
    }
    r++;
  }
  free(used);
  free(stamp);
  *rounds = r;
  return nc;
}

/* ------------------------------------------------------------------------ */
/* Vector helpers and Gauss-Seidel (Alg. 2). */

static double vsum(int n, const double *x) {
  double s = 0.0;
  for (int i = 0; i < n; i++) s += x[i];
  return s;
}

static double vdot(int n, const double *x, const double *y) {
  double s = 0.0;
  for (int i = 0; i < n; i++) s += x[i] * y[i];
  return s;
}

/* x <- x - mean(x) 1 ; returns ||x|| after deflation */
static double deflate(int n, double *x) {
  double mu = vsum(n, x) / (double)n;
  for (int i = 0; i < n; i++) x[i] -= mu;
  return sqrt(vdot(n, x, x));
}

static void vscale(int n, double *x, double s) {
  for (int i = 0; i < n; i++) x[i] /= s;
}

/* One forward Gauss-Seidel sweep for A x = b with A = diag(d) - W (W the CSR
 * off-diagonal weights): x_i <- (b_i + sum_j w_ij x_j) / d_i, rows visited in
 * `order` (all rows; NULL = lexicographic), newest values used as they appear. */
static void gs_sweep(int n, const int *rowptr, const int *col, const double *w, const double *d,
                     const double *b, double *x, const int *order) {
  for (int t = 0; t < n; t++) {
    int i = order ? order[t] : t;
    double s = b ? b[i] : 0.0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; e++) s += w[e] * x[col[e]];
    x[i] = s / d[i];
  }
}

/* Alg. 2 with N sweeps (the tolerance test is not used): exported for pins. */
void oracle_gauss_seidel(int n, const int *rowptr, const int *col, const double *w, const double *d,
                         const double *b, double *x, int sweeps, const int *order) {
  for (int k = 0; k < sweeps; k++) gs_sweep(n, rowptr, col, w, d, b, x, order);
}

/* y = L x with L = D - W written as (Lx)_i = sum_j w_ij (x_i - x_j) */
static void lap_apply(const orc_lap *L, const double *x, double *y) {
  for (int i = 0; i < L->n; i++) {
    double s = 0.0;
    for (int e = L->rowptr[i]; e < L->rowptr[i + 1]; e++) s += L->w[e] * (x[i] - x[L->col[e]]);
    y[i] = s;
  }
}

/* Rayleigh quotient x^T L x / x^T x with x^T L x = 1/2 sum_i sum_j w_ij (x_i - x_j)^2 */
static double rayleigh(const orc_lap *L, const double *x) {
  double num = 0.0;
  for (int i = 0; i < L->n; i++)
    for (int e = L->rowptr[i]; e < L->rowptr[i + 1]; e++) {
      double t = x[i] - x[L->col[e]];
      num += L->w[e] * t * t;
    }
  return 0.5 * num / vdot(L->n, x, x);
}

/* ||L x - rho x|| / ||x|| */
static double residual_norm(const orc_lap *L, const double *x, double rho, double *tmp) {
  lap_apply(L, x, tmp);
  double s = 0.0;
  for (int i = 0; i < L->n; i++) {
    double t = tmp[i] - rho * x[i];
    s += t * t;
  }
  return sqrt(s / vdot(L->n, x, x));
}

/* ------------------------------------------------------------------------ */
/* Dense cyclic Jacobi eigensolver for symmetric matrices (Golub & Van Loan,
 * Matrix Computations, Sec. 8.5).  A (row-major n x n) is overwritten.  On exit
 * evals ascending and V (row-major) holds the matching eigenvectors as columns.
 * Returns the number of sweeps used. */
int oracle_jacobi_eig(int n, double *A, double *evals, double *V, int max_sweeps, double tol) {
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  double frob = 0.0;
  for (int i = 0; i < n * n; i++) frob += A[i] * A[i];
  frob = sqrt(frob);
  int sweep = 0;
  for (; sweep < max_sweeps; sweep++) {
    double off = 0.0;
    for (int p = 0; p < n; p++)
      for (int q = 0; q < n; q++)
        if (p != q) off += A[p * n + q] * A[p * n + q];
    if (sqrt(off) <= tol * frob) break;
    for (int p = 0; p < n - 1; p++)
      for (int q = p + 1; q < n; q++) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau)) : -1.0 / (-tau + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; k++) { /* A <- A J */
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; k++) { /* A <- J^T A */
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; k++) { /* V <- V J */
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; i++) evals[i] = A[i * n + i];
  /* selection sort of eigenpairs, ascending */
  for (int i = 0; i < n; i++) {
    int m = i;
    for (int j = i + 1; j < n; j++)
      if (evals[j] < evals[m]) m = j;
    if (m != i) {
      double t = evals[i]; evals[i] = evals[m]; evals[m] = t;
      for (int k = 0; k < n; k++) {
        double u = V[k * n + i]; V[k * n + i] = V[k * n + m]; V[k * n + m] = u;
      }
    }
  }
  return sweep;
}

/* ------------------------------------------------------------------------ */
/* Level smoothing: Gauss-Seidel sweeps (R5) then power iteration (R6). */

/* colour classes ascending, ascending index within a class (lexicographic
 * when the level has no colouring) */
static int *colour_order(const orc_level *lv) {
  int n = lv->L.n;
  int *order = (int *)malloc(sizeof(int) * (size_t)n);
  if (!order) return NULL;
  if (!lv->color) {
    for (int i = 0; i < n; i++) order[i] = i;
    return order;
  }
  int t = 0;
  for (int c = 0; c < lv->ncolors; c++)
    for (int i = 0; i < n; i++)
      if (lv->color[i] == c) order[t++] = i;
  return order;
}

static int smooth_level(orc_level *lv, double *x, const oracle_opts *o, int kmax, int forced) {
  int n = lv->L.n;
  double *old = (double *)malloc(sizeof(double) * (size_t)n);
  double *y = (double *)malloc(sizeof(double) * (size_t)n);
  double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
  int *order = (o->gs_order == 1) ? colour_order(lv) : NULL;
  if (!old || !y || !tmp || (o->gs_order == 1 && !order)) {
    free(old); free(y); free(tmp); free(order);
    return ORC_ENOMEM;
  }
  const orc_lap *L = &lv->L;
  lv->gs_sweeps_done = 0;
  for (int k = 0; k < o->gs_sweeps; k++) {
    memcpy(old, x, sizeof(double) * (size_t)n);
    gs_sweep(n, L->rowptr, L->col, L->w, L->d, NULL, x, order);
    double s = deflate(n, x);
    if (!(s > o->guard)) { /* annihilated: discard the sweep, stop smoothing */
      memcpy(x, old, sizeof(double) * (size_t)n);
      break;
    }
    vscale(n, x, s);
    lv->gs_sweeps_done++;
  }
  double sigma = lv->sigma;
  lv->pi_iters = 0;
  lv->last_cos = 0.0;
  int limit = forced >= 0 ? forced : kmax;
  for (int k = 1; k <= limit; k++) {
    lap_apply(L, x, tmp);
    for (int i = 0; i < n; i++) y[i] = sigma * x[i] - tmp[i];
    double s = deflate(n, y);
    if (!(s > o->guard * sigma)) break;
    vscale(n, y, s);
    double c = vdot(n, y, x);
    double r = 0.0;
    if (o->resid_tol > 0.0 && forced < 0) r = residual_norm(L, x, rayleigh(L, x), tmp);
    memcpy(x, y, sizeof(double) * (size_t)n);
    lv->pi_iters = k;
    lv->last_cos = c;
    if (forced >= 0) continue;
    if (c > 1.0 - o->pi_cos_tol && (o->resid_tol <= 0.0 || r <= o->resid_tol * sigma)) break;
    if (k == limit) lv->capped = 1;
  }
  free(old); free(y); free(tmp); free(order);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Krylov refinement of the finest level (reading R12). */

/* Rayleigh-Ritz on the k <= 3 columns S[0..k) (unit-free): Gram matrix
 * G = S^T S and projection H = S^T L S are formed from the columns and their
 * L-products; the columns are scaled to unit norm; column 2 (p), then column 1
 * (w), is dropped while its Cholesky pivot of the scaled Gram matrix is
 * <= 1e-10; the reduced symmetric problem R^-1 Hs R^-T is solved by the dense
 * Jacobi eigensolver.  On return c[0..3) holds the coefficients of the smallest
 * Ritz vector in the original columns (0 for dropped ones); the return value
 * is the number of columns kept (1: no step possible). */
static int rayleigh_ritz(int n, double *const *Sv, double *const *LS, int k, double *c) {
  double G[3][3], H[3][3];
  for (int a = 0; a < k; a++)
    for (int b = 0; b < k; b++) {
      G[a][b] = vdot(n, Sv[a], Sv[b]);
      H[a][b] = vdot(n, Sv[a], LS[b]);
    }
  int act[3], m;
  double D[3], R[3][3];
  int keep[3] = {1, k > 1, k > 2};
  for (;;) {
    m = 0;
    for (int a = 0; a < k; a++)
      if (keep[a]) act[m++] = a;
    for (int i = 0; i < m; i++) D[i] = 1.0 / sqrt(G[act[i]][act[i]]);
    int bad = -1;
    for (int i = 0; i < m && bad < 0; i++)
      for (int j = 0; j <= i; j++) {
        double sum = G[act[i]][act[j]] * D[i] * D[j];
        for (int q = 0; q < j; q++) sum -= R[i][q] * R[j][q];
        if (i == j) {
          if (!(sum > 1e-10)) { bad = i; break; }
          R[i][i] = sqrt(sum);
        } else {
          R[i][j] = sum / R[j][j];
        }
      }
    if (bad < 0) break;
    if (bad == 0) return 1;
    keep[act[bad]] = 0;
  }
  c[0] = c[1] = c[2] = 0.0;
  if (m == 1) return 1;
  /* M = R^-1 Hs R^-T, Hs = D H D */
  double Rinv[3][3], M[9], ev[3], V[9];
  for (int i = 0; i < m; i++)
    for (int j = 0; j < m; j++) {
      double sum = (i == j) ? 1.0 : 0.0;
      for (int q = 0; q < i; q++) sum -= R[i][q] * Rinv[q][j];
      Rinv[i][j] = sum / R[i][i];
    }
  for (int i = 0; i < m; i++)
    for (int j = 0; j < m; j++) {
      double sum = 0.0;
      for (int a = 0; a < m; a++)
        for (int b = 0; b < m; b++)
          sum += Rinv[i][a] * (H[act[a]][act[b]] * D[a] * D[b]) * Rinv[j][b];
      M[i * m + j] = sum;
    }
  for (int i = 0; i < m; i++)
    for (int j = 0; j < i; j++) M[i * m + j] = M[j * m + i] = 0.5 * (M[i * m + j] + M[j * m + i]);
  oracle_jacobi_eig(m, M, ev, V, 100, 1e-16);
  /* y = R^-T u for the smallest pair, then undo the column scaling */
  for (int a = 0; a < m; a++) {
    double y = 0.0;
    for (int i = 0; i < m; i++) y += Rinv[i][a] * V[i * m + 0];
    c[act[a]] = D[a] * y;
  }
  return m;
}

/* One V-cycle (reading R13) for L_l e = b on levels l..J of the run's
 * hierarchy; e is overwritten. */
static int vcycle(const oracle_run *r, int l, const double *b, double *e) {
  const orc_level *lv = &r->lv[l];
  const orc_lap *L = &lv->L;
  int n = L->n, J = r->nlevels - 1;
  int *order = colour_order(lv);
  if (!order) return ORC_ENOMEM;
  for (int i = 0; i < n; i++) e[i] = 0.0;
  if (l == J) {
    for (int k = 0; k < 20; k++) gs_sweep(n, L->rowptr, L->col, L->w, L->d, b, e, order);
    double mu = vsum(n, e) / (double)n;
    for (int i = 0; i < n; i++) e[i] -= mu;
    free(order);
    return ORC_OK;
  }
  gs_sweep(n, L->rowptr, L->col, L->w, L->d, b, e, order);
  int nc = lv->nc;
  double *t = (double *)malloc(sizeof(double) * (size_t)n);
  double *bc = (double *)calloc((size_t)nc, sizeof(double));
  double *ec = (double *)malloc(sizeof(double) * (size_t)nc);
  if (!t || !bc || !ec) { free(order); free(t); free(bc); free(ec); return ORC_ENOMEM; }
  lap_apply(L, e, t);
  for (int i = 0; i < n; i++) bc[lv->agg[i]] += b[i] - t[i];
  int st = vcycle(r, l + 1, bc, ec);
  if (st == ORC_OK) {
    for (int i = 0; i < n; i++) e[i] += ec[lv->agg[i]];
    for (int a = 0, z = n - 1; a < z; a++, z--) { int q = order[a]; order[a] = order[z]; order[z] = q; }
    gs_sweep(n, L->rowptr, L->col, L->w, L->d, b, e, order);
  }
  free(order); free(t); free(bc); free(ec);
  return st;
}

/* exported for the pins: e = V(b) on the hierarchy of a finished run */
int oracle_vcycle(const oracle_run *r, const double *b, double *e) {
  if (!r || r->nlevels < 1) return ORC_EINVAL;
  return vcycle(r, 0, b, e);
}

/* (1) LOBPCG with preconditioner D^-1 or one V-cycle (R13) on 1-perp.  x:
 * unit vector, orthogonal to 1, replaced by the refined vector.  forced >= 0
 * runs that many steps. */
static int refine_lobpcg(const oracle_run *run, orc_level *lv, double *x, const oracle_opts *o) {
  const orc_lap *L = &lv->L;
  int n = L->n;
  double *lx = (double *)malloc(sizeof(double) * (size_t)n);
  double *w = (double *)malloc(sizeof(double) * (size_t)n);
  double *lw = (double *)malloc(sizeof(double) * (size_t)n);
  double *p = (double *)calloc((size_t)n, sizeof(double));
  double *lp = (double *)calloc((size_t)n, sizeof(double));
  double *xn = (double *)malloc(sizeof(double) * (size_t)n);
  if (!lx || !w || !lw || !p || !lp || !xn) {
    free(lx); free(w); free(lw); free(p); free(lp); free(xn);
    return ORC_ENOMEM;
  }
  int forced = o->refine_forced, pvalid = 0, flat = 0, k = 0;
  lap_apply(L, x, lx);
  double theta = vdot(n, x, lx) / vdot(n, x, x), theta_best = 0.0;
  for (;;) {
    double rr = 0.0;
    for (int i = 0; i < n; i++) {
      w[i] = lx[i] - theta * x[i]; /* residual r, then w = D^-1 r */
      rr += w[i] * w[i];
    }
    if (forced < 0 && sqrt(rr) <= o->refine_tol * theta * sqrt(vdot(n, x, x))) break;
    /* no new lowest Rayleigh quotient (only rounding can cause it): restart
     * without p; eight such steps in a row end the iteration */
    if (k == 0 || theta < theta_best) {
      theta_best = theta;
      flat = 0;
    } else {
      pvalid = 0;
      if (++flat >= 8 && forced < 0) break;
    }
    if (forced >= 0 && k >= forced) break;
    if (forced < 0 && k >= o->refine_max_iters) { lv->capped = 1; break; }
    if (o->refine_precond == 1) {
      memcpy(xn, w, sizeof(double) * (size_t)n);
      int vst = vcycle(run, 0, xn, w);
      if (vst != ORC_OK) { free(lx); free(w); free(lw); free(p); free(lp); free(xn); return vst; }
    } else {
      for (int i = 0; i < n; i++) w[i] /= L->d[i];
    }
    double mw = vsum(n, w) / (double)n;
    for (int i = 0; i < n; i++) w[i] -= mw;
    lap_apply(L, w, lw);
    k++;
    double *Sv[3] = {x, w, p}, *LS[3] = {lx, lw, lp};
    double c[3];
    int kept = rayleigh_ritz(n, Sv, LS, pvalid ? 3 : 2, c);
    if (kept == 1) break; /* no step left: x is final */
    for (int i = 0; i < n; i++) {
      xn[i] = c[0] * x[i] + c[1] * w[i] + c[2] * p[i];
      p[i] = c[1] * w[i] + c[2] * p[i];
    }
    double pn = sqrt(vdot(n, p, p));
    pvalid = pn > 0.0;
    if (pvalid) {
      for (int i = 0; i < n; i++) p[i] /= pn;
      lap_apply(L, p, lp);
    }
    double s = deflate(n, xn);
    for (int i = 0; i < n; i++) x[i] = xn[i] / s;
    lap_apply(L, x, lx);
    theta = vdot(n, x, lx) / vdot(n, x, x);
  }
  lv->refine_iters = k;
  free(lx); free(w); free(lw); free(p); free(lp); free(xn);
  return ORC_OK;
}

/* (2) Lanczos on 1-perp with full reorthogonalisation, restarted from the
 * smallest Ritz vector every lanczos_basis steps (Golub & Van Loan, Sec. 10.1;
 * explicit restart).  Convergence is tested at the end of each cycle with the
 * Ritz estimate beta_m |s_m| (the residual of the Ritz pair in exact
 * arithmetic). */
static int refine_lanczos(orc_level *lv, double *x, const oracle_opts *o) {
  const orc_lap *L = &lv->L;
  int n = L->n, m = o->lanczos_basis;
  if (m < 1) return ORC_EINVAL;
  double *Q = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(m + 1));
  double *u = (double *)malloc(sizeof(double) * (size_t)n);
  double *h = (double *)malloc(sizeof(double) * (size_t)(m + 1));
  double *al = (double *)malloc(sizeof(double) * (size_t)m);
  double *be = (double *)malloc(sizeof(double) * (size_t)m);
  double *T = (double *)malloc(sizeof(double) * (size_t)m * (size_t)m);
  double *V = (double *)malloc(sizeof(double) * (size_t)m * (size_t)m);
  double *ev = (double *)malloc(sizeof(double) * (size_t)m);
  if (!Q || !u || !h || !al || !be || !T || !V || !ev) {
    free(Q); free(u); free(h); free(al); free(be); free(T); free(V); free(ev);
    return ORC_ENOMEM;
  }
  int forced = o->refine_forced, total = 0;
  double s0 = deflate(n, x);
  for (int i = 0; i < n; i++) x[i] /= s0;
  for (;;) {
    memcpy(Q, x, sizeof(double) * (size_t)n);
    int kk = 0;
    for (int j = 0; j < m; j++) {
      if (forced >= 0 ? total >= forced : total >= o->refine_max_iters) break;
      const double *q = Q + (size_t)j * n;
      lap_apply(L, q, u);
      total++;
      double mu = vsum(n, u) / (double)n;
      for (int i = 0; i < n; i++) u[i] -= mu;
      al[j] = vdot(n, q, u);
      for (int i = 0; i < n; i++) u[i] -= al[j] * q[i];
      if (j > 0)
        for (int i = 0; i < n; i++) u[i] -= be[j - 1] * Q[(size_t)(j - 1) * n + i];
      for (int pass = 0; pass < 2; pass++) {
        for (int t = 0; t <= j; t++) h[t] = vdot(n, Q + (size_t)t * n, u);
        for (int t = 0; t <= j; t++)
          for (int i = 0; i < n; i++) u[i] -= h[t] * Q[(size_t)t * n + i];
      }
      be[j] = sqrt(vdot(n, u, u));
      kk = j + 1;
      if (!(be[j] > 1e-12 * fabs(al[j]))) break; /* invariant subspace */
      for (int i = 0; i < n; i++) Q[(size_t)(j + 1) * n + i] = u[i] / be[j];
    }
    if (kk == 0) { /* cap reached at a cycle boundary */
      if (forced < 0) lv->capped = 1;
      break;
    }
    for (int a = 0; a < kk * kk; a++) T[a] = 0.0;
    for (int a = 0; a < kk; a++) {
      T[a * kk + a] = al[a];
      if (a + 1 < kk) T[a * kk + a + 1] = T[(a + 1) * kk + a] = be[a];
    }
    oracle_jacobi_eig(kk, T, ev, V, 100, 1e-16);
    double theta = ev[0];
    for (int i = 0; i < n; i++) {
      double y = 0.0;
      for (int t = 0; t < kk; t++) y += V[t * kk + 0] * Q[(size_t)t * n + i];
      x[i] = y;
    }
    double s = deflate(n, x);
    for (int i = 0; i < n; i++) x[i] /= s;
    double est = be[kk - 1] * fabs(V[(kk - 1) * kk + 0]);
    if (forced >= 0) {
      if (total >= forced) break;
      continue;
    }
    if (est <= o->refine_tol * theta) break;
    if (total >= o->refine_max_iters) { lv->capped = 1; break; }
  }
  lv->refine_iters = total;
  free(Q); free(u); free(h); free(al); free(be); free(T); free(V); free(ev);
  return ORC_OK;
}

static int connected(const orc_lap *L) {
  int n = L->n;
  int *seen = (int *)calloc((size_t)n, sizeof(int));
  int *stack = (int *)malloc(sizeof(int) * (size_t)n);
  if (!seen || !stack) { free(seen); free(stack); return -1; }
  int top = 0, count = 1;
  stack[top++] = 0;
  seen[0] = 1;
  while (top > 0) {
    int u = stack[--top];
    for (int e = L->rowptr[u]; e < L->rowptr[u + 1]; e++) {
      int v = L->col[e];
      if (!seen[v]) { seen[v] = 1; count++; stack[top++] = v; }
    }
  }
  free(seen);
  free(stack);
  return count == n;
}

static double lap_sigma(const orc_lap *L) {
  double m = 0.0;
  for (int i = 0; i < L->n; i++)
    if (L->d[i] > m) m = L->d[i];
  return 2.0 * m;
}

/* ------------------------------------------------------------------------ */
/* Setup phase of Alg. 3 (hierarchy only). */

static int build_hierarchy(oracle_run *r, const oracle_opts *o) {
  for (;;) {
    orc_level *lv = &r->lv[r->nlevels - 1];
    int n = lv->L.n;
    lv->sigma = lap_sigma(&lv->L);
    if (o->gs_order == 1) {
      lv->color = (int *)malloc(sizeof(int) * (size_t)n);
      if (!lv->color) return ORC_ENOMEM;
      int nc = color_greedy(&lv->L, lv->color);
      if (nc < 0) return nc;
      lv->ncolors = nc;
    }
    if (n <= o->coarse_max_n || r->nlevels >= o->max_levels || r->nlevels >= ORC_MAX_LEVELS) break;
    int *agg = (int *)malloc(sizeof(int) * (size_t)n);
    if (!agg) return ORC_ENOMEM;
    int nc;
    if (o->hec_mode == 2) {
      nc = hec_paper(&lv->L, o->seed + (uint64_t)(r->nlevels - 1), NULL, agg);
    } else {
      lv->mate = (int *)malloc(sizeof(int) * (size_t)n);
      if (!lv->mate) { free(agg); return ORC_ENOMEM; }
      int st = (o->hec_mode == 0) ? match_handshake(&lv->L, o->tie_rule, lv->mate, &lv->match_rounds)
                                  : match_sorted_greedy(&lv->L, o->tie_rule, lv->mate);
      if (st != ORC_OK) { free(agg); return st; }
      nc = aggregate_from_matching(&lv->L, lv->mate, o->tie_rule, agg);
    }
    if (nc < 0) { free(agg); return nc; }
    if (nc < 2 || (double)nc > o->stall_ratio * (double)n) { free(agg); break; }
    lv->agg = agg;
    lv->nc = nc;
    orc_level *next = &r->lv[r->nlevels];
    memset(next, 0, sizeof(*next));
    int st = galerkin(&lv->L, agg, nc, &next->L);
    r->nlevels++;
    if (st != ORC_OK) return st;
  }
  return ORC_OK;
}

static int ingest_into(oracle_run *r, int n, long long nnz, const int *rowptr, const int *col, const double *w) {
  run_clear(r);
  r->nlevels = 1;
  int st = lap_ingest(n, nnz, rowptr, col, w, &r->lv[0].L, &r->bad_index);
  r->n = n;
  return st;
}

int oracle_build(oracle_run *r, int n, long long nnz, const int *rowptr, const int *col, const double *w,
                 const oracle_opts *o) {
  int st = ingest_into(r, n, nnz, rowptr, col, w);
  if (st == ORC_OK) st = build_hierarchy(r, o);
  r->status = st;
  return st;
}

/* Whole method (Alg. 3 + power iteration + Rayleigh quotient).  forced_pi may
 * hold one count per level (-1 = use the stop rule). */
int oracle_solve(oracle_run *r, int n, long long nnz, const int *rowptr, const int *col, const double *w,
                 const oracle_opts *o, const int *forced_pi) {
  int st = oracle_build(r, n, nnz, rowptr, col, w, o);
  if (st != ORC_OK) return st;
  int J = r->nlevels - 1;
  orc_level *cl = &r->lv[J];
  int nJ = cl->L.n;
  if (connected(&cl->L) != 1) { r->status = ORC_EDISCONNECTED; return ORC_EDISCONNECTED; }
  double *x = (double *)malloc(sizeof(double) * (size_t)nJ);
  if (!x) return ORC_ENOMEM;
  /* coarsest level (Alg. 3, step 2) */
  if (o->coarsest_dense) {
    double *A = (double *)calloc((size_t)nJ * nJ, sizeof(double));
    double *V = (double *)malloc(sizeof(double) * (size_t)nJ * nJ);
    double *ev = (double *)malloc(sizeof(double) * (size_t)nJ);
    if (!A || !V || !ev) { free(A); free(V); free(ev); free(x); return ORC_ENOMEM; }
    for (int i = 0; i < nJ; i++) {
      A[i * nJ + i] = cl->L.d[i];
      for (int e = cl->L.rowptr[i]; e < cl->L.rowptr[i + 1]; e++) A[i * nJ + cl->L.col[e]] = -cl->L.w[e];
    }
    oracle_jacobi_eig(nJ, A, ev, V, 100, 1e-15);
    for (int i = 0; i < nJ; i++) x[i] = V[i * nJ + 1];
    double s = deflate(nJ, x);
    vscale(nJ, x, s);
    free(A); free(V); free(ev);
  } else {
    for (int i = 0; i < nJ; i++) x[i] = orc_uniform(o->seed, (uint64_t)i);
    double s = deflate(nJ, x);
    if (!(s > o->guard)) { free(x); r->status = ORC_EDEGENERATE; return ORC_EDEGENERATE; }
    vscale(nJ, x, s);
    st = smooth_level(cl, x, o, (J == 0 && o->refine) ? 0 : o->pi_max_iters_coarsest,
                      (J == 0 && o->refine) ? 0 : (forced_pi ? forced_pi[J] : -1));
    if (st != ORC_OK) { free(x); return st; }
  }
  cl->x = x;
  /* cascadic refinement (Alg. 3, step 3) */
  for (int j = J - 1; j >= 0; j--) {
    orc_level *lv = &r->lv[j];
    int nf = lv->L.n;
    double *xf = (double *)malloc(sizeof(double) * (size_t)nf);
    if (!xf) return ORC_ENOMEM;
    const double *xc = r->lv[j + 1].x;
    for (int i = 0; i < nf; i++) xf[i] = xc[lv->agg[i]]; /* y^j = (I_j^{j+1})^T y^{j+1} */
    double s = deflate(nf, xf);
    if (!(s > o->guard)) { free(xf); r->status = ORC_EDEGENERATE; return ORC_EDEGENERATE; }
    vscale(nf, xf, s);
    st = smooth_level(lv, xf, o, (j == 0 && o->refine) ? 0 : o->pi_max_iters,
                      (j == 0 && o->refine) ? 0 : (forced_pi ? forced_pi[j] : -1));
    if (st != ORC_OK) { free(xf); return st; }
    lv->x = xf;
  }
  /* finest-level Krylov refinement (reading R12) */
  if (o->refine == 1 || o->refine == 2) {
    orc_level *l0 = &r->lv[0];
    st = (o->refine == 1) ? refine_lobpcg(r, l0, l0->x, o) : refine_lanczos(l0, l0->x, o);
    if (st != ORC_OK) return st;
  }
  /* Rayleigh quotient on the finest level, residual, orthogonality, sign */
  orc_lap *L0 = &r->lv[0].L;
  r->x = (double *)malloc(sizeof(double) * (size_t)n);
  double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
  if (!r->x || !tmp) { free(tmp); return ORC_ENOMEM; }
  memcpy(r->x, r->lv[0].x, sizeof(double) * (size_t)n);
  int imax = 0;
  for (int i = 1; i < n; i++)
    if (fabs(r->x[i]) > fabs(r->x[imax])) imax = i;
  if (r->x[imax] < 0.0)
    for (int i = 0; i < n; i++) r->x[i] = -r->x[i];
  r->lambda = rayleigh(L0, r->x);
  r->residual = residual_norm(L0, r->x, r->lambda, tmp);
  r->ortho = fabs(vsum(n, r->x)) / (sqrt((double)n) * sqrt(vdot(n, r->x, r->x)));
  free(tmp);
  r->status = ORC_OK;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Accessors for the tests. */

int oracle_run_status(const oracle_run *r) { return r->status; }
long long oracle_run_bad_index(const oracle_run *r) { return r->bad_index; }
int oracle_run_num_levels(const oracle_run *r) { return r->nlevels; }
double oracle_run_lambda(const oracle_run *r) { return r->lambda; }
double oracle_run_residual(const oracle_run *r) { return r->residual; }
double oracle_run_ortho(const oracle_run *r) { return r->ortho; }

void oracle_run_copy_x(const oracle_run *r, double *x) {
  if (r->x) memcpy(x, r->x, sizeof(double) * (size_t)r->n);
}

/* info[0..9] = n, nnz, nc, ncolors, match_rounds, gs_sweeps_done, pi_iters, has_agg, has_x, color_rounds
 * dinfo[0..1] = sigma, last_cos */
void oracle_run_level_info(const oracle_run *r, int l, long long *info, double *dinfo) {
  const orc_level *lv = &r->lv[l];
  info[0] = lv->L.n;
  info[1] = lv->L.nnz;
  info[2] = lv->nc;
  info[3] = lv->ncolors;
  info[4] = lv->match_rounds;
  info[5] = lv->gs_sweeps_done;
  info[6] = lv->pi_iters;
  info[7] = lv->agg != NULL;
  info[8] = lv->x != NULL;
  info[9] = lv->color_rounds;
  info[10] = lv->refine_iters;
  info[11] = lv->capped;
  dinfo[0] = lv->sigma;
  dinfo[1] = lv->last_cos;
}

/* any pointer may be NULL */
void oracle_run_copy_level(const oracle_run *r, int l, int *rowptr, int *col, double *w, double *d, int *agg,
                           int *mate, int *color, double *x) {
  const orc_level *lv = &r->lv[l];
  int n = lv->L.n;
  if (rowptr) memcpy(rowptr, lv->L.rowptr, sizeof(int) * (size_t)(n + 1));
  if (col) memcpy(col, lv->L.col, sizeof(int) * (size_t)lv->L.nnz);
  if (w) memcpy(w, lv->L.w, sizeof(double) * (size_t)lv->L.nnz);
  if (d) memcpy(d, lv->L.d, sizeof(double) * (size_t)n);
  if (agg && lv->agg) memcpy(agg, lv->agg, sizeof(int) * (size_t)n);
  if (mate && lv->mate) memcpy(mate, lv->mate, sizeof(int) * (size_t)n);
  if (color && lv->color) memcpy(color, lv->color, sizeof(int) * (size_t)n);
  if (x && lv->x) memcpy(x, lv->x, sizeof(double) * (size_t)n);
}

/* ------------------------------------------------------------------------ */
/* Stand-alone pieces on a caller-given Laplacian (level 0 of a fresh run),
 * exported so the tests can pin each step separately. */

int oracle_match(int n, long long nnz, const int *rowptr, const int *col, const double *w, int mode, int tie_rule,
                 int *mate, int *rounds) {
  orc_lap L;
  long long bad;
  memset(&L, 0, sizeof(L));
  int st = lap_ingest(n, nnz, rowptr, col, w, &L, &bad);
  if (st == ORC_OK) {
    *rounds = 0;
    st = (mode == 0) ? match_handshake(&L, tie_rule, mate, rounds) : match_sorted_greedy(&L, tie_rule, mate);
  }
  lap_free(&L);
  return st;
}

int oracle_aggregate(int n, long long nnz, const int *rowptr, const int *col, const double *w, const int *mate,
                     int tie_rule, int *agg) {
  orc_lap L;
  long long bad;
  memset(&L, 0, sizeof(L));
  int st = lap_ingest(n, nnz, rowptr, col, w, &L, &bad);
  if (st == ORC_OK) st = aggregate_from_matching(&L, mate, tie_rule, agg);
  lap_free(&L);
  return st;
}

int oracle_hec_paper(int n, long long nnz, const int *rowptr, const int *col, const double *w, uint64_t seed,
                     const int *perm, int *agg) {
  orc_lap L;
  long long bad;
  memset(&L, 0, sizeof(L));
  int st = lap_ingest(n, nnz, rowptr, col, w, &L, &bad);
  if (st == ORC_OK) st = hec_paper(&L, seed, perm, agg);
  lap_free(&L);
  return st;
}

int oracle_color(int n, long long nnz, const int *rowptr, const int *col, const double *w, int jp, int *color,
                 int *rounds) {
  orc_lap L;
  long long bad;
  memset(&L, 0, sizeof(L));
  int st = lap_ingest(n, nnz, rowptr, col, w, &L, &bad);
  if (st == ORC_OK) {
    *rounds = 0;
    st = jp ? color_jp(&L, color, rounds) : color_greedy(&L, color);
  }
  lap_free(&L);
  return st;
}

/* coarse operator from a caller-given aggregate map; writes sizes into
 * out_sizes[0..1] = (nc, nnz_c) and, when the arrays are non-NULL and large
 * enough (cap entries), the coarse CSR and diagonal */
int oracle_galerkin(int n, long long nnz, const int *rowptr, const int *col, const double *w, const int *agg,
                    int nc, long long cap, int *crowptr, int *ccol, double *cw, double *cd, long long *out_sizes) {
  orc_lap L, C;
  long long bad;
  memset(&L, 0, sizeof(L));
  memset(&C, 0, sizeof(C));
  int st = lap_ingest(n, nnz, rowptr, col, w, &L, &bad);
  if (st == ORC_OK) st = galerkin(&L, agg, nc, &C);
  if (st == ORC_OK) {
    out_sizes[0] = C.n;
    out_sizes[1] = C.nnz;
    if (crowptr && C.nnz <= cap) {
      memcpy(crowptr, C.rowptr, sizeof(int) * (size_t)(nc + 1));
      memcpy(ccol, C.col, sizeof(int) * (size_t)C.nnz);
      memcpy(cw, C.w, sizeof(double) * (size_t)C.nnz);
      memcpy(cd, C.d, sizeof(double) * (size_t)nc);
    }
  }
  lap_free(&L);
  lap_free(&C);
  return st;
}

double oracle_uniform01(uint64_t seed, uint64_t k) { return orc_uniform(seed, k); }
