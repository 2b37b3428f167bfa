// engine.cuh -- the level engine of the cascadic multigrid Fiedler solver.
//
// One templated engine walks the whole method of Alg. 3 on the device:
//   setup   (Alg. 1 + Alg. 3 step 1): ingest (Def 2.1), colouring + colour-order
//           copy of each level, heavy-edge matching, aggregation, Galerkin
//           coarse operator L^{i+1} = I L^i I^T, until n <= coarse_max_n;
//   coarsest (Alg. 3 step 2): connectivity check, random start, Gauss-Seidel
//           sweeps (Alg. 2) and power iteration on sigma I - L;
//   refinement (Alg. 3 step 3): y^j = I^T y^{j+1}, Gauss-Seidel sweeps, power
//           iteration with deflation of the constant vector;
//   final:  Rayleigh quotient, residual, orthogonality, sign (Sec. 2).
//
// The same code runs in two shapes.  GRID = true: a cooperative launch over
// all SMs, phases separated by a bounded grid barrier, for levels with
// n > tail_max_n.  GRID = false: one block with __syncthreads, for the small
// levels at the bottom of the hierarchy, where grid barriers would dominate.
// Every thread of every block runs the same control flow: decisions are taken
// from grid reductions that every block finishes redundantly (same data, same
// order, same result), and arena offsets are advanced identically by every
// thread, so no extra barrier is needed to publish them.
//
// GB300 notes: FP64 issues at a small fraction of the FP32 rate, so counts,
// scans, maxima and weight comparisons are integer work (bit patterns of
// positive floats order like their values), and the FP64 sums the method
// needs go through a shared halving tree instead of all-lane shuffles.
// Data-dependent rounds (colouring, matching) walk atomic-append worklists, so
// late rounds touch only live vertices and need one barrier and no reduction.
#pragma once
#include <cuda_runtime.h>
#include <float.h>
#include <limits.h>
#include <stdint.h>

#include "fz_state.h"

namespace fz {

#define FZD __device__ __forceinline__
// the colouring round (run at every setup barrier), the refinement, the
// V-cycle and Alg. 1's random-order coarsening are real calls: inlined into
// the kernels beside the rest of the engine they multiply compile time and
// register pressure (their inner loops stay inline)
#define FZN __device__ __noinline__

// ---------------------------------------------------------------------------
// splitmix64 (S. Vigna): output k of the stream seeded with s is
// mix(s + (k + 1) * 0x9E3779B97F4A7C15).  Used for the heavy-edge tie-break
// hash, the colouring priority and the coarsest-level random start.
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

FZD uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
FZD uint64_t sm64(uint64_t seed, uint64_t k) { return mix64(seed + (k + 1) * kGamma); }
FZD uint64_t edge_hash(int lo, int hi) { return sm64(((uint64_t)(uint32_t)lo << 32) | (uint32_t)hi, 0); }
FZD uint64_t vtx_hash(int v) { return sm64((uint64_t)(uint32_t)v, 0); }
FZD double uniform01(uint64_t seed, uint64_t k) {
  return (double)(sm64(seed, k) >> 11) * (1.0 / 9007199254740992.0);
}

// gpu-scope release / acquire primitives of the grid barrier
FZD unsigned atom_add_release(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
FZD unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
FZD void fence_acquire() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

FZD uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// Heavy-edge order K(e) = (w desc, h(min,max) asc, min asc, max asc).  Weights
// are positive, so their IEEE bit patterns order like their values: keys are
// the float bits (fine level in float) or the double bits (FP64 levels).  The
// hash is only evaluated when weights tie exactly.
struct Best {
  uint64_t wk;
  uint64_t h;
  int v, lo, hi, hok;
};
FZD void best_init(Best &b) {
  b.v = -1;
  b.hok = 0;
}
FZD bool best_beats(Best &b, uint64_t wk, int u, int v, int tie) {
  if (b.v < 0) return true;
  if (wk != b.wk) return wk > b.wk;
  const int lo = min(u, v), hi = max(u, v);
  if (tie == 0) {
    if (!b.hok) {
      b.h = edge_hash(b.lo, b.hi);
      b.hok = 1;
    }
    const uint64_t h = edge_hash(lo, hi);
    if (h != b.h) return h < b.h;
  }
  if (lo != b.lo) return lo < b.lo;
  return hi < b.hi;
}
FZD void best_set(Best &b, uint64_t wk, int u, int v) {
  b.wk = wk;
  b.v = v;
  b.lo = min(u, v);
  b.hi = max(u, v);
  b.hok = 0;
}

// ---------------------------------------------------------------------------
// Rayleigh-Ritz step of the LOBPCG refinement (one thread, FP64).  G and H are
// the Gram matrix S^T S and the projection S^T L S of the basis S = [x, w, p]
// (row-major 3 x 3).  The basis is scaled to unit columns, w and then p are
// dropped when their Cholesky pivot of the scaled Gram matrix falls below
// `pivot` (nearly dependent directions), the k x k problem R^-1 H R^-T u =
// theta u (G = R R^T) is solved by cyclic Jacobi rotations, and the smallest
// Ritz value is returned with its coefficients c in the unscaled basis (0 for
// dropped or unused vectors).  Returns a negative value if x alone is left
// and no step is possible.  The pivot bound follows the accuracy of the sums:
// with float vectors a direction less than 1e-3 away (in sine) from the span
// of the others is lost in the rounding of H, and R^-1 would amplify it.
constexpr double kRrPivot64 = 1e-10;
constexpr double kRrPivot32 = 1e-6;
// LOBPCG ends after this many steps in a row without a new lowest Rayleigh
// quotient (in exact arithmetic every step lowers it).  Not fewer: when
// lambda_3 lies within ~1% of lambda_2 the iteration can sit a few steps on a
// lambda_3 plateau, where a float run's descent hides under rounding, before
// the lambda_2 component takes over
constexpr int kRefineFlat = 8;

FZD double rr3(const double *G, const double *H, bool use_w, bool use_p, double *c, double pivot) {
  int act[3], k;
  double D[3], R[3][3], M[3][3], Vv[3][3];
  for (;;) {
    k = 0;
    act[k++] = 0;
    if (use_w) act[k++] = 1;
    if (use_p) act[k++] = 2;
    for (int i = 0; i < k; i++) D[i] = 1.0 / sqrt(G[act[i] * 3 + act[i]]);
    int bad = -1;
    for (int i = 0; i < k && bad < 0; i++) {
      for (int j = 0; j <= i; j++) {
        double sum = G[act[i] * 3 + act[j]] * D[i] * D[j];
        for (int m = 0; m < j; m++) sum -= R[i][m] * R[j][m];
        if (i == j) {
          if (!(sum > pivot)) {
            bad = i;
            break;
          }
          R[i][i] = sqrt(sum);
        } else {
          R[i][j] = sum / R[j][j];
        }
      }
    }
    if (bad < 0) break;
    if (bad == 0) return -1.0;
    if (act[bad] == 2) use_p = false;
    else use_w = false;
  }
  if (k == 1) return -1.0;
  // Y = R^-1 Hs (forward substitution, column by column), M = R^-1 Y^T
  double Y[3][3];
  for (int col = 0; col < k; col++)
    for (int i = 0; i < k; i++) {
      double sum = H[act[i] * 3 + act[col]] * D[i] * D[col];
      for (int m = 0; m < i; m++) sum -= R[i][m] * Y[m][col];
      Y[i][col] = sum / R[i][i];
    }
  for (int col = 0; col < k; col++)
    for (int i = 0; i < k; i++) {
      double sum = Y[col][i];
      for (int m = 0; m < i; m++) sum -= R[i][m] * M[m][col];
      M[i][col] = sum / R[i][i];
    }
  for (int i = 0; i < k; i++)
    for (int j = 0; j < i; j++) M[i][j] = M[j][i] = 0.5 * (M[i][j] + M[j][i]);
  for (int i = 0; i < k; i++)
    for (int j = 0; j < k; j++) Vv[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 50; sweep++) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < k; i++)
      for (int j = 0; j < k; j++) {
        tot += M[i][j] * M[i][j];
        if (i != j) off += M[i][j] * M[i][j];
      }
    if (off <= 1e-30 * tot) break;
    for (int a = 0; a < k - 1; a++)
      for (int b = a + 1; b < k; b++) {
        if (M[a][b] == 0.0) continue;
        const double th = (M[b][b] - M[a][a]) / (2.0 * M[a][b]);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int m = 0; m < k; m++) {  // columns a, b
          const double ma = M[m][a], mb = M[m][b];
          M[m][a] = cs * ma - sn * mb;
          M[m][b] = sn * ma + cs * mb;
        }
        for (int m = 0; m < k; m++) {  // rows a, b
          const double ma = M[a][m], mb = M[b][m];
          M[a][m] = cs * ma - sn * mb;
          M[b][m] = sn * ma + cs * mb;
        }
        for (int m = 0; m < k; m++) {
          const double va = Vv[m][a], vb = Vv[m][b];
          Vv[m][a] = cs * va - sn * vb;
          Vv[m][b] = sn * va + cs * vb;
        }
      }
  }
  int mi = 0;
  for (int i = 1; i < k; i++)
    if (M[i][i] < M[mi][mi]) mi = i;
  // y = R^-T u (back substitution), c = D y
  double y[3];
  for (int i = k - 1; i >= 0; i--) {
    double sum = Vv[i][mi];
    for (int m = i + 1; m < k; m++) sum -= R[m][i] * y[m];
    y[i] = sum / R[i][i];
  }
  c[0] = c[1] = c[2] = 0.0;
  for (int i = 0; i < k; i++) c[act[i]] = D[i] * y[i];
  return M[mi][mi];
}

// Smallest eigenpair of the symmetric tridiagonal matrix with diagonal
// al[0..k) and off-diagonal be[0..k-1) (one thread, FP64): the eigenvalue by
// bisection on the Sturm count (number of eigenvalues below x = negative
// pivots of the LDL^T factorisation of T - x I) inside the Gershgorin
// interval, the eigenvector by two steps of inverse iteration (tridiagonal
// elimination with partial pivoting) from the all-ones vector, normalised.
FZD double tri_smallest(const double *al, const double *be, int k, double *s, double *work) {
  double lo = al[0], hi = al[0];
  for (int i = 0; i < k; i++) {
    const double r = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i + 1 < k ? fabs(be[i]) : 0.0);
    lo = fmin(lo, al[i] - r);
    hi = fmax(hi, al[i] + r);
  }
  const double scale = fmax(fabs(lo), fabs(hi)) + DBL_MIN;
  for (int it = 0; it < 200 && hi - lo > 4.0 * DBL_EPSILON * scale; it++) {
    const double x = 0.5 * (lo + hi);
    int neg = 0;
    double q = al[0] - x;
    if (q == 0.0) q = -DBL_EPSILON * scale;
    neg += q < 0.0;
    for (int i = 1; i < k; i++) {
      q = al[i] - x - be[i - 1] * be[i - 1] / q;
      if (q == 0.0) q = -DBL_EPSILON * scale;
      neg += q < 0.0;
    }
    if (neg >= 1) hi = x;
    else lo = x;
  }
  const double th = 0.5 * (lo + hi);
  // inverse iteration: solve (T - th I) y = s with partial pivoting; work holds
  // the three diagonals of U and the multipliers (4k doubles)
  double *u0 = work, *u1 = work + k, *u2 = work + 2 * k, *ml = work + 3 * k;
  for (int i = 0; i < k; i++) s[i] = 1.0;
  for (int rep = 0; rep < 2; rep++) {
    // forward elimination with row interchanges: the pivot row carries entries
    // in columns i, i+1, i+2 (c_d, c_e, c_f) and its right-hand side
    double rhs_prev = s[0];
    double c_d = al[0] - th, c_e = k > 1 ? be[0] : 0.0, c_f = 0.0;
    for (int i = 0; i < k - 1; i++) {
      const double sub = be[i], nd = al[i + 1] - th, ne = i + 2 < k ? be[i + 1] : 0.0;
      double rn = s[i + 1];
      if (fabs(c_d) >= fabs(sub)) {  // no interchange
        const double mlt = c_d != 0.0 ? sub / c_d : 0.0;
        u0[i] = c_d;
        u1[i] = c_e;
        u2[i] = c_f;
        ml[i] = mlt;
        s[i] = rhs_prev;
        c_d = nd - mlt * c_e;
        c_e = ne - mlt * c_f;
        c_f = 0.0;
        rhs_prev = rn - mlt * rhs_prev;
      } else {  // interchange rows i and i+1
        const double mlt = c_d / sub;
        u0[i] = sub;
        u1[i] = nd;
        u2[i] = ne;
        ml[i] = mlt;
        s[i] = rn;
        const double od = c_e - mlt * nd, oe = c_f - mlt * ne;
        c_d = od;
        c_e = oe;
        c_f = 0.0;
        rhs_prev = rhs_prev - mlt * rn;
      }
    }
    u0[k - 1] = c_d;
    u1[k - 1] = 0.0;
    u2[k - 1] = 0.0;
    s[k - 1] = rhs_prev;
    // back substitution (tiny pivots replaced: the solution grows along the eigenvector)
    double nrm = 0.0;
    for (int i = k - 1; i >= 0; i--) {
      double v = s[i];
      if (i + 1 < k) v -= u1[i] * s[i + 1];
      if (i + 2 < k) v -= u2[i] * s[i + 2];
      double piv = u0[i];
      if (fabs(piv) < DBL_EPSILON * scale) piv = piv < 0.0 ? -DBL_EPSILON * scale : DBL_EPSILON * scale;
      s[i] = v / piv;
    }
    for (int i = 0; i < k; i++) nrm += s[i] * s[i];
    nrm = 1.0 / sqrt(nrm);
    for (int i = 0; i < k; i++) s[i] *= nrm;
  }
  return th;
}

// ---------------------------------------------------------------------------
// shared storage: a static __shared__ declared in a function is one allocation
// per kernel
constexpr int kShSort = 2560;  // u64 words of the raw buffer (20 KB): block sums, Gram and
                                // basis dots of up to 32 warps, sorts (kWarpSeg per warp)
constexpr int kSmallSeg = 32;  // segments up to this length are sorted by one thread
constexpr int kWarpSeg = 128;  // longer ones up to this length by one warp (in shared memory)
constexpr int kWarpSegG = 2048;  // longer ones up to this length by one warp in place (global memory)
constexpr int kHeavyDeg = 32;  // rows of at least this degree are processed by a whole warp
constexpr int kJposDeg = 16;   // colouring: vertices of at least this degree remember their blocker
constexpr int kWarpNnz = 512;  // tiny levels up to this many entries are smoothed by one warp

FZD uint64_t *sh_raw() {
  __shared__ uint64_t raw[kShSort];
  return raw;
}
FZD int *sh_list() {
  __shared__ int list[kMaxThreads];
  return list;
}
FZD int *sh_list2() {
  __shared__ int list[kMaxThreads];
  return list;
}
FZD int *sh_ints() {
  __shared__ int v[8];
  return v;
}
FZD long long *sh_ll() {
  __shared__ long long v[3 * 33];
  return v;
}
// heavy vertices (degree >= kHeavyDeg) met by a block in one colouring round
// or matching phase are listed (in the block's range of a scratch array) for
// the block's warps; these are the list lengths (zero between uses).
// 0: colouring, 1: matching.
FZD int *sh_hcnt() {
  __shared__ int c[2];
  return c;
}
FZD double *sh_bc() {  // scalars computed by one thread, read by the block
  __shared__ double v[8];
  return v;
}
FZD double *sh_prof() {  // [2][PH_COUNT] totals, then [kMaxLevels][PH_COUNT] per level
  __shared__ double v[2 * PH_COUNT + kMaxLevels * PH_COUNT];
  return v;
}

// exclusive block scan of an int; *total = block sum.  All threads must call.
FZD int block_scan(int v, int *total) {
  __shared__ int wsum[33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = lane < nw ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    wsum[lane] = t;
  }
  __syncthreads();
  int incl = x + (w > 0 ? wsum[w - 1] : 0);
  *total = wsum[nw - 1];
  __syncthreads();
  return incl - v;
}

// integer block reduction of (a sum, b sum, mx max); result in every thread
FZD void block_ired(IRed &r) {
  long long *s = sh_ll();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    r.a += __shfl_xor_sync(0xffffffffu, r.a, o);
    r.b += __shfl_xor_sync(0xffffffffu, r.b, o);
    r.mx = max(r.mx, __shfl_xor_sync(0xffffffffu, r.mx, o));
  }
  if (lane == 0) {
    s[w] = r.a;
    s[33 + w] = r.b;
    s[66 + w] = r.mx;
  }
  __syncthreads();
  if (w == 0) {
    long long a = lane < nw ? s[lane] : 0, b = lane < nw ? s[33 + lane] : 0;
    long long m = lane < nw ? s[66 + lane] : LLONG_MIN;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
      m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if (lane == 0) {
      s[32] = a;
      s[65] = b;
      s[98] = m;
    }
  }
  __syncthreads();
  r.a = s[32];
  r.b = s[65];
  r.mx = s[98];
  __syncthreads();
}

// FP64 block sum of K <= 4 values by a shared halving tree (few FP64 adds),
// then one warp; fixed order, result in every thread
template <int K>
FZD void block_dsum(double (&v)[K]) {
  static_assert(K >= 1 && K <= 4, "block_dsum: K <= 4");
  double *sh = reinterpret_cast<double *>(sh_raw());
  const int t = threadIdx.x;
  for (int s = blockDim.x >> 1; s >= 32; s >>= 1) {
    if (t >= s && t < 2 * s) {
#pragma unroll
      for (int k = 0; k < K; k++) sh[k * s + (t - s)] = v[k];
    }
    __syncthreads();
    if (t < s) {
#pragma unroll
      for (int k = 0; k < K; k++) v[k] += sh[k * s + t];
    }
    __syncthreads();
  }
  if (t < 32) {
#pragma unroll
    for (int k = 0; k < K; k++)
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (t == 0)
#pragma unroll
      for (int k = 0; k < K; k++) sh[k] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; k++) v[k] = sh[k];
  __syncthreads();
}

// A group of G lanes (G in 4..32, aligned inside the warp) walks the entries
// [e0, e1) of one heavy row: a head of up to three entries, then aligned
// quads (each lane loads four column indices and four weights with 16-byte
// loads; the arrays start on 256-byte boundaries), then the tail.  f(j, w) is
// called for the lane's entries in a fixed order.
template <int G, class V, class F>
FZD void group_row(int e0, int e1, const int *scol, const V *sw, F f) {
  const int lane = threadIdx.x & (G - 1);
  const int ea = min(e1, (e0 + 3) & ~3);
  if (e0 + lane < ea) f(scol[e0 + lane], sw[e0 + lane]);
  const int nq = (e1 - ea) >> 2;
#pragma unroll 2
  for (int q = lane; q < nq; q += G) {
    const int b = ea + 4 * q;
    const int4 c = *reinterpret_cast<const int4 *>(scol + b);
    if constexpr (sizeof(V) == 4) {
      const float4 w = *reinterpret_cast<const float4 *>(sw + b);
      f(c.x, (V)w.x);
      f(c.y, (V)w.y);
      f(c.z, (V)w.z);
      f(c.w, (V)w.w);
    } else {
      const double2 w0 = *reinterpret_cast<const double2 *>(sw + b);
      const double2 w1 = *reinterpret_cast<const double2 *>(sw + b + 2);
      f(c.x, (V)w0.x);
      f(c.y, (V)w0.y);
      f(c.z, (V)w1.x);
      f(c.w, (V)w1.y);
    }
  }
  const int eb = ea + 4 * nq;
  if (eb + lane < e1) f(scol[eb + lane], sw[eb + lane]);
}
template <class V, class F>
FZD void warp_row(int e0, int e1, const int *scol, const V *sw, F f) {
  group_row<32>(e0, e1, scol, sw, f);
}

// sum over an aligned group of G lanes (xor tree); result in every lane of it
template <int G, class V>
FZD V group_sum(V v) {
#pragma unroll
  for (int o = G >> 1; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <int G>
struct GroupSize {
  static constexpr int value = G;
};

// lanes per heavy row from the level's mean heavy-row length: short heavy
// rows share a warp (more rows in flight), long ones get a whole warp
FZD int heavy_group(const int *srp, int nl, int n) {
  const int nh = n - nl;
  if (nh <= 0) return 32;
  const int mean = (srp[n] - srp[nl]) / nh;
  return mean < 1024 ? 8 : mean < 4096 ? 16 : 32;
}
// calls f(GroupSize<G>{}) for the group size g (8, 16 or 32); the grid-wide
// engine has thousands of warps for the heavy rows and keeps to whole warps
template <bool GRID, class F>
FZD void with_group(int g, F f) {
  if constexpr (GRID) {
    f(GroupSize<32>{});
  } else {
    if (g == 8) f(GroupSize<8>{});
    else if (g == 16) f(GroupSize<16>{});
    else f(GroupSize<32>{});
  }
}

// Per-thread sum of a sweep's row values for the FP64 reductions.  With
// float iterates it is a float-float pair (hi + lo): every term goes in by
// Knuth's TwoSum and every product of two floats by TwoProduct (its rounding
// error from an FMA) before the TwoSum, so the pair holds the exact sum up
// to the roundings of lo, about 2^-48 of it per term.  GB300 issues FP64 at
// 1/56 of the FP32 rate with 64-cycle latency, and a row's four FP64 updates
// were the power iteration's throughput limit.  The pair goes into the FP64
// block sums.  With double iterates it is a plain double.
template <class V>
struct RowSum {
  double d = 0.0;
  FZD void add(V b) { d += (double)b; }
  FZD void add_prod(V a, V b) { d += (double)a * (double)b; }
  FZD double value() const { return d; }
};
template <>
struct RowSum<float> {
  float hi = 0.f, lo = 0.f;
  FZD void add(float b) {
    const float s = __fadd_rn(hi, b);
    const float bb = __fsub_rn(s, hi);
    lo += __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    hi = s;
  }
  FZD void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    add(p);
    lo += e;
  }
  FZD double value() const { return (double)hi + (double)lo; }
};

// warp sum of one value by a fixed xor tree; result in every lane
template <class V>
FZD V warp_sum(V v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP64 warp sum of K values by a fixed xor tree; result in every lane
template <int K>
FZD void warp_dsum(double (&v)[K]) {
#pragma unroll
  for (int k = 0; k < K; k++)
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}

// ---------------------------------------------------------------------------
// sorting of short segments: one thread (insertion) or one block (bitonic
// network for any length: merge blocks start with a reversed-partner step, so
// missing elements past len act as +infinity and are never touched)
template <class K>
FZD void thread_sort(K *a, int len) {
  for (int i = 1; i < len; i++) {
    K v = a[i];
    int j = i - 1;
    while (j >= 0 && a[j] > v) {
      a[j + 1] = a[j];
      j--;
    }
    a[j + 1] = v;
  }
}

template <class K>
FZD void block_bitonic(K *a, int len) {
  int P = 1;
  while (P < len) P <<= 1;
  for (int k = 2; k <= P; k <<= 1) {
    const int half = k >> 1;
    for (int p = threadIdx.x; p < (P >> 1); p += blockDim.x) {
      int blk = p / half, t = p - blk * half;
      int i = blk * k + t, j = blk * k + k - 1 - t;
      if (j < len) {
        K x = a[i], y = a[j];
        if (y < x) {
          a[i] = y;
          a[j] = x;
        }
      }
    }
    __syncthreads();
    for (int jj = k >> 2; jj >= 1; jj >>= 1) {
      for (int p = threadIdx.x; p < (P >> 1); p += blockDim.x) {
        int blk = p / jj, t = p - blk * jj;
        int i = blk * 2 * jj + t, j = i + jj;
        if (j < len) {
          K x = a[i], y = a[j];
          if (y < x) {
            a[i] = y;
            a[j] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// the same network run by one warp on a shared-memory segment (len <= 2^k)
template <class K>
FZD void warp_bitonic(K *a, int len) {
  const int lane = threadIdx.x & 31;
  int P = 1;
  while (P < len) P <<= 1;
  for (int k = 2; k <= P; k <<= 1) {
    const int half = k >> 1;
    for (int p = lane; p < (P >> 1); p += 32) {
      int blk = p / half, t = p - blk * half;
      int i = blk * k + t, j = blk * k + k - 1 - t;
      if (j < len) {
        K x = a[i], y = a[j];
        if (y < x) {
          a[i] = y;
          a[j] = x;
        }
      }
    }
    __syncwarp();
    for (int jj = k >> 2; jj >= 1; jj >>= 1) {
      for (int p = lane; p < (P >> 1); p += 32) {
        int blk = p / jj, t = p - blk * jj;
        int i = blk * 2 * jj + t, j = i + jj;
        if (j < len) {
          K x = a[i], y = a[j];
          if (y < x) {
            a[i] = y;
            a[j] = x;
          }
        }
      }
      __syncwarp();
    }
  }
}

// sorts g[0, len) (len <= kWarpSegG) by the calling warp: through its slice
// of the shared raw buffer up to kWarpSeg, in place beyond (__syncwarp orders
// the lanes' global accesses too)
template <class K>
FZD void warp_sort(K *g, int len) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // warps whose slice would lie beyond the raw buffer sort in place (the same order)
  if (len > kWarpSeg || (w + 1) * kWarpSeg * (int)sizeof(K) > kShSort * (int)sizeof(uint64_t)) {
    warp_bitonic(g, len);
    return;
  }
  K *s = reinterpret_cast<K *>(sh_raw()) + w * kWarpSeg;
  for (int i = lane; i < len; i += 32) s[i] = g[i];
  __syncwarp();
  warp_bitonic(s, len);
  for (int i = lane; i < len; i += 32) g[i] = s[i];
  __syncwarp();
}

template <class K>
FZD void block_sort(K *g, int len) {
  K *s = reinterpret_cast<K *>(sh_raw());
  const int cap = (int)(kShSort * sizeof(uint64_t) / sizeof(K));
  if (len <= cap) {
    for (int i = threadIdx.x; i < len; i += blockDim.x) s[i] = g[i];
    __syncthreads();
    block_bitonic(s, len);
    for (int i = threadIdx.x; i < len; i += blockDim.x) g[i] = s[i];
    __syncthreads();
  } else {
    block_bitonic(g, len);
  }
}

// ---------------------------------------------------------------------------
struct GalerkinScratch {
  int *cnt, *fill, *tcnt, *aggptr, *segptr, *members, *cc, *memoff, *dcnt;
  uint64_t *keys;
  double *segw;
};

// Jones-Plassmann colouring of one level, advanced one round per barrier
// (see Eng::jp_start); one copy per block in shared memory, written by
// thread 0 behind a block barrier
struct JPState {
  int active, ready, l, r, n, lo, hi;
  int *cround, *color;
  int *list[3];
  int *heavy;
  int *jpos;  // per blocked vertex: position of the neighbour that last blocked it
  long long visits;
};
FZD JPState &jps() {
  __shared__ JPState s;
  return s;
}

template <class T, bool GRID>
struct Eng {
  State *S;
  int tid, nthr, bid, nb, rb, kind;
  unsigned long long aoff, soff;
  uint64_t t_last;  // lead thread only
  unsigned ngen;    // grid barriers passed in this launch (same in every block)
  int cur_level;    // level being worked on (profile)
  // control flow, identical in every thread
  int nlevels, setup_done, coarsest, coarsest_solved, solved, finalized, refined;
  // grid form only: block 0 working alone (barriers and sums within the block)
  bool local_;

  // ---- infrastructure ------------------------------------------------------
  FZD void init(State *s) {
    S = s;
    // the one-block form treats its block as the whole grid, whichever block
    // of a batched launch it is
    bid = GRID ? blockIdx.x : 0;
    nb = GRID ? gridDim.x : 1;
    tid = GRID ? blockIdx.x * blockDim.x + threadIdx.x : threadIdx.x;
    nthr = GRID ? gridDim.x * blockDim.x : blockDim.x;
    rb = 0;
    kind = GRID ? 0 : 1;
    aoff = S->arena_off;
    soff = 0;
    nlevels = S->nlevels;
    setup_done = S->setup_done;
    coarsest = S->coarsest;
    coarsest_solved = S->coarsest_solved;
    solved = S->solved;
    finalized = S->finalized;
    refined = S->refined;
    t_last = 0;
    ngen = 0;
    cur_level = 0;
    local_ = false;
    if (threadIdx.x == 0) jps().active = 0;
    if (bid == 0) {
      for (int i = threadIdx.x; i < 2 * PH_COUNT + kMaxLevels * PH_COUNT; i += blockDim.x) sh_prof()[i] = 0.0;
      if (threadIdx.x == 0) t_last = gtime();
    }
    __syncthreads();
  }
  FZD bool lead() const { return bid == 0 && threadIdx.x == 0; }
  FZD void fail(int code) {
    atomicCAS(&S->failword, 0ull, ((unsigned long long)ngen << 32) | (unsigned)code);
    atomicCAS(&S->status, 0, code);
  }
  FZD int status() const { return *(volatile int *)&S->status; }
  FZD void persist() {
    if (lead()) {
      S->nlevels = nlevels;
      S->setup_done = setup_done;
      S->coarsest = coarsest;
      S->coarsest_solved = coarsest_solved;
      S->solved = solved;
      S->finalized = finalized;
      S->refined = refined;
      if (status() == 0) S->arena_off = aoff;
    }
  }
  FZD void flush_profile() {
    if (lead()) {
      for (int i = 0; i < PH_COUNT; i++) {
        S->phase_ns[kind][i] += sh_prof()[i];
        S->phase_bytes[kind][i] += sh_prof()[PH_COUNT + i];
      }
      for (int l = 0; l < kMaxLevels; l++)
        for (int i = 0; i < PH_COUNT; i++) S->level_ns[l][i] += sh_prof()[2 * PH_COUNT + l * PH_COUNT + i];
    }
  }

  FZD void *aalloc(unsigned long long bytes) {
    unsigned long long sz = (bytes + 255ull) & ~255ull;
    if (aoff + sz > S->arena_size) {
      fail(ST_ARENA);
      return nullptr;
    }
    void *p = S->arena + aoff;
    aoff += sz;
    return p;
  }
  FZD void *salloc(unsigned long long bytes) {
    unsigned long long sz = (bytes + 255ull) & ~255ull;
    if (soff + sz > S->scratch_size) {
      fail(ST_SCRATCH);
      return nullptr;
    }
    void *p = S->scratch + soff;
    soff += sz;
    return p;
  }

  // Barrier over every participating thread; false if the solve has failed.
  // Grid form: one atomic per block on a word whose top bit flips when the
  // last block arrives (block 0 adds 2^31 - (nb - 1), the others add 1, so the
  // low bits return to their start value), a bounded spin
  // (barrier_timeout_ns), and a verdict every block agrees on: a failure
  // counts at this barrier only if it was raised before it (failword carries
  // the number of barriers the failing block had passed).
  // plain barrier
  FZD bool sync() { return barrier(); }

  // barrier that also advances the colouring of the level being set up by one
  // round (used inside the matching, aggregation and Galerkin steps only)
  FZD bool sync_p() {
    JPState &jp = jps();
    if (jp.active && jp.ready) jp_round();
    const bool ok = barrier();
    if (ok && jp.active) {
      if (!jp.ready) {
        __syncthreads();
        if (threadIdx.x == 0) jp.ready = 1;
        __syncthreads();
      } else {
        jp_after();
      }
    }
    return ok;
  }

  FZD bool barrier() {
    if (!GRID || local_) return __syncthreads_and(status() == 0);
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned add = bid == 0 ? 0x80000000u - (unsigned)(nb - 1) : 1u;
      // the arrival releases the block's writes (ordered before it by the
      // block barrier, release is cumulative); the load that sees the flip
      // acquires every other block's
      const unsigned old = atom_add_release(&S->bar_word, add);
      bool done = (((old + add) ^ old) & 0x80000000u) != 0u;
      if (done) {
        fence_acquire();
      } else {
        const uint64_t t0 = gtime();
        const uint64_t lim = S->opt.barrier_timeout_ns;
        unsigned spins = 0;
        while (!done) {
          done = ((ld_acquire(&S->bar_word) ^ old) & 0x80000000u) != 0u;
          if (!done && (++spins & 255u) == 0u && gtime() - t0 > lim) break;
        }
      }
      if (!done) {
        fail(ST_ETIMEOUT);
        s_ok = 0;
      } else {
        const unsigned long long fw = *(volatile unsigned long long *)&S->failword;
        s_ok = fw == 0ull || (unsigned)(fw >> 32) > ngen;
      }
    }
    __syncthreads();
    ngen++;
    return s_ok != 0;
  }

  // profile: attribute the time since the last mark to phase ph (lead only)
  FZD void mark(int ph, double bytes) {
    const uint64_t t = gtime();
    const double dt = (double)(t - t_last);
    sh_prof()[ph] += dt;
    sh_prof()[PH_COUNT + ph] += bytes;
    sh_prof()[2 * PH_COUNT + cur_level * PH_COUNT + ph] += dt;
    t_last = t;
  }
#define FZ_MARK(ph, bytes)           \
  do {                               \
    if (lead()) mark((ph), (bytes)); \
  } while (0)

  FZD void chunk(long long n, int &lo, int &hi) const {
    long long ch = (n + nb - 1) / nb;
    long long a = (long long)bid * ch;
    if (a > n) a = n;
    long long b = a + ch;
    if (b > n) b = n;
    lo = (int)a;
    hi = (int)b;
  }

  // Integer grid reduction: sums a, b and maximum mx; pre_a / pre_b receive
  // the sums over the blocks before this one (chunked scans).
  template <bool PUMP = false>
  FZD bool grid_ired(IRed &r, long long *pre_a = nullptr, long long *pre_b = nullptr) {
    block_ired(r);
    long long pa = 0, pb = 0;
    if (GRID && !local_) {
      IRed *part = S->ipart + rb * kMaxBlocks;
      if (threadIdx.x == 0) part[bid] = r;
      if (!(PUMP ? sync_p() : sync())) return false;
      long long *s = sh_ll();
      if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        long long a = 0, b = 0, m = LLONG_MIN, qa = 0, qb = 0;
        for (int k = lane; k < nb; k += 32) {
          const IRed p = part[k];
          a += p.a;
          b += p.b;
          m = max(m, p.mx);
          if (k < bid) {
            qa += p.a;
            qb += p.b;
          }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
          qa += __shfl_xor_sync(0xffffffffu, qa, o);
          qb += __shfl_xor_sync(0xffffffffu, qb, o);
        }
        if (lane == 0) {
          s[0] = a;
          s[1] = b;
          s[2] = m;
          s[3] = qa;
          s[4] = qb;
        }
      }
      __syncthreads();
      r.a = s[0];
      r.b = s[1];
      r.mx = s[2];
      pa = s[3];
      pb = s[4];
      __syncthreads();
      rb ^= 1;
    } else {
      if (!(PUMP ? sync_p() : sync())) return false;
    }
    if (pre_a) *pre_a = pa;
    if (pre_b) *pre_b = pb;
    return true;
  }

  // FP64 grid sum of K <= 4 values (deterministic order)
  template <int K>
  FZD bool grid_dsum(double (&v)[K]) {
    block_dsum<K>(v);
    if (GRID && !local_) {
      double *part = S->dpart + (size_t)rb * kMaxBlocks * kDSum;
      if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; k++) part[bid * kDSum + k] = v[k];
      if (!sync()) return false;
      double *sh = reinterpret_cast<double *>(sh_raw());
      if (threadIdx.x < 32) {
        double a[K];
#pragma unroll
        for (int k = 0; k < K; k++) a[k] = 0.0;
        for (int b = threadIdx.x; b < nb; b += 32)
#pragma unroll
          for (int k = 0; k < K; k++) a[k] += part[b * kDSum + k];
#pragma unroll
        for (int k = 0; k < K; k++)
#pragma unroll
          for (int o = 16; o >= 1; o >>= 1) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
        if (threadIdx.x == 0)
#pragma unroll
          for (int k = 0; k < K; k++) sh[k] = a[k];
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < K; k++) v[k] = sh[k];
      __syncthreads();
      rb ^= 1;
    } else {
      if (!__syncthreads_and(status() == 0)) return false;
    }
    return true;
  }

  // FP64 grid sum of K <= kDSum values (the Krylov refinement's Gram sums):
  // warp xor trees, the block's warps in fixed order, then (grid form) the
  // blocks' partials in fixed order; result in every thread
  template <int K>
  FZD bool grid_wsum(double (&v)[K]) {
    static_assert(K >= 1 && K <= kDSum, "grid_wsum: K <= kDSum");
    double *sh = reinterpret_cast<double *>(sh_raw());  // [warps][K], then the K totals
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    warp_dsum<K>(v);
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < K; k++) sh[w * K + k] = v[k];
    __syncthreads();
    if (threadIdx.x < K) {
      double a = 0.0;
      for (int q = 0; q < nw; q++) a += sh[q * K + threadIdx.x];
      sh[32 * K + threadIdx.x] = a;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = sh[32 * K + k];
    __syncthreads();
    if (GRID && !local_) {
      double *part = S->dpart + (size_t)rb * kMaxBlocks * kDSum;
      if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; k++) part[bid * kDSum + k] = v[k];
      if (!sync()) return false;
      if (threadIdx.x < K) {
        double a = 0.0;
        for (int b = 0; b < nb; b++) a += part[b * kDSum + threadIdx.x];
        sh[threadIdx.x] = a;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < K; k++) v[k] = sh[k];
      __syncthreads();
      rb ^= 1;
    } else {
      if (!__syncthreads_and(status() == 0)) return false;
    }
    return true;
  }

  // setup weights: FP64 on coarse levels, the caller's float or double on the
  // fine level; key() gives the order-preserving bit pattern for comparisons
  struct W {
    const double *w64;
    const float *w32;
    FZD double operator[](int e) const { return w64 ? w64[e] : (double)w32[e]; }
    FZD uint64_t key(int e) const {
      return w64 ? (uint64_t)__double_as_longlong(w64[e]) : (uint64_t)__float_as_uint(w32[e]);
    }
  };
  FZD static W wof(const Level *L) { return W{L->w64, L->w32}; }

  // Small levels run in the one-block engine, large ones in the grid-wide
  // engine.  n and nnz never grow from a level to the next, so once a level
  // is small every coarser level is too.
  FZD static bool tiny(int n, int nnz) { return n <= kTinyN && nnz <= kTinyNnz; }
  FZD bool small(int n, int nnz) const {
    return tiny(n, nnz) || (n <= S->opt.tail_max_n && nnz <= S->opt.tail_max_nnz);
  }
  FZD bool elig(int n, int nnz) const { return GRID ? !small(n, nnz) : small(n, nnz); }
  // Value type of a level's solve weights and iterates: T, except that the
  // FP32 form keeps tiny levels in FP64.  Those levels are latency-bound (one
  // warp smooths them), so FP64 costs next to nothing there, and their
  // power-iteration stop decisions set the coarse start vector that the whole
  // cascade refines: one iteration more or less on a 51-vertex level moves
  // the final lambda2 of a 2048 x 1536 grid by 4e-5.  In FP64 those
  // decisions, and the tiny levels' vectors, are the FP64 form's own.
  FZD static bool vdbl(int n, int nnz) { return sizeof(T) == 8 || tiny(n, nnz); }

  FZD int wl_read(int slot) const { return *(volatile int *)&S->wl_cnt[slot]; }

  // ---- A1: ingest the fine level (Def 2.1) ---------------------------------
  FZD bool ingest() {
    const int n = S->n0, nnz = S->nnz0;
    const int *rp = S->in_rowptr, *ci = S->in_col;
    const bool wf64 = S->in_w_f64 != 0;
    const double *wd = (const double *)S->in_w;
    const float *wf = (const float *)S->in_w;
    const int validate = S->opt.validate;
    if (validate) {
      for (int i = tid; i <= n; i += nthr) {
        const int a = rp[i];
        const bool bad =
            a < 0 || a > nnz || (i == 0 && a != 0) || (i == n && a != nnz) || (i < n && rp[i + 1] < a);
        if (bad) {
          atomicMin((unsigned long long *)&S->bad_index, (unsigned long long)i);
          fail(ST_EINVAL);
        }
      }
      if (!sync()) return false;
    }
    double *d = (double *)aalloc(8ull * n);
    if (!d) return false;
    int lo, hi;
    chunk(n, lo, hi);
    IRed r{0, 0, 0};
    // entry checks: the column order, the weight, and the mirrored entry (a
    // binary search in row j for i); light rows one thread each, heavy rows
    // (degree >= kHeavyDeg) one warp each
    auto check = [&](int i, int e0, int e, int j, double w) {
      bool bad = j < 0 || j >= n || (e > e0 && ci[e - 1] >= j) || !isfinite(w) || (j != i && !(w > 0.0));
      if (!bad && j != i) {
        int a = rp[j], b = rp[j + 1] - 1, f = -1;
        while (a <= b) {
          const int m = (a + b) >> 1, cm = ci[m];
          if (cm == i) {
            f = m;
            break;
          }
          if (cm < i) a = m + 1;
          else b = m - 1;
        }
        bad = f < 0 || (wf64 ? wd[f] != wd[e] : wf[f] != wf[e]);
      }
      if (bad) {
        atomicMin((unsigned long long *)&S->bad_index, (unsigned long long)e);
        fail(ST_EINVAL);
      }
      return bad;
    };
    {
      const int lane = threadIdx.x & 31;
      for (int g0 = lo + (threadIdx.x >> 5) * 32; g0 < hi; g0 += blockDim.x) {
        const int i0 = g0 + lane;
        const bool hv = i0 < hi && rp[i0 + 1] - rp[i0] >= kHeavyDeg;
        unsigned mask = __ballot_sync(0xffffffffu, hv);
        while (mask) {
          const int i = g0 + __ffs(mask) - 1;
          mask &= mask - 1;
          const int e0 = rp[i], e1 = rp[i + 1];
          double di = 0.0;
          int loops = 0;
          bool bad = false;
          for (int e = e0 + lane; e < e1; e += 32) {
            const int j = ci[e];
            const double w = wf64 ? wd[e] : (double)wf[e];
            if (validate && check(i, e0, e, j, w)) bad = true;
            if (j == i) loops++;
            else di += w;
          }
          di = warp_sum(di);
          loops = warp_sum(loops);
          bad = __any_sync(0xffffffffu, bad);
          if (lane == 0 && !bad) {
            d[i] = di;
            r.a += e1 - e0 - loops;
            r.b += loops;
            r.mx = max(r.mx, (long long)__double_as_longlong(di));
          }
        }
      }
    }
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const int e0 = rp[i], e1 = rp[i + 1];
      if (e1 - e0 >= kHeavyDeg) continue;  // done by a warp above
      double di = 0.0;
      int loops = 0;
      for (int e = e0; e < e1; e++) {
        const int j = ci[e];
        const double w = wf64 ? wd[e] : (double)wf[e];
        if (validate && check(i, e0, e, j, w)) break;
        if (j == i) {
          loops++;
          continue;
        }
        di += w;
      }
      d[i] = di;
      r.a += e1 - e0 - loops;
      r.b += loops;
      r.mx = max(r.mx, (long long)__double_as_longlong(di));  // d >= 0: bit order = value order
    }
    long long pre = 0;
    if (!grid_ired(r, &pre)) return false;
    const long long m = r.a;
    const double maxd = __longlong_as_double(r.mx);
    int *rowptr = (int *)rp, *col = (int *)ci;
    double *w64 = wf64 ? (double *)wd : nullptr;
    float *w32 = wf64 ? nullptr : (float *)wf;
    if (r.b > 0) {  // drop self-loops
      rowptr = (int *)aalloc(4ull * (n + 1));
      col = (int *)aalloc(4ull * (m > 0 ? m : 1));
      void *wn = aalloc((wf64 ? 8ull : 4ull) * (m > 0 ? m : 1));
      if (!rowptr || !col || !wn) return false;
      w64 = wf64 ? (double *)wn : nullptr;
      w32 = wf64 ? nullptr : (float *)wn;
      long long run = pre;
      for (int t0 = lo; t0 < hi; t0 += blockDim.x) {
        const int i = t0 + threadIdx.x;
        int kept = 0;
        if (i < hi)
          for (int e = rp[i]; e < rp[i + 1]; e++) kept += ci[e] != i;
        int tot;
        const int ex = block_scan(kept, &tot);
        if (i < hi) {
          int o = (int)(run + ex);
          rowptr[i] = o;
          for (int e = rp[i]; e < rp[i + 1]; e++) {
            if (ci[e] == i) continue;
            col[o] = ci[e];
            if (wf64) w64[o] = wd[e];
            else w32[o] = wf[e];
            o++;
          }
        }
        run += tot;
      }
      if (lead()) rowptr[n] = (int)m;
    }
    if (lead()) {
      Level &L = S->lv[0];
      L.n = n;
      L.nnz = (int)m;
      L.rowptr = rowptr;
      L.col = col;
      L.w64 = w64;
      L.w32 = w32;
      L.d = d;
      L.sigma = 2.0 * maxd;
    }
    if (!sync()) return false;
    FZ_MARK(PH_INGEST, 12.0 * n + (4.0 + (wf64 ? 8.0 : 4.0)) * nnz * (validate ? 2.0 : 1.0));
    return true;
  }

  // ---- A6: Jones-Plassmann colouring, priority (h(v), v) --------------------
  // The colouring of level l runs alongside the matching, aggregation and
  // Galerkin steps of the same level (they do not depend on it): jp_start()
  // sets it up, and every barrier of those steps does one round first
  // (jp_round) and reads the round's outcome after passing (jp_after).  A round
  // colours every uncoloured vertex whose priority beats all neighbours still
  // uncoloured at the start of the round, with the smallest colour unused by
  // its neighbours coloured earlier.  Each block owns the vertices of its
  // chunk and keeps its own worklists (three rotating lists inside the chunk's
  // range, counters in shared memory); one global atomic per block per round
  // sums the survivors for the termination test, and the global counter of
  // list (r+2)%3 is cleared meanwhile (nobody uses it in round r).
  FZD bool jp_start(int l) {
    cur_level = l;
    Level *L = &S->lv[l];
    const int n = L->n;
    int *cround = (int *)salloc(4ull * n);
    int *list[3];
    for (int k = 0; k < 3; k++) list[k] = (int *)salloc(4ull * n);
    int *heavy = (int *)salloc(4ull * n);
    int *jpos = (int *)salloc(4ull * n);
    int *color = (int *)aalloc(4ull * n);
    if (!cround || !list[0] || !list[1] || !list[2] || !heavy || !jpos || !color) return false;
    int lo, hi;
    chunk(n, lo, hi);
    int *s_cnt = sh_ints() + 4;  // [0..2] block list counters, [3] block colour max
    for (int v = tid; v < n; v += nthr) cround[v] = INT_MAX;
    __syncthreads();
    if (threadIdx.x == 0) {
      s_cnt[0] = hi - lo;
      s_cnt[1] = 0;
      s_cnt[2] = 0;
      s_cnt[3] = -1;
      sh_hcnt()[0] = 0;
    }
    if (lead()) {
      S->jp_cnt[1] = 0;
      S->jp_cnt[2] = 0;
      S->col_max = -1;
      L->color = color;
    }
    if (threadIdx.x == 0) {
      JPState &jp = jps();
      jp.active = 1;
      jp.ready = 0;
      jp.l = l;
      jp.r = 0;
      jp.n = n;
      jp.lo = lo;
      jp.hi = hi;
      jp.cround = cround;
      jp.color = color;
      for (int k = 0; k < 3; k++) jp.list[k] = list[k];
      jp.heavy = heavy;
      jp.jpos = jpos;
      jp.visits = 0;
    }
    __syncthreads();
    return true;
  }

  FZN void jp_round() {
    JPState &jp = jps();
    const Level *L = &S->lv[jp.l];
    const int *rp = L->rowptr, *ci = L->col;
    int *cround = jp.cround, *color = jp.color;
    const int r = jp.r, lo = jp.lo;
    const int cur = r % 3, nxt = (r + 1) % 3, clr = (r + 2) % 3;
    int *s_cnt = sh_ints() + 4;
    if (lead() && r > 0) S->jp_cnt[clr] = 0;
    const int cnt = s_cnt[cur];
    int *lcur = jp.list[cur], *lnxt = jp.list[nxt];
    // threads in reverse order, so that on small levels the colouring runs on
    // other warps than the step it accompanies
    int *hc = sh_hcnt();
    int *hl = jp.heavy + lo;
    for (int q = blockDim.x - 1 - threadIdx.x; q < cnt; q += blockDim.x) {
      const int v = r == 0 ? lo + q : lcur[lo + q];
      const int e0 = rp[v], e1 = rp[v + 1];
      if (e1 - e0 >= kHeavyDeg) {  // to the warps
        hl[atomicAdd(&hc[0], 1)] = v;
        continue;
      }
      // a blocked vertex of degree >= kJposDeg resumes its scan at the
      // neighbour that blocked it: the neighbours before it had lower priority
      // or were coloured, and stay so, so only that one and the later ones can
      // block it now (short rows are cheaper to rescan than to remember)
      const uint64_t hv = vtx_hash(v);
      bool top = true;
      const bool keep = e1 - e0 >= kJposDeg;
      int e = (r == 0 || !keep) ? e0 : jp.jpos[v];
      for (; e < e1; e++) {
        const int u = ci[e];
        if (cround[u] >= r) {
          const uint64_t hu = vtx_hash(u);
          if (hu > hv || (hu == hv && u > v)) {
            top = false;
            break;
          }
        }
      }
      if (!top) {
        if (keep) jp.jpos[v] = e;
        lnxt[lo + atomicAdd(&s_cnt[nxt], 1)] = v;
        continue;
      }
      int base = 0, c = 0;
      for (;;) {
        uint64_t m = 0;
        for (int e = e0; e < e1; e++) {
          const int u = ci[e];
          if (cround[u] < r) {
            const int cu = color[u] - base;
            if (cu >= 0 && cu < 64) m |= 1ull << cu;
          }
        }
        if (m != ~0ull) {
          c = base + __ffsll((long long)~m) - 1;
          break;
        }
        base += 64;
      }
      color[v] = c;
      cround[v] = r;
      atomicMax(&s_cnt[3], c);
    }
    __syncthreads();
    {
      const int nh = hc[0];
      const int mean = L->nnz / (L->n > 0 ? L->n : 1);
      with_group<GRID>(mean < 128 ? 8 : mean < 512 ? 16 : 32, [&](auto gs) {
        constexpr int G = decltype(gs)::value, GW = 32 / G;
        const int gi = (threadIdx.x & 31) / G;
        for (int kb = (threadIdx.x >> 5) * GW; kb < nh; kb += (blockDim.x >> 5) * GW) {
          const int k = kb + gi;
          const bool valid = k < nh;
          jp_heavy_g<G>(valid ? hl[k] : 0, valid, r, rp, ci, cround, color, jp.jpos, lnxt + lo, &s_cnt[nxt],
                        &s_cnt[3]);
        }
      });
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (s_cnt[nxt]) atomicAdd(&S->jp_cnt[nxt], s_cnt[nxt]);
      if (s_cnt[3] >= 0) atomicMax(&S->col_max, s_cnt[3]);
      s_cnt[cur] = 0;  // becomes the append target of round r + 2
      hc[0] = 0;
      jp.visits += cnt;
    }
  }

  // One heavy vertex's colouring round, by an aligned group of G lanes
  // (several vertices in flight per warp): the same decision as the
  // one-thread path (top priority among the neighbours uncoloured at the start
  // of round r; smallest colour unused by neighbours coloured earlier), with
  // the neighbour scans split across the group.  Every lane of the warp calls it
  // (valid = false for lanes without a vertex); the loops run until no group
  // in the warp has work left, so the warp-wide votes see every lane.
  template <int G>
  FZD static void jp_heavy_g(int v, bool valid, int r, const int *rp, const int *ci, int *cround, int *color,
                             int *jpos, int *lnxt, int *cnt_nxt, int *cmax) {
    const int lane = threadIdx.x & 31, gl = lane & (G - 1), g0 = lane & ~(G - 1);
    const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << g0;
    const uint64_t hv = valid ? vtx_hash(v) : 0;
    const int e0 = valid ? rp[v] : 0, e1 = valid ? rp[v + 1] : 0;
    int b = valid ? (r == 0 ? e0 : jpos[v]) : 0;  // resume at the last blocker (see jp_round)
    bool active = valid && b < e1, beaten = false;
    while (__any_sync(0xffffffffu, active)) {
      bool beat = false;
      if (active) {
        const int e = b + gl;
        if (e < e1) {
          const int u = ci[e];
          if (cround[u] >= r) {
            const uint64_t hu = vtx_hash(u);
            beat = hu > hv || (hu == hv && u > v);
          }
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, beat) & gmask;
      if (active) {
        if (bal) {
          beaten = true;
          active = false;
          if (gl == 0) jpos[v] = b + __ffs(bal >> g0) - 1;  // the first blocker of the chunk
        } else {
          b += G;
          active = b < e1;
        }
      }
    }
    if (valid && beaten && gl == 0) lnxt[atomicAdd(cnt_nxt, 1)] = v;
    bool need = valid && !beaten;
    int base = 0;
    while (__any_sync(0xffffffffu, need)) {
      unsigned long long m = 0;
      if (need)
        for (int e = e0 + gl; e < e1; e += G) {
          const int u = ci[e];
          if (cround[u] < r) {
            const int cu = color[u] - base;
            if (cu >= 0 && cu < 64) m |= 1ull << cu;
          }
        }
#pragma unroll
      for (int o = G >> 1; o >= 1; o >>= 1) m |= __shfl_xor_sync(0xffffffffu, m, o);
      if (need) {
        if (m != ~0ull) {
          const int c = base + __ffsll((long long)~m) - 1;
          need = false;
          if (gl == 0) {
            color[v] = c;
            cround[v] = r;
            atomicMax(cmax, c);
          }
        } else {
          base += 64;
        }
      }
    }
  }

  FZN void jp_after() {
    JPState &jp = jps();
    const int r = jp.r, l = jp.l;
    const int left = *(volatile int *)&S->jp_cnt[(r + 1) % 3];
    __syncthreads();
    if (left != 0) {
      if (threadIdx.x == 0) jp.r = r + 1;
      __syncthreads();
      return;
    }
    const int ncol = *(volatile int *)&S->col_max + 1;
    if (2 * ncol > kMaxColors) fail(ST_ENOTSUP);  // the reorder buckets (colour, heavy)
    if (lead()) {
      Level *L = &S->lv[l];
      L->ncolors = ncol;
      L->color_rounds = r + 1;
    }
    if (threadIdx.x == 0) jp.active = 0;
    __syncthreads();
  }

  // run the remaining colouring rounds on their own barriers
  FZD bool jp_finish() {
    while (jps().active)
      if (!sync_p()) return false;
    if (!sync()) return false;  // publishes ncolors / color_rounds
    const Level *L = &S->lv[jps().l];
    FZ_MARK(PH_COLOR, 8.0 * L->n + (double)jps().visits * 12.0 * nb + 4.0 * L->nnz);
    return true;
  }

  // ---- colour-order copy of the level for the solve phase -------------------
  // Solve order: every light row (degree < kHeavyDeg) before every heavy
  // row; within each group colour classes in ascending order, each in
  // ascending vertex order.  Bucket b = heavy * C + colour (C colours);
  // colstart[b] is the first solve position of bucket b (2C + 1 entries):
  // light rows of colour c at [colstart[c], colstart[c + 1]), heavy rows of
  // colour c at [colstart[C + c], colstart[C + c + 1]).
  FZD bool reorder(int l) {
    cur_level = l;
    Level *L = &S->lv[l];
    const int n = L->n, nnz = L->nnz, C = 2 * L->ncolors;
    const int *rp = L->rowptr, *ci = L->col, *color = L->color;
    const int C0 = L->ncolors;
    auto bucket = [&](int v) { return (rp[v + 1] - rp[v] >= kHeavyDeg ? C0 : 0) + color[v]; };
    int *hist = (int *)salloc(4ull * C * nb);
    int *perm = (int *)aalloc(4ull * n);
    int *iperm = (int *)aalloc(4ull * n);
    int *colstart = (int *)aalloc(4ull * (C + 1));
    int *srp = (int *)aalloc(4ull * (n + 1));
    int *scol = (int *)aalloc(4ull * (nnz > 0 ? nnz : 1));
    const bool vd = vdbl(n, nnz);
    const unsigned long long vsz = vd ? 8ull : sizeof(T);
    void *sw = aalloc(vsz * (unsigned long long)(nnz > 0 ? nnz : 1));
    void *x = aalloc(vsz * (unsigned long long)n);
    void *y = aalloc(vsz * (unsigned long long)n);
    int *sagg = (int *)aalloc(4ull * n);
    if (!hist || !perm || !iperm || !colstart || !srp || !scol || !sw || !x || !y || !sagg) return false;
    int *sh_cnt = reinterpret_cast<int *>(sh_raw());                     // [kMaxColors]
    int *sh_base = sh_cnt + kMaxColors;                                 // [kMaxColors]
    int(*wc)[64] = reinterpret_cast<int(*)[64]>(sh_base + kMaxColors);  // [32][64], C <= 64 only
    int lo, hi;
    chunk(n, lo, hi);
    for (int c = threadIdx.x; c < C; c += blockDim.x) sh_cnt[c] = 0;
    __syncthreads();
    for (int v = lo + threadIdx.x; v < hi; v += blockDim.x) atomicAdd(&sh_cnt[bucket(v)], 1);
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) hist[(size_t)c * nb + bid] = sh_cnt[c];
    if (!sync()) return false;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
      int t = 0, p = 0;
      for (int b = 0; b < nb; b++) {
        const int h = hist[(size_t)c * nb + b];
        t += h;
        if (b < bid) p += h;
      }
      sh_cnt[c] = t;
      sh_base[c] = p;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int c = 0; c < C; c++) {
        if (bid == 0) colstart[c] = acc;
        sh_base[c] += acc;
        acc += sh_cnt[c];
      }
      if (bid == 0) colstart[C] = acc;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (C <= 64) {
      for (int t0 = lo; t0 < hi; t0 += blockDim.x) {
        const int v = t0 + threadIdx.x;
        const int cv = v < hi ? bucket(v) : -1;
        for (int k = threadIdx.x; k < nw * 64; k += blockDim.x) wc[k >> 6][k & 63] = 0;
        __syncthreads();
        const unsigned peers = __match_any_sync(0xffffffffu, cv);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (cv >= 0 && rank == 0) wc[w][cv] = __popc(peers);
        __syncthreads();
        if (threadIdx.x < C) {
          const int c = threadIdx.x;
          int acc = sh_base[c];
          for (int ww = 0; ww < nw; ww++) {
            const int t = wc[ww][c];
            wc[ww][c] = acc;
            acc += t;
          }
          sh_base[c] = acc;
        }
        __syncthreads();
        if (cv >= 0) {
          const int pos = wc[w][cv] + rank;
          perm[pos] = v;
          iperm[v] = pos;
        }
        __syncthreads();
      }
    } else {
      for (int t0 = lo; t0 < hi; t0 += blockDim.x) {
        const int v = t0 + threadIdx.x;
        const int cv = v < hi ? bucket(v) : -1;
        for (int c = 0; c < C; c++) {
          if (!__syncthreads_or(cv == c)) continue;
          int tot;
          const int ex = block_scan(cv == c, &tot);
          if (cv == c) {
            const int pos = sh_base[c] + ex;
            perm[pos] = v;
            iperm[v] = pos;
          }
          __syncthreads();
          if (threadIdx.x == 0) sh_base[c] += tot;
          __syncthreads();
        }
      }
    }
    if (!sync()) return false;
    // row pointers of the colour-order copy
    IRed red{0, 0, 0};
    for (int k = lo + threadIdx.x; k < hi; k += blockDim.x) {
      const int v = perm[k];
      red.a += rp[v + 1] - rp[v];
    }
    long long pre = 0;
    if (!grid_ired(red, &pre)) return false;
    long long run = pre;
    const W wl = wof(L);
    for (int t0 = lo; t0 < hi; t0 += blockDim.x) {
      const int k = t0 + threadIdx.x;
      const int v = k < hi ? perm[k] : 0;
      const int deg = k < hi ? rp[v + 1] - rp[v] : 0;
      int tot;
      const int ex = block_scan(deg, &tot);
      if (k < hi) {
        int o = (int)(run + ex);
        srp[k] = o;
        for (int e = rp[v]; e < rp[v + 1]; e++, o++) {
          scol[o] = iperm[ci[e]];
          if (vd) ((double *)sw)[o] = wl[e];
          else ((T *)sw)[o] = (T)wl[e];
        }
      }
      run += tot;
    }
    if (lead()) srp[n] = nnz;
    // solve positions of the previous level map through this level's order
    if (l > 0) {
      Level *F = &S->lv[l - 1];
      const int nf = F->n;
      const int *fperm = F->perm, *fagg = F->agg;
      int *fsagg = F->sagg;
      for (int k = tid; k < nf; k += nthr) fsagg[k] = iperm[fagg[fperm[k]]];
    }
    if (lead()) {
      L->perm = perm;
      L->iperm = iperm;
      L->colstart = colstart;
      L->srowptr = srp;
      L->scol = scol;
      L->sw = sw;
      L->x = x;
      L->y = y;
      L->sagg = sagg;
    }
    if (!sync()) return false;
    FZ_MARK(PH_REORDER, 28.0 * n + (8.0 + (L->w64 ? 8.0 : 4.0) + 4.0 + vsz) * nnz);
    return true;
  }

  // ---- A2: heavy-edge matching by handshake rounds ---------------------------
  // Round k: every active vertex picks its best free neighbour under K; mutual
  // picks become pairs; the others stay active, and a vertex left without a
  // free neighbour drops out (the free set only shrinks, so it never gets one
  // again).  Phase k settles the pairs of round k - 1 and makes the picks of
  // round k in one pass over block-owned worklists, so one barrier separates
  // two rounds.  The picks live in two buffers (round parity) as (round << 32 |
  // vertex): during phase k a vertex u counts as taken iff it was matched
  // before round k - 1 (mate) or its round-(k - 1) pick points at a vertex whose
  // round-(k - 1) pick points back at u.  Stop after a phase with no pick.
  FZD bool match(int l) {
    cur_level = l;
    Level *L = &S->lv[l];
    const int n = L->n;
    const int *rp = L->rowptr, *ci = L->col;
    const int tie = S->opt.tie_rule;
    const W wl = wof(L);
    int *mate = (int *)aalloc(4ull * n);
    unsigned long long *pick[2];
    for (int k = 0; k < 2; k++) pick[k] = (unsigned long long *)salloc(8ull * n);
    int *list[3];
    for (int k = 0; k < 3; k++) list[k] = (int *)salloc(4ull * n);
    int *heavy = (int *)salloc(4ull * n);
    if (!mate || !pick[0] || !pick[1] || !list[0] || !list[1] || !list[2] || !heavy) return false;
    int lo, hi;
    chunk(n, lo, hi);
    int *s_cnt = sh_ints();
    int *hc = sh_hcnt();
    int *hl = heavy + lo;
    if (threadIdx.x == 0) {
      s_cnt[0] = hi - lo;
      s_cnt[1] = 0;
      s_cnt[2] = 0;
      hc[1] = 0;
    }
    if (lead()) {
      S->wl_cnt[1] = 0;
      S->wl_cnt[2] = 0;
      L->mate = mate;  // published by the barrier below; complete after the last phase's
    }
    constexpr unsigned long long kNoPick = ~0ull;  // round tag 2^32 - 1: never current
    for (int v = tid; v < n; v += nthr) {
      mate[v] = -1;
      pick[0][v] = kNoPick;
      pick[1][v] = kNoPick;
    }
    if (!sync_p()) return false;
    int rounds = 0;
    long long visits = 0;
    for (int ph = 0;; ph++) {
      const int cur = ph % 3, nxt = (ph + 1) % 3, clr = (ph + 2) % 3;
      if (lead() && ph > 0) S->wl_cnt[clr] = 0;
      const int cnt = s_cnt[cur];
      const unsigned long long *pp = pick[(ph + 1) & 1];  // round ph - 1
      unsigned long long *pn = pick[ph & 1];              // round ph
      const unsigned long long tprev = (unsigned long long)(unsigned)(ph - 1) << 32;
      const unsigned long long tcur = (unsigned long long)(unsigned)ph << 32;
      auto taken = [&](int u) {
        if (ph == 0) return false;
        if (mate[u] >= 0) return true;
        const unsigned long long a = pp[u];
        if ((a >> 32) != (tprev >> 32)) return false;
        return pp[(unsigned)a] == (tprev | (unsigned)u);
      };
      for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int v = ph == 0 ? lo + q : list[cur][lo + q];
        if (ph > 0) {
          // v picked in round ph - 1 (that is why it is on the list)
          const int c = (int)(unsigned)pp[v];
          if (pp[c] == (tprev | (unsigned)v)) {  // a pair of round ph - 1
            mate[v] = c;
            continue;
          }
          if (!taken(c)) {
            // the best free neighbour of the last pick is still free, and the
            // free set only shrinks, so it is still the best: no rescan
            pn[v] = tcur | (unsigned)c;
            list[nxt][lo + atomicAdd(&s_cnt[nxt], 1)] = v;
            continue;
          }
        }
        if (rp[v + 1] - rp[v] >= kHeavyDeg) {  // to the warps
          hl[atomicAdd(&hc[1], 1)] = v;
          continue;
        }
        Best b;
        best_init(b);
        for (int e = rp[v]; e < rp[v + 1]; e++) {
          const int u = ci[e];
          if (taken(u)) continue;
          const uint64_t wk = wl.key(e);
          if (best_beats(b, wk, v, u, tie)) best_set(b, wk, v, u);
        }
        if (b.v >= 0) {
          pn[v] = tcur | (unsigned)b.v;
          list[nxt][lo + atomicAdd(&s_cnt[nxt], 1)] = v;
        }
      }
      __syncthreads();
      // heavy vertices: one warp each, lanes over the neighbours, then the
      // warp's best under the same total order (unique, so the merge order
      // does not matter)
      const int nh = hc[1];
      const int lane = threadIdx.x & 31;
      const int mean = L->nnz / (n > 0 ? n : 1);
      with_group<GRID>(mean < 128 ? 8 : mean < 512 ? 16 : 32, [&](auto gs) {
        constexpr int G = decltype(gs)::value, GW = 32 / G;
        const int gl = lane & (G - 1), gi = lane / G;
        for (int kb = (threadIdx.x >> 5) * GW; kb < nh; kb += (blockDim.x >> 5) * GW) {
          const int k = kb + gi;
          const int v = k < nh ? hl[k] : 0;
          Best b;
          best_init(b);
          b.wk = 0;
          if (k < nh)
            for (int e = rp[v] + gl; e < rp[v + 1]; e += G) {
              const int u = ci[e];
              if (taken(u)) continue;
              const uint64_t wk = wl.key(e);
              if (best_beats(b, wk, v, u, tie)) best_set(b, wk, v, u);
            }
          for (int o = G >> 1; o >= 1; o >>= 1) {
            const uint64_t owk = __shfl_xor_sync(0xffffffffu, b.wk, o);
            const int ov = __shfl_xor_sync(0xffffffffu, b.v, o);
            if (ov >= 0 && best_beats(b, owk, v, ov, tie)) best_set(b, owk, v, ov);
          }
          if (k < nh && gl == 0 && b.v >= 0) {
            pn[v] = tcur | (unsigned)b.v;
            list[nxt][lo + atomicAdd(&s_cnt[nxt], 1)] = v;
          }
        }
      });
      __syncthreads();
      if (threadIdx.x == 0) {
        if (s_cnt[nxt]) atomicAdd(&S->wl_cnt[nxt], s_cnt[nxt]);
        s_cnt[cur] = 0;
        hc[1] = 0;
      }
      visits += cnt;
      if (!sync_p()) return false;
      if (wl_read(nxt) == 0) break;  // no pick: the last pairs are settled
      rounds++;
    }
    if (lead()) L->match_rounds = rounds;
    FZ_MARK(PH_MATCH, 20.0 * n + (double)visits * nb * (8.0 + 4.0 * 4 + 8.0 * 2 + (L->w64 ? 8.0 : 4.0) * 4));
    return true;
  }

  // ---- A3: aggregates from the matching; returns nc (or -1: stop coarsening)
  FZD bool aggregate(int l, int &nc_out, GalerkinScratch &G) {
    cur_level = l;
    Level *L = &S->lv[l];
    const int n = L->n;
    const int *rp = L->rowptr, *ci = L->col, *mate = L->mate;
    const int tie = S->opt.tie_rule;
    const W wl = wof(L);
    const double stall = S->opt.stall_ratio;
    int lo, hi;
    chunk(n, lo, hi);
    IRed red{0, 0, 0};
    for (int v = lo + threadIdx.x; v < hi; v += blockDim.x) {
      const int m = mate[v];
      red.a += (m >= 0) ? (v < m) : (rp[v + 1] == rp[v]);
    }
    long long pre = 0;
    if (!grid_ired<true>(red, &pre)) return false;
    const long long nc = red.a;
    nc_out = -1;
    if (nc < 2 || (double)nc > stall * (double)n) return true;
    int *agg = (int *)aalloc(4ull * n);
    G.cnt = (int *)salloc(4ull * nc);
    G.fill = (int *)salloc(4ull * nc);
    G.tcnt = (int *)salloc(4ull * nc);
    G.aggptr = (int *)salloc(4ull * (nc + 1));
    G.segptr = (int *)salloc(4ull * (nc + 1));
    G.dcnt = (int *)salloc(4ull * nc);
    G.members = (int *)salloc(4ull * n);
    G.cc = (int *)salloc(4ull * n);
    G.memoff = (int *)salloc(4ull * n);
    if (!agg || !G.cnt || !G.fill || !G.tcnt || !G.aggptr || !G.segptr || !G.dcnt || !G.members || !G.cc ||
        !G.memoff)
      return false;
    long long run = pre;
    for (int t0 = lo; t0 < hi; t0 += blockDim.x) {
      const int v = t0 + threadIdx.x;
      int f = 0;
      if (v < hi) {
        const int m = mate[v];
        f = (m >= 0) ? (v < m) : (rp[v + 1] == rp[v]);
      }
      int tot;
      const int ex = block_scan(f, &tot);
      if (f) agg[v] = (int)(run + ex);
      run += tot;
    }
    for (long long I = tid; I < nc; I += nthr) {
      G.cnt[I] = 0;
      G.fill[I] = 0;
      G.tcnt[I] = 0;
    }
    if (!sync_p()) return false;
    for (int v = tid; v < n; v += nthr) {
      const int m = mate[v];
      int a;
      if (m >= 0) {
        a = agg[v < m ? v : m];
        if (v > m) agg[v] = a;
      } else if (rp[v + 1] == rp[v]) {
        a = agg[v];
      } else {
        Best b;
        best_init(b);
        for (int e = rp[v]; e < rp[v + 1]; e++) {
          const int u = ci[e];
          const uint64_t wk = wl.key(e);
          if (best_beats(b, wk, v, u, tie)) best_set(b, wk, v, u);
        }
        const int u = b.v, mu = mate[u];
        if (mu < 0) {  // matching not maximal: cannot happen
          fail(ST_EINVAL);
          a = 0;
        } else {
          a = agg[u < mu ? u : mu];
        }
        agg[v] = a;
      }
      atomicAdd(&G.cnt[a], 1);
    }
    if (lead()) {  // published before the barrier: the Galerkin phase reads it
      L->agg = agg;
      L->nc = (int)nc;
    }
    if (!sync_p()) return false;
    FZ_MARK(PH_AGG, 24.0 * n + 12.0 * L->nnz);
    nc_out = (int)nc;
    return true;
  }

  // ---- A2 + A3, Alg. 1 as printed (hec_mode PAPER) -------------------------
  // The sequential greedy: vertices visited in ascending order of the keys
  // (splitmix64(seed + l, v), v); an unaggregated vertex u takes m(u), its
  // heaviest neighbour (lowest index on ties); it founds the aggregate
  // {u, m(u)} if m(u) is unaggregated, else joins m(u)'s aggregate; a vertex
  // without neighbours founds a singleton; aggregate ids count up in visit
  // order.  Reproduced exactly by rounds: A(u) = "u is unaggregated at its
  // turn" is false iff some earlier v with m(v) = u has A(v) (decided once
  // every such v is decided; the earliest undecided vertex is always
  // decidable); first(u) = the earliest v with A(v) and m(v) = u took u (if u
  // was not earlier than it) or joined it; u with A(u) founds iff m(u) < 0 or
  // (u precedes m(u) and first(m(u)) = u), else joins m(u); an u without A(u)
  // belongs to first(u)'s aggregate; joins are followed by pointer jumping
  // (chains of m end in a founder: m has no cycles longer than two), and the
  // founders are numbered in visit order by a bucket sort of their keys.
  FZN bool hec_paper(int l, int &nc_out, GalerkinScratch &G) {
    cur_level = l;
    Level *L = &S->lv[l];
    const int n = L->n;
    const int *rp = L->rowptr, *ci = L->col;
    const W wl = wof(L);
    const uint64_t seed = S->opt.seed + (uint64_t)l;
    const double stall = S->opt.stall_ratio;
    int *hm = (int *)salloc(4ull * n);
    int *st = (int *)salloc(4ull * n);  // 0 undecided, 1 A(u), 2 not A(u)
    unsigned long long *fk = (unsigned long long *)salloc(8ull * n);
    int *fv = (int *)salloc(4ull * n);
    int *lab = (int *)salloc(4ull * n);
    int *fid = (int *)salloc(4ull * n);
    if (!hm || !st || !fk || !fv || !lab || !fid) return false;
    auto key = [&](int v) { return sm64(seed, (uint64_t)(uint32_t)v); };
    auto before = [&](int a, uint64_t ka, int b, uint64_t kb) { return ka < kb || (ka == kb && a < b); };
    // m(v): heaviest neighbour, lowest index among equal weights (columns ascend)
    for (int v = tid; v < n; v += nthr) {
      int m = -1;
      uint64_t bk = 0;
      for (int e = rp[v]; e < rp[v + 1]; e++) {
        const uint64_t wk = wl.key(e);
        if (m < 0 || wk > bk) {
          bk = wk;
          m = ci[e];
        }
      }
      hm[v] = m;
      st[v] = 0;
      fk[v] = ~0ull;
      fv[v] = INT_MAX;
    }
    if (!sync_p()) return false;
    int rounds = 0;
    for (;; rounds++) {
      IRed red{0, 0, 0};
      for (int u = tid; u < n; u += nthr) {
        if (st[u] != 0) continue;
        const uint64_t ku = key(u);
        bool pend = false, killed = false;
        for (int e = rp[u]; e < rp[u + 1]; e++) {
          const int v = ci[e];
          if (hm[v] != u || !before(v, key(v), u, ku)) continue;
          const int sv = *(volatile int *)&st[v];
          if (sv == 1) {
            killed = true;
            break;
          }
          if (sv == 0) pend = true;
        }
        if (killed) st[u] = 2;
        else if (!pend) st[u] = 1;
        else red.a++;
      }
      if (!grid_ired<true>(red)) return false;
      if (red.a == 0) break;
      if (rounds > n) {
        fail(ST_EINVAL);
        return false;
      }
    }
    // first(m): the earliest vertex with A that points at m
    for (int w = tid; w < n; w += nthr)
      if (st[w] == 1 && hm[w] >= 0) atomicMin(&fk[hm[w]], (unsigned long long)key(w));
    if (!sync_p()) return false;
    for (int w = tid; w < n; w += nthr)
      if (st[w] == 1 && hm[w] >= 0 && (unsigned long long)key(w) == fk[hm[w]]) atomicMin(&fv[hm[w]], w);
    if (!sync_p()) return false;
    // founders, and a label per vertex: founders themselves, joiners m(u),
    // the others the founder that took them
    IRed nf_red{0, 0, 0};
    for (int u = tid; u < n; u += nthr) {
      int lb;
      bool founder = false;
      if (st[u] == 1) {
        const int m = hm[u];
        founder = m < 0 || (before(u, key(u), m, key(m)) && fv[m] == u);
        lb = founder ? u : m;
      } else {
        lb = fv[u];
      }
      lab[u] = lb;
      fid[u] = founder ? 1 : 0;
      nf_red.a += founder;
    }
    if (!grid_ired<true>(nf_red)) return false;
    const long long nc = nf_red.a;
    for (;;) {
      IRed red{0, 0, 0};
      for (int u = tid; u < n; u += nthr) {
        const int a = lab[u], b = lab[a];
        if (b != a) {
          lab[u] = b;
          red.a++;
        }
      }
      if (!grid_ired<true>(red)) return false;
      if (red.a == 0) break;
    }
    nc_out = -1;
    if (lead()) {
      L->mate = nullptr;
      L->match_rounds = rounds;
    }
    if (nc < 2 || (double)nc > stall * (double)n) return sync_p();
    // founders in visit order: buckets by the top kb bits of the key
    int kb = 1;
    while (kb < 30 && (1ll << kb) < nc) kb++;
    const int B = 1 << kb;
    int *bcnt = (int *)salloc(4ull * B);
    int *bst = (int *)salloc(4ull * (B + 1));
    int *slot = (int *)salloc(4ull * nc);
    if (!bcnt || !bst || !slot) return false;
    for (int b = tid; b < B; b += nthr) bcnt[b] = 0;
    if (!sync_p()) return false;
    for (int u = tid; u < n; u += nthr)
      if (fid[u]) atomicAdd(&bcnt[(int)(key(u) >> (64 - kb))], 1);
    if (!sync_p()) return false;
    {
      int lo, hi;
      chunk(B, lo, hi);
      IRed red{0, 0, 0};
      for (int b = lo + threadIdx.x; b < hi; b += blockDim.x) red.a += bcnt[b];
      long long pre = 0;
      if (!grid_ired<true>(red, &pre)) return false;
      long long run = pre;
      for (int t0 = lo; t0 < hi; t0 += blockDim.x) {
        const int b = t0 + threadIdx.x;
        const int c = b < hi ? bcnt[b] : 0;
        int tot;
        const int ex = block_scan(c, &tot);
        if (b < hi) bst[b] = (int)(run + ex);
        run += tot;
      }
      if (lead()) bst[B] = (int)nc;
    }
    // every block has read its chunk of the counts before any clears them
    if (!sync_p()) return false;
    for (int b = tid; b < B; b += nthr) bcnt[b] = 0;
    if (!sync_p()) return false;
    for (int u = tid; u < n; u += nthr)
      if (fid[u]) {
        const int b = (int)(key(u) >> (64 - kb));
        slot[bst[b] + atomicAdd(&bcnt[b], 1)] = u;
      }
    if (!sync_p()) return false;
    // each bucket in key order (insertion sort: buckets hold ~1 founder)
    for (int b = tid; b < B; b += nthr) {
      const int s0 = bst[b], s1 = bst[b + 1];
      for (int i = s0 + 1; i < s1; i++) {
        const int v = slot[i];
        const uint64_t kv = key(v);
        int j = i - 1;
        while (j >= s0 && before(v, kv, slot[j], key(slot[j]))) {
          slot[j + 1] = slot[j];
          j--;
        }
        slot[j + 1] = v;
      }
    }
    if (!sync_p()) return false;
    for (int p = tid; p < nc; p += nthr) fid[slot[p]] = p;
    if (!sync_p()) return false;
    int *agg = (int *)aalloc(4ull * n);
    G.cnt = (int *)salloc(4ull * nc);
    G.fill = (int *)salloc(4ull * nc);
    G.tcnt = (int *)salloc(4ull * nc);
    G.aggptr = (int *)salloc(4ull * (nc + 1));
    G.segptr = (int *)salloc(4ull * (nc + 1));
    G.dcnt = (int *)salloc(4ull * nc);
    G.members = (int *)salloc(4ull * n);
    G.cc = (int *)salloc(4ull * n);
    G.memoff = (int *)salloc(4ull * n);
    if (!agg || !G.cnt || !G.fill || !G.tcnt || !G.aggptr || !G.segptr || !G.dcnt || !G.members || !G.cc ||
        !G.memoff)
      return false;
    for (long long I = tid; I < nc; I += nthr) {
      G.cnt[I] = 0;
      G.fill[I] = 0;
      G.tcnt[I] = 0;
    }
    if (!sync_p()) return false;
    for (int u = tid; u < n; u += nthr) {
      const int a = fid[lab[u]];
      agg[u] = a;
      atomicAdd(&G.cnt[a], 1);
    }
    if (lead()) {  // published before the barrier: the Galerkin phase reads it
      L->agg = agg;
      L->nc = (int)nc;
    }
    if (!sync_p()) return false;
    FZ_MARK(PH_MATCH, (4.0 * (n + 1) + (4.0 + (L->w64 ? 8.0 : 4.0)) * L->nnz) * (2.0 + rounds) + 60.0 * n);
    nc_out = (int)nc;
    return true;
  }

  // ---- A4: Galerkin coarse operator I L I^T ---------------------------------
  FZD bool galerkin(int l, int nc, GalerkinScratch &G) {
    cur_level = l;
    Level *L = &S->lv[l];
    const int n = L->n;
    const int *rp = L->rowptr, *ci = L->col;
    const int *agg = L->agg;
    const W wl = wof(L);
    // G1: cross-aggregate entries per fine row and per aggregate (heavy rows
    // by a warp each, found by the warps in groups of 32 rows)
    const int lane = threadIdx.x & 31, gw = tid >> 5, nwarp = nthr >> 5;
    for (int v = tid; v < n; v += nthr) {
      if (rp[v + 1] - rp[v] >= kHeavyDeg) continue;
      const int I = agg[v];
      int k = 0;
      for (int e = rp[v]; e < rp[v + 1]; e++) k += agg[ci[e]] != I;
      G.cc[v] = k;
      if (k) atomicAdd(&G.tcnt[I], k);
    }
    for (int g0 = gw * 32; g0 < n; g0 += nwarp * 32) {
      const int v0 = g0 + lane;
      unsigned mask = __ballot_sync(0xffffffffu, v0 < n && rp[v0 + 1] - rp[v0] >= kHeavyDeg);
      while (mask) {
        const int v = g0 + __ffs(mask) - 1;
        mask &= mask - 1;
        const int I = agg[v];
        int k = 0;
        for (int e = rp[v] + lane; e < rp[v + 1]; e += 32) k += agg[ci[e]] != I;
        k = warp_sum(k);
        if (lane == 0) {
          G.cc[v] = k;
          if (k) atomicAdd(&G.tcnt[I], k);
        }
      }
    }
    if (!sync_p()) return false;
    // G2: member and segment pointers (chunked scans over aggregates)
    int lo, hi;
    chunk(nc, lo, hi);
    IRed red{0, 0, 0};
    for (int I = lo + threadIdx.x; I < hi; I += blockDim.x) {
      red.a += G.cnt[I];
      red.b += G.tcnt[I];
    }
    long long preA = 0, preB = 0;
    if (!grid_ired<true>(red, &preA, &preB)) return false;
    const long long ttot = red.b;
    {
      long long ra = preA, rbb = preB;
      for (int t0 = lo; t0 < hi; t0 += blockDim.x) {
        const int I = t0 + threadIdx.x;
        const int a = I < hi ? G.cnt[I] : 0, b = I < hi ? G.tcnt[I] : 0;
        int ta, tb;
        const int ea = block_scan(a, &ta);
        const int eb = block_scan(b, &tb);
        if (I < hi) {
          G.aggptr[I] = (int)(ra + ea);
          G.segptr[I] = (int)(rbb + eb);
        }
        ra += ta;
        rbb += tb;
      }
      if (lead()) {
        G.aggptr[nc] = n;
        G.segptr[nc] = (int)ttot;
      }
    }
    G.keys = (uint64_t *)salloc(8ull * (ttot > 0 ? ttot : 1));
    G.segw = (double *)salloc(8ull * (ttot > 0 ? ttot : 1));
    if (!G.keys || !G.segw) return false;
    if (!sync_p()) return false;
    // G3: members of each aggregate
    for (int v = tid; v < n; v += nthr) {
      const int I = agg[v];
      const int s = atomicAdd(&G.fill[I], 1);
      G.members[G.aggptr[I] + s] = v;
    }
    if (!sync_p()) return false;
    // G4: members ascending; offset of each member's entries inside its segment
    // (short member lists by one thread, medium ones by one warp, long ones by
    // the whole block)
    {
      int *s_big = sh_list(), *s_mid = sh_list2();
      int &s_nbig = sh_ints()[0];
      int &s_nmid = sh_ints()[2];
      const int lane = threadIdx.x & 31;
      for (int t0 = lo; t0 < hi; t0 += blockDim.x) {
        if (threadIdx.x == 0) {
          s_nbig = 0;
          s_nmid = 0;
        }
        __syncthreads();
        const int I = t0 + threadIdx.x;
        if (I < hi) {
          const int a = G.aggptr[I], len = G.aggptr[I + 1] - a;
          if (len <= kSmallSeg) {
            thread_sort(G.members + a, len);
            int off = 0;
            for (int k = 0; k < len; k++) {
              const int m = G.members[a + k];
              G.memoff[m] = off;
              off += G.cc[m];
            }
          } else if (len <= kWarpSegG) {
            s_mid[atomicAdd(&s_nmid, 1)] = I;
          } else {
            s_big[atomicAdd(&s_nbig, 1)] = I;
          }
        }
        __syncthreads();
        const int nmid = s_nmid;
        for (int q = threadIdx.x >> 5; q < nmid; q += blockDim.x >> 5) {
          const int Im = s_mid[q];
          const int a = G.aggptr[Im], len = G.aggptr[Im + 1] - a;
          warp_sort(G.members + a, len);
          int run = 0;
          for (int k0 = 0; k0 < len; k0 += 32) {
            const int k = k0 + lane;
            const int m = k < len ? G.members[a + k] : 0;
            const int c = k < len ? G.cc[m] : 0;
            int x = c;
            for (int o = 1; o < 32; o <<= 1) {
              const int y = __shfl_up_sync(0xffffffffu, x, o);
              if (lane >= o) x += y;
            }
            if (k < len) G.memoff[m] = run + x - c;
            run += __shfl_sync(0xffffffffu, x, 31);
          }
        }
        __syncthreads();
        const int nbig = s_nbig;
        for (int q = 0; q < nbig; q++) {
          const int Ib = s_big[q];
          const int a = G.aggptr[Ib], len = G.aggptr[Ib + 1] - a;
          block_sort(G.members + a, len);
          int run = 0;
          for (int k0 = 0; k0 < len; k0 += blockDim.x) {
            const int k = k0 + threadIdx.x;
            const int m = k < len ? G.members[a + k] : 0;
            const int c = k < len ? G.cc[m] : 0;
            int tot;
            const int ex = block_scan(c, &tot);
            if (k < len) G.memoff[m] = run + ex;
            run += tot;
          }
        }
        __syncthreads();
      }
    }
    if (!sync_p()) return false;
    // the V-cycle preconditioner of the refinement restricts through these
    // sorted member lists: kept in the arena
    if (S->opt.refine == 1 && S->opt.refine_precond == 1) {
      int *mptr = (int *)aalloc(4ull * (nc + 1));
      int *mem = (int *)aalloc(4ull * n);
      if (!mptr || !mem) return false;
      for (long long I = tid; I <= nc; I += nthr) mptr[I] = G.aggptr[I];
      for (int k = tid; k < n; k += nthr) mem[k] = G.members[k];
      if (lead()) {
        L->mptr = mptr;
        L->mem = mem;
      }
    }
    // G5: cross entries into their aggregate's segment, key = (J, slot); a
    // heavy row's slots are handed out in entry order by ballots over chunks
    for (int v = tid; v < n; v += nthr) {
      if (rp[v + 1] - rp[v] >= kHeavyDeg) continue;
      const int I = agg[v];
      const int base = G.segptr[I];
      int slot = G.memoff[v];
      for (int e = rp[v]; e < rp[v + 1]; e++) {
        const int J = agg[ci[e]];
        if (J == I) continue;
        G.keys[base + slot] = ((uint64_t)(uint32_t)J << 32) | (uint32_t)slot;
        G.segw[base + slot] = wl[e];
        slot++;
      }
    }
    for (int g0 = gw * 32; g0 < n; g0 += nwarp * 32) {
      const int v0 = g0 + lane;
      unsigned mask = __ballot_sync(0xffffffffu, v0 < n && rp[v0 + 1] - rp[v0] >= kHeavyDeg);
      while (mask) {
        const int v = g0 + __ffs(mask) - 1;
        mask &= mask - 1;
        const int I = agg[v];
        const int base = G.segptr[I];
        int slot = G.memoff[v];
        for (int e0 = rp[v]; e0 < rp[v + 1]; e0 += 32) {
          const int e = e0 + lane;
          const int J = e < rp[v + 1] ? agg[ci[e]] : I;
          const unsigned cross = __ballot_sync(0xffffffffu, J != I);
          if (J != I) {
            const int sl = slot + __popc(cross & ((1u << lane) - 1u));
            G.keys[base + sl] = ((uint64_t)(uint32_t)J << 32) | (uint32_t)sl;
            G.segw[base + sl] = wl[e];
          }
          slot += __popc(cross);
        }
      }
    }
    if (!sync_p()) return false;
    // G6: sort each segment by (J, slot); distinct J per coarse row (short
    // segments by one thread, medium ones by one warp, long ones by the block)
    red = IRed{0, 0, 0};
    {
      int *s_big = sh_list(), *s_mid = sh_list2();
      int &s_nbig = sh_ints()[0];
      int &s_dist = sh_ints()[1];
      int &s_nmid = sh_ints()[2];
      const int lane = threadIdx.x & 31;
      for (int t0 = lo; t0 < hi; t0 += blockDim.x) {
        if (threadIdx.x == 0) {
          s_nbig = 0;
          s_nmid = 0;
        }
        __syncthreads();
        const int I = t0 + threadIdx.x;
        if (I < hi) {
          const int s = G.segptr[I], len = G.segptr[I + 1] - s;
          if (len <= kSmallSeg) {
            thread_sort(G.keys + s, len);
            int dcount = 0;
            for (int k = 0; k < len; k++)
              dcount += (k == 0) || ((G.keys[s + k] >> 32) != (G.keys[s + k - 1] >> 32));
            G.dcnt[I] = dcount;
            red.a += dcount;
          } else if (len <= kWarpSegG) {
            s_mid[atomicAdd(&s_nmid, 1)] = I;
          } else {
            s_big[atomicAdd(&s_nbig, 1)] = I;
          }
        }
        __syncthreads();
        const int nmid = s_nmid;
        for (int q = threadIdx.x >> 5; q < nmid; q += blockDim.x >> 5) {
          const int Im = s_mid[q];
          const int s = G.segptr[Im], len = G.segptr[Im + 1] - s;
          warp_sort(G.keys + s, len);
          int dc = 0;
          for (int k0 = 0; k0 < len; k0 += 32) {
            const int k = k0 + lane;
            const bool nw = k < len && ((k == 0) || ((G.keys[s + k] >> 32) != (G.keys[s + k - 1] >> 32)));
            dc += __popc(__ballot_sync(0xffffffffu, nw));
          }
          if (lane == 0) {
            G.dcnt[Im] = dc;
            red.a += dc;
          }
        }
        __syncthreads();
        const int nbig = s_nbig;
        for (int q = 0; q < nbig; q++) {
          const int Ib = s_big[q];
          const int s = G.segptr[Ib], len = G.segptr[Ib + 1] - s;
          block_sort(G.keys + s, len);
          if (threadIdx.x == 0) s_dist = 0;
          __syncthreads();
          int dc = 0;
          for (int k = threadIdx.x; k < len; k += blockDim.x)
            dc += (k == 0) || ((G.keys[s + k] >> 32) != (G.keys[s + k - 1] >> 32));
          if (dc) atomicAdd(&s_dist, dc);
          __syncthreads();
          if (threadIdx.x == 0) {
            G.dcnt[Ib] = s_dist;
            red.a += s_dist;
          }
          __syncthreads();
        }
      }
    }
    long long pre = 0;
    if (!grid_ired<true>(red, &pre)) return false;
    const long long nnzc = red.a;
    int *crp = (int *)aalloc(4ull * (nc + 1));
    int *ccol = (int *)aalloc(4ull * (nnzc > 0 ? nnzc : 1));
    double *cw = (double *)aalloc(8ull * (nnzc > 0 ? nnzc : 1));
    double *cd = (double *)aalloc(8ull * nc);
    if (!crp || !ccol || !cw || !cd) return false;
    // G7: coarse row pointers, then the summed weights in (J, slot) order
    red = IRed{0, 0, 0};
    {
      long long run = pre;
      int *s_big = sh_list(), *s_mid = sh_list2();
      int &s_nbig = sh_ints()[0];
      int &s_nmid = sh_ints()[2];
      for (int t0 = lo; t0 < hi; t0 += blockDim.x) {
        if (threadIdx.x == 0) {
          s_nbig = 0;
          s_nmid = 0;
        }
        const int I = t0 + threadIdx.x;
        const int dc = I < hi ? G.dcnt[I] : 0;
        int tot;
        const int ex = block_scan(dc, &tot);
        if (I < hi) crp[I] = (int)(run + ex);
        run += tot;
        __syncthreads();
        if (I < hi) {
          const int s = G.segptr[I], len = G.segptr[I + 1] - s;
          if (len <= kSmallSeg) {
            int p = crp[I];
            double dI = 0.0;
            int k = 0;
            while (k < len) {
              const uint32_t J = (uint32_t)(G.keys[s + k] >> 32);
              double sum = 0.0;
              while (k < len && (uint32_t)(G.keys[s + k] >> 32) == J) {
                sum += G.segw[s + (uint32_t)G.keys[s + k]];
                k++;
              }
              ccol[p] = (int)J;
              cw[p] = sum;
              p++;
            }
            for (int q = crp[I]; q < p; q++) dI += cw[q];
            cd[I] = dI;
            red.mx = max(red.mx, (long long)__double_as_longlong(dI));
          } else if (len <= kWarpSegG) {
            s_mid[atomicAdd(&s_nmid, 1)] = I;
          } else {
            s_big[atomicAdd(&s_nbig, 1)] = I;
          }
        }
        __syncthreads();
        // medium segments: one warp each; group starts found by ballots, each
        // group summed by the lane at its start in slot order, the diagonal
        // summed by lane 0 in column order (the same orders as below)
        const int nmid = s_nmid;
        for (int qm = threadIdx.x >> 5; qm < nmid; qm += blockDim.x >> 5) {
          const int Im = s_mid[qm];
          const int s = G.segptr[Im], len = G.segptr[Im + 1] - s;
          const int p0 = crp[Im];
          int gr = 0;
          for (int k0 = 0; k0 < len; k0 += 32) {
            const int k = k0 + lane;
            const bool st = k < len && (k == 0 || (G.keys[s + k] >> 32) != (G.keys[s + k - 1] >> 32));
            const unsigned sm = __ballot_sync(0xffffffffu, st);
            if (st) {
              const uint32_t J = (uint32_t)(G.keys[s + k] >> 32);
              double sum = 0.0;
              for (int kk = k; kk < len && (uint32_t)(G.keys[s + kk] >> 32) == J; kk++)
                sum += G.segw[s + (uint32_t)G.keys[s + kk]];
              const int pos = p0 + gr + __popc(sm & ((1u << lane) - 1u));
              ccol[pos] = (int)J;
              cw[pos] = sum;
            }
            gr += __popc(sm);
          }
          __syncwarp();
          if (lane == 0) {
            double dI = 0.0;
            for (int q2 = p0; q2 < p0 + gr; q2++) dI += cw[q2];
            cd[Im] = dI;
            red.mx = max(red.mx, (long long)__double_as_longlong(dI));
          }
        }
        __syncthreads();
        const int nbig = s_nbig;
        for (int q = 0; q < nbig; q++) {
          const int Ib = s_big[q];
          const int s = G.segptr[Ib], len = G.segptr[Ib + 1] - s;
          const int p0 = crp[Ib];
          int gr = 0;
          for (int k0 = 0; k0 < len; k0 += blockDim.x) {
            const int k = k0 + threadIdx.x;
            const bool st = k < len && (k == 0 || (G.keys[s + k] >> 32) != (G.keys[s + k - 1] >> 32));
            int tot2;
            const int ex2 = block_scan(st ? 1 : 0, &tot2);
            if (st) {
              const uint32_t J = (uint32_t)(G.keys[s + k] >> 32);
              double sum = 0.0;
              for (int kk = k; kk < len && (uint32_t)(G.keys[s + kk] >> 32) == J; kk++)
                sum += G.segw[s + (uint32_t)G.keys[s + kk]];
              ccol[p0 + gr + ex2] = (int)J;
              cw[p0 + gr + ex2] = sum;
            }
            gr += tot2;
          }
          __syncthreads();
          if (threadIdx.x == 0) {
            double dI = 0.0;
            for (int q2 = p0; q2 < p0 + gr; q2++) dI += cw[q2];
            cd[Ib] = dI;
            red.mx = max(red.mx, (long long)__double_as_longlong(dI));
          }
          __syncthreads();
        }
      }
      if (lead()) crp[nc] = (int)nnzc;
    }
    if (!grid_ired<true>(red)) return false;
    if (lead()) {
      Level &C = S->lv[l + 1];
      C.n = nc;
      C.nnz = (int)nnzc;
      C.rowptr = crp;
      C.col = ccol;
      C.w64 = cw;
      C.w32 = nullptr;
      C.d = cd;
      C.sigma = 2.0 * __longlong_as_double(red.mx);
      C.agg = nullptr;
      C.mate = nullptr;
      C.nc = 0;
    }
    if (!sync_p()) return false;
    FZ_MARK(PH_GALERKIN, 40.0 * n + (12.0 + 8.0 + 16.0 * 3.0) * L->nnz);
    return true;
  }

  // mean and inverse deflated norm from (sum x, sum x^2), computed by thread 0
  // and broadcast; false (EDEGEN) if the deflated vector vanished
  FZD bool deflate_scalars(const double (&acc)[2], int n, double &mu, double &sc) {
    double *bc = sh_bc();
    if (threadIdx.x == 0) {
      const double g = S->opt.guard;
      const double m = acc[0] / n, var = acc[1] - acc[0] * m;
      bc[0] = var > g * g ? 1.0 : 0.0;
      bc[1] = m;
      bc[2] = var > g * g ? 1.0 / sqrt(var) : 0.0;
    }
    __syncthreads();
    const bool ok = bc[0] != 0.0;
    mu = bc[1];
    sc = bc[2];
    __syncthreads();
    if (!ok) fail(ST_EDEGEN);
    return ok;
  }

  // ---- A7: coarsest level: connectivity, random start ---------------------
  FZD bool coarsest_solve(int J) {
    cur_level = J;
    Level *L = &S->lv[J];
    const int n = L->n;
    const int *rp = L->rowptr, *ci = L->col, *iperm = L->iperm;
    soff = 0;
    int *lab = (int *)salloc(4ull * n);
    if (!lab) return false;
    for (int v = tid; v < n; v += nthr) lab[v] = v;
    if (!sync()) return false;
    for (int it = 0;; it++) {
      IRed red{0, 0, 0};
      for (int v = tid; v < n; v += nthr) {
        int m = lab[v];
        for (int e = rp[v]; e < rp[v + 1]; e++) m = min(m, lab[ci[e]]);
        if (m < lab[v]) {
          lab[v] = m;
          red.a++;
        }
      }
      if (!grid_ired(red)) return false;
      if (red.a == 0) break;
      if (it > n) {
        fail(ST_EINVAL);
        return false;
      }
    }
    {
      IRed red{0, 0, 0};
      for (int v = tid; v < n; v += nthr) red.a += lab[v] != 0;
      if (!grid_ired(red)) return false;
      if (red.a != 0) {
        fail(ST_EDISC);
        return false;
      }
    }
    double acc[2] = {0.0, 0.0};
    const uint64_t seed = S->opt.seed;
    const bool vd = vdbl(n, L->nnz);
    for (int i = tid; i < n; i += nthr) {
      const double v = vd ? uniform01(seed, (uint64_t)i) : (double)(T)uniform01(seed, (uint64_t)i);
      if (vd) ((double *)L->x)[iperm[i]] = v;
      else ((T *)L->x)[iperm[i]] = (T)v;
      acc[0] += (double)v;
      acc[1] += (double)v * (double)v;
    }
    if (!grid_dsum<2>(acc)) return false;
    double mu, sc;
    if (!deflate_scalars(acc, n, mu, sc)) return false;
    FZ_MARK(PH_COARSEST, 16.0 * n + 8.0 * L->nnz);
    // with a Krylov refinement the finest level's power iteration is replaced by it
    return smooth(J, (J == 0 && S->opt.refine) ? 0 : S->opt.pi_max_iters_coarsest, mu, sc, PH_COARSEST);
  }

  // ---- A8: prolongation y^j = I^T y^{j+1} ----------------------------------
  FZD bool prolong(int l) {
    const bool vf = vdbl(S->lv[l].n, S->lv[l].nnz), vc = vdbl(S->lv[l + 1].n, S->lv[l + 1].nnz);
    if (vf) return prolong_v<double, double>(l);
    if (vc) return prolong_v<T, double>(l);
    return prolong_v<T, T>(l);
  }

  // VF, VC: value types of the fine and the coarse level
  template <class VF, class VC>
  FZD bool prolong_v(int l) {
    cur_level = l;
    Level *F = &S->lv[l];
    const Level *Cl = &S->lv[l + 1];
    const int n = F->n;
    const VC *xc = (const VC *)Cl->x;
    const VC muc = (VC)Cl->mu, scc = (VC)Cl->s;
    VF *x = (VF *)F->x;
    const int *sagg = F->sagg;
    RowSum<VF> r0, r1;
    for (int k = tid; k < n; k += nthr) {
      const VF v = (VF)((xc[sagg[k]] - muc) * scc);
      x[k] = v;
      r0.add(v);
      r1.add_prod(v, v);
    }
    double acc[2] = {r0.value(), r1.value()};
    if (!grid_dsum<2>(acc)) return false;
    double mu, sc;
    if (!deflate_scalars(acc, n, mu, sc)) return false;
    FZ_MARK(PH_PROLONG, 4.0 * n + (double)(sizeof(VF) + sizeof(VC)) * n);
    return smooth(l, (l == 0 && S->opt.refine) ? 0 : S->opt.pi_max_iters, mu, sc, PH_GS);
  }

  // ---- A9 + A10: Gauss-Seidel sweeps, then shifted power iteration ----------
  FZD bool smooth(int l, int kmax, double mu, double s, int gs_phase) {
    const int n = S->lv[l].n, nnz = S->lv[l].nnz;
    if (GRID) {
      // tiny levels, the FP64-valued ones of the FP32 form, are always small
      if (vdbl(n, nnz) && sizeof(T) != 8) {
        fail(ST_ENOTSUP);
        return false;
      }
      return smooth_v<T>(l, kmax, mu, s, gs_phase);
    }
    // one warp for the sparse tiny levels; denser ones need the whole block
    if (tiny(n, nnz) && nnz <= kWarpNnz) return smooth_warp<double>(l, kmax, mu, s, gs_phase);
    if (vdbl(n, nnz)) return smooth_v<double>(l, kmax, mu, s, gs_phase);
    return smooth_v<T>(l, kmax, mu, s, gs_phase);
  }

  template <class V>
  FZD bool smooth_v(int l, int kmax, double mu, double s, int gs_phase) {
    Level *L = &S->lv[l];
    const int n = L->n, nnz = L->nnz, C = L->ncolors;
    const int *srp = L->srowptr, *scol = L->scol, *cst = L->colstart;
    const int lane = threadIdx.x & 31, gw = tid >> 5, nwarp = nthr >> 5;
    const int nl = cst[C];  // light rows [0, nl), heavy rows [nl, n)
    const int hg = heavy_group(srp, nl, n);
    const V *sw = (const V *)L->sw;
    V *A = (V *)L->x, *B = (V *)L->y;
    const double g = S->opt.guard;
    const int nsweeps = S->opt.gs_sweeps;
    const double sweep_bytes = 4.0 * (n + 1) + (4.0 + sizeof(V)) * nnz + 2.0 * sizeof(V) * n;
    const int ph_gs = gs_phase == PH_COARSEST ? PH_COARSEST : PH_GS;
    const int ph_pi = gs_phase == PH_COARSEST ? PH_COARSEST : PH_PI;
    // FP64 scalars (means, norms, cos test) are computed by thread 0 of each
    // block from the grid totals and broadcast through shared memory; the
    // V copies used in the inner loops come with them
    double *bc = sh_bc();
    const double inv_n = 1.0 / (double)n;
    V muT = (V)mu, sT = (V)s;
    int sweeps = 0;
    for (int k = 0; k < nsweeps; k++) {
      double acc[2] = {0.0, 0.0};
      RowSum<V> rs0, rs1;
      for (int c = 0; c < C; c++) {
        // class c: light rows [cs, ce), heavy rows [hs, he); a neighbour j is
        // already updated in this sweep iff its class is below c
        const int cs = cst[c], ce = cst[c + 1], hs = cst[C + c], he = cst[C + c + 1];
        auto done = [&](int j) { return j < cs || (j >= nl && j < hs); };
        for (int i = cs + tid; i < ce; i += nthr) {
          V num = (V)0, dsum = (V)0;
          const int e1 = srp[i + 1];
          for (int e = srp[i]; e < e1; e++) {
            const int j = scol[e];
            const V wv = sw[e];
            const V xj = done(j) ? B[j] : (A[j] - muT) * sT;
            num += wv * xj;
            dsum += wv;
          }
          const V xi = num / dsum;
          B[i] = xi;
          rs0.add(xi);
          rs1.add_prod(xi, xi);
        }
        with_group<GRID>(hg, [&](auto gs) {  // heavy rows: a group of lanes each
          constexpr int G = decltype(gs)::value, GW = 32 / G;
          const int gl = lane & (G - 1), gi = lane / G;
          for (int base = hs + gw * GW; base < he; base += nwarp * GW) {
            const int i = base + gi;
            V num = (V)0, dsum = (V)0;
            if (i < he)
              group_row<G>(srp[i], srp[i + 1], scol, sw, [&](int j, V wv) {
                const V xj = done(j) ? B[j] : (A[j] - muT) * sT;
                num += wv * xj;
                dsum += wv;
              });
            num = group_sum<G>(num);
            dsum = group_sum<G>(dsum);
            if (gl == 0 && i < he) {
              const V xi = num / dsum;
              B[i] = xi;
              rs0.add(xi);
              rs1.add_prod(xi, xi);
            }
          }
        });
        if (c + 1 < C && !sync()) return false;
      }
      acc[0] = rs0.value();
      acc[1] = rs1.value();
      if (!grid_dsum<2>(acc)) return false;
      FZ_MARK(ph_gs, sweep_bytes);
      if (threadIdx.x == 0) {
        const double m2 = acc[0] * inv_n, var = acc[1] - acc[0] * m2;
        bc[0] = var > g * g ? 1.0 : 0.0;  // else: the sweep annihilated the iterate
        bc[1] = m2;
        bc[2] = var > g * g ? 1.0 / sqrt(var) : 0.0;
      }
      __syncthreads();
      const bool keep = bc[0] != 0.0;
      const double m2 = bc[1], s2 = bc[2];
      __syncthreads();
      if (!keep) break;  // keep the previous iterate
      V *t = A;
      A = B;
      B = t;
      mu = m2;
      s = s2;
      muT = (V)mu;
      sT = (V)s;
      sweeps++;
    }
    const double sigma = L->sigma;
    const double tol = S->opt.pi_cos_tol, rtol = S->opt.resid_tol;
    const bool resid = rtol > 0.0;
    const V sigT = (V)sigma;
    int done = 0, capped = 0;
    double lastc = 0.0;
    for (int it = 1; it <= kmax; it++) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      double acr[2] = {0.0, 0.0};
      RowSum<V> ps0, ps1, ps2, ps3;
      auto row = [&](int i, V xi, V lx) {
        const V xh = (xi - muT) * sT;
        const V yi = sigT * xh - sT * lx;
        B[i] = yi;
        ps0.add(yi);
        ps1.add_prod(yi, yi);
        ps2.add_prod(yi, xh);
        ps3.add(xh);
        if (resid) {
          const double ld = (double)sT * (double)lx, xd = (double)xh;
          acr[0] += ld * ld;
          acr[1] += xd * ld;
        }
      };
      // rows in any order here: light rows [0, nl) one thread each, heavy
      // rows [nl, n) one warp each
      for (int i = tid; i < nl; i += nthr) {
        const V xi = A[i];
        V lx = (V)0;
        const int e1 = srp[i + 1];
        for (int e = srp[i]; e < e1; e++) lx += sw[e] * (xi - A[scol[e]]);
        row(i, xi, lx);
      }
      with_group<GRID>(hg, [&](auto gs) {
        constexpr int G = decltype(gs)::value, GW = 32 / G;
        const int gl = lane & (G - 1), gi = lane / G;
        // the bound is uniform in the warp: every lane reaches the group sums
        for (int base = nl + gw * GW; base < n; base += nwarp * GW) {
          const int i = base + gi;
          V xi = (V)0, lx = (V)0;
          if (i < n) {
            xi = A[i];
            group_row<G>(srp[i], srp[i + 1], scol, sw, [&](int j, V wv) { lx += wv * (xi - A[j]); });
          }
          lx = group_sum<G>(lx);
          if (gl == 0 && i < n) row(i, xi, lx);
        }
      });
      acc[0] = ps0.value();
      acc[1] = ps1.value();
      acc[2] = ps2.value();
      acc[3] = ps3.value();
      if (!grid_dsum<4>(acc)) return false;
      if (resid && !grid_dsum<2>(acr)) return false;
      FZ_MARK(ph_pi, sweep_bytes);
      if (threadIdx.x == 0) {
        const double my = acc[0] * inv_n, var = acc[1] - acc[0] * my;
        const bool ok = var > (g * sigma) * (g * sigma);  // else the step vanished
        const double sy = ok ? 1.0 / sqrt(var) : 0.0;
        const double cosv = (acc[2] - my * acc[3]) * sy;
        const double rr = resid ? sqrt(fmax(acr[0] - acr[1] * acr[1], 0.0)) : 0.0;
        bc[0] = ok ? 1.0 : 0.0;
        bc[1] = my;
        bc[2] = sy;
        bc[3] = cosv;
        bc[4] = (ok && cosv > 1.0 - tol && (!resid || rr <= rtol * sigma)) ? 1.0 : 0.0;
      }
      __syncthreads();
      const bool ok = bc[0] != 0.0, stop = bc[4] != 0.0;
      const double my = bc[1], sy = bc[2], cosv = bc[3];
      __syncthreads();
      if (!ok) break;  // keep the previous vector
      V *t = A;
      A = B;
      B = t;
      mu = my;
      s = sy;
      muT = (V)mu;
      sT = (V)s;
      lastc = cosv;
      done = it;
      if (stop) break;
      if (it == kmax) capped = 1;
    }
    if (lead()) {
      L->x = A;
      L->y = B;
      L->mu = mu;
      L->s = s;
      L->gs_sweeps = sweeps;
      L->pi_iters = done;
      L->last_cos = lastc;
      L->capped = capped;
    }
    return sync();
  }

  // The same Gauss-Seidel sweeps and power iteration for tiny levels
  // (tiny levels, one-block kernel only): warp 0 runs them alone, with warp
  // syncs between colour passes and warp-shuffle FP64 sums, while the other
  // warps wait at one block barrier.  Identical arithmetic per row; only the
  // order of the FP64 sums differs from smooth().
  template <class V>
  FZD bool smooth_warp(int l, int kmax, double mu, double s, int gs_phase) {
    Level *L = &S->lv[l];
    const int n = L->n, nnz = L->nnz, C = L->ncolors;
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      const int *srp = L->srowptr, *scol = L->scol, *cst = L->colstart;
      const V *sw = (const V *)L->sw;
      V *A = (V *)L->x, *B = (V *)L->y;
      const double g = S->opt.guard;
      const int nsweeps = S->opt.gs_sweeps;
      const double sweep_bytes = 4.0 * (n + 1) + (4.0 + sizeof(V)) * nnz + 2.0 * sizeof(V) * n;
      const int ph_gs = gs_phase == PH_COARSEST ? PH_COARSEST : PH_GS;
      const int ph_pi = gs_phase == PH_COARSEST ? PH_COARSEST : PH_PI;
      int sweeps = 0;
      for (int k = 0; k < nsweeps; k++) {
        double acc[2] = {0.0, 0.0};
        const V muT = (V)mu, sT = (V)s;
        const int nl = cst[C];
        for (int c = 0; c < C; c++) {
          const int cs = cst[c], ce = cst[c + 1], hs = cst[C + c], he = cst[C + c + 1];
          auto done = [&](int j) { return j < cs || (j >= nl && j < hs); };
          for (int i = cs + lane; i < ce; i += 32) {
            V num = (V)0, dsum = (V)0;
            const int e1 = srp[i + 1];
            for (int e = srp[i]; e < e1; e++) {
              const int j = scol[e];
              const V wv = sw[e];
              const V xj = done(j) ? B[j] : (A[j] - muT) * sT;
              num += wv * xj;
              dsum += wv;
            }
            const V xi = num / dsum;
            B[i] = xi;
            acc[0] += (double)xi;
            acc[1] += (double)xi * (double)xi;
          }
          for (int i = hs; i < he; i++) {  // heavy rows: the warp together
            V num = (V)0, dsum = (V)0;
            const int e1 = srp[i + 1];
#pragma unroll 4
            for (int e = srp[i] + lane; e < e1; e += 32) {
              const int j = scol[e];
              const V wv = sw[e];
              const V xj = done(j) ? B[j] : (A[j] - muT) * sT;
              num += wv * xj;
              dsum += wv;
            }
            num = warp_sum(num);
            dsum = warp_sum(dsum);
            const V xi = num / dsum;
            if (lane == 0) {
              B[i] = xi;
              acc[0] += (double)xi;
              acc[1] += (double)xi * (double)xi;
            }
          }
          __syncwarp();
        }
        warp_dsum<2>(acc);
        FZ_MARK(ph_gs, sweep_bytes);
        double m2 = 0.0, s2 = 0.0;
        int keep = 0;
        if (lane == 0) {
          m2 = acc[0] / n;
          const double var = acc[1] - acc[0] * m2;
          keep = var > g * g;
          s2 = keep ? 1.0 / sqrt(var) : 0.0;
        }
        keep = __shfl_sync(0xffffffffu, keep, 0);
        m2 = __shfl_sync(0xffffffffu, m2, 0);
        s2 = __shfl_sync(0xffffffffu, s2, 0);
        if (!keep) break;
        V *t = A;
        A = B;
        B = t;
        mu = m2;
        s = s2;
        sweeps++;
      }
      const double sigma = L->sigma;
      const double tol = S->opt.pi_cos_tol, rtol = S->opt.resid_tol;
      const bool resid = rtol > 0.0;
      int done = 0, capped = 0;
      double lastc = 0.0;
      for (int it = 1; it <= kmax; it++) {
        double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        const V muT = (V)mu, sT = (V)s, sigT = (V)sigma;
        auto row = [&](int i, V xi, V lx) {
          const V xh = (xi - muT) * sT;
          const V yi = sigT * xh - sT * lx;
          B[i] = yi;
          const double yd = (double)yi, xd = (double)xh;
          acc[0] += yd;
          acc[1] += yd * yd;
          acc[2] += yd * xd;
          acc[3] += xd;
          if (resid) {
            const double ld = (double)sT * (double)lx;
            acc[4] += ld * ld;
            acc[5] += xd * ld;
          }
        };
        const int nl = cst[C];  // light rows [0, nl), heavy rows [nl, n)
        for (int i = lane; i < nl; i += 32) {
          const V xi = A[i];
          V lx = (V)0;
          const int e1 = srp[i + 1];
          for (int e = srp[i]; e < e1; e++) lx += sw[e] * (xi - A[scol[e]]);
          row(i, xi, lx);
        }
        for (int i = nl; i < n; i++) {
          const V xi = A[i];
          V lx = (V)0;
          const int e1 = srp[i + 1];
#pragma unroll 4
          for (int e = srp[i] + lane; e < e1; e += 32) lx += sw[e] * (xi - A[scol[e]]);
          lx = warp_sum(lx);
          if (lane == 0) row(i, xi, lx);
        }
        __syncwarp();
        warp_dsum<6>(acc);
        FZ_MARK(ph_pi, sweep_bytes);
        double my = 0.0, sy = 0.0, cosv = 0.0;
        int ok = 0, stop = 0;
        if (lane == 0) {
          my = acc[0] / n;
          const double var = acc[1] - acc[0] * my;
          ok = var > (g * sigma) * (g * sigma);
          sy = ok ? 1.0 / sqrt(var) : 0.0;
          cosv = (acc[2] - my * acc[3]) * sy;
          const double rr = resid ? sqrt(fmax(acc[4] - acc[5] * acc[5], 0.0)) : 0.0;
          stop = ok && cosv > 1.0 - tol && (!resid || rr <= rtol * sigma);
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        stop = __shfl_sync(0xffffffffu, stop, 0);
        my = __shfl_sync(0xffffffffu, my, 0);
        sy = __shfl_sync(0xffffffffu, sy, 0);
        cosv = __shfl_sync(0xffffffffu, cosv, 0);
        if (!ok) break;
        V *t = A;
        A = B;
        B = t;
        mu = my;
        s = sy;
        lastc = cosv;
        done = it;
        if (stop) break;
        if (it == kmax) capped = 1;
      }
      if (lane == 0) {
        L->x = A;
        L->y = B;
        L->mu = mu;
        L->s = s;
        L->gs_sweeps = sweeps;
        L->pi_iters = done;
        L->last_cos = lastc;
        L->capped = capped;
      }
    }
    return sync();
  }

  // ---- finest-level Krylov refinement (Sec. 4's Krylov smoother) ----------
  // Runs in place of the finest level's power iteration, after its
  // Gauss-Seidel sweeps, until ||L x - theta x|| <= refine_tol theta ||x||.
  FZN bool refine() {
    cur_level = 0;
    const int n = S->lv[0].n, nnz = S->lv[0].nnz;
    if (GRID && vdbl(n, nnz) && sizeof(T) != 8) {  // see smooth()
      fail(ST_ENOTSUP);
      return false;
    }
    if (S->opt.refine == 1) return (!GRID && vdbl(n, nnz)) ? lobpcg_v<double>() : lobpcg_v<T>();
    if (S->opt.refine == 2) return (!GRID && vdbl(n, nnz)) ? lanczos_v<double>() : lanczos_v<T>();
    fail(ST_ENOTSUP);
    return false;
  }

  // h[t] = sum_i Q_t[i] U[i] for t < k (k <= kMaxBasis + 1), FP64, in every
  // thread's view of the shared array h: per warp by xor trees, the block's
  // warps and (grid form) the blocks' partials in fixed order
  template <class V>
  FZN bool basis_dots(const V *Q, size_t ldq, const V *U, int n, int k, double *h) {
    double *wp = reinterpret_cast<double *>(sh_raw());  // [warps][kMaxBasis + 1]
    constexpr int LD = kMaxBasis + 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = 0; t < k; t++) {
      const V *q = Q + (size_t)t * ldq;
      double a = 0.0;
      for (int i = tid; i < n; i += nthr) a += (double)q[i] * (double)U[i];
      a = warp_sum(a);
      if (lane == 0) wp[w * LD + t] = a;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
      double a = 0.0;
      for (int q = 0; q < nw; q++) a += wp[q * LD + t];
      h[t] = a;
    }
    __syncthreads();
    if (GRID && !local_) {
      double *part = S->dpart + (size_t)rb * kMaxBlocks * kDSum;
      for (int t = threadIdx.x; t < k; t += blockDim.x) part[bid * kDSum + t] = h[t];
      if (!sync()) return false;
      for (int t = threadIdx.x; t < k; t += blockDim.x) {
        double a = 0.0;
        for (int b = 0; b < nb; b++) a += part[b * kDSum + t];
        h[t] = a;
      }
      __syncthreads();
      rb ^= 1;
    } else {
      if (!__syncthreads_and(status() == 0)) return false;
    }
    return true;
  }

  // Lanczos with full reorthogonalisation (classical Gram-Schmidt, twice) on
  // 1-perp, restarted from the smallest Ritz vector every lanczos_basis steps;
  // the Ritz estimate beta_m |s_m| is tested at the end of each cycle.  Basis
  // Q_0..Q_m (rows of n values), work vector U; the tridiagonal problem is
  // solved by one thread.
  template <class V>
  FZN bool lanczos_v() {
    Level *L = &S->lv[0];
    const int n = L->n, nnz = L->nnz;
    const int m = S->opt.lanczos_basis;
    const size_t ld = ((size_t)n + 63) & ~(size_t)63;  // rows start on 256-byte boundaries
    V *A = (V *)L->x;
    V *Q = (V *)aalloc(sizeof(V) * ld * (size_t)(m + 1));
    V *U = (V *)aalloc(sizeof(V) * (size_t)n);
    if (!Q || !U) return false;
    __shared__ double lz_al[kMaxBasis], lz_be[kMaxBasis], lz_h[kMaxBasis + 1], lz_s[kMaxBasis], lz_w[4 * kMaxBasis];
    double *bc = sh_bc();
    const double tol = S->opt.refine_tol;
    const int kmax = S->opt.refine_max_iters;
    const double inv_n = 1.0 / (double)n;
    const double step_bytes = 4.0 * (n + 1) + (4.0 + sizeof(V)) * nnz + 2.0 * sizeof(V) * n;
    // start: Q_0 = x (deflated, unit)
    {
      const V muT = (V)L->mu, sT = (V)L->s;
      double acc[2] = {0.0, 0.0};
      for (int i = tid; i < n; i += nthr) {
        const V v = (A[i] - muT) * sT;
        U[i] = v;
        acc[0] += (double)v;
        acc[1] += (double)v * (double)v;
      }
      if (!grid_wsum<2>(acc)) return false;
      const double mq = acc[0] * inv_n, nq = 1.0 / sqrt(fmax(acc[1] - acc[0] * mq, DBL_MIN));
      for (int i = tid; i < n; i += nthr) Q[i] = (V)(((double)U[i] - mq) * nq);
      if (!sync()) return false;
    }
    int total = 0, capped = 0;
    for (;;) {
      int kk = 0;
      for (int j = 0; j < m; j++) {
        if (total >= kmax) break;
        const V *qj = Q + (size_t)j * ld;
        double acc[2] = {0.0, 0.0};
        lap_rows<V>(L, qj, [&](int i, V lv, V dv) {
          U[i] = lv;
          acc[0] += (double)qj[i] * (double)lv;
          acc[1] += (double)lv;
        });
        if (!grid_wsum<2>(acc)) return false;
        total++;
        const double al = acc[0], mu_u = acc[1] * inv_n, bprev = j > 0 ? lz_be[j - 1] : 0.0;
        {
          const V a = (V)al, mu = (V)mu_u, bp = (V)bprev;
          const V *qp = j > 0 ? Q + (size_t)(j - 1) * ld : qj;
          for (int i = tid; i < n; i += nthr) U[i] = U[i] - mu - a * qj[i] - bp * qp[i];
        }
        if (threadIdx.x == 0) lz_al[j] = al;
        if (!sync()) return false;
        for (int pass = 0; pass < 2; pass++) {
          if (!basis_dots<V>(Q, ld, U, n, j + 1, lz_h)) return false;
          for (int i = tid; i < n; i += nthr) {
            double u = (double)U[i];
            for (int t = 0; t <= j; t++) u -= lz_h[t] * (double)Q[(size_t)t * ld + i];
            U[i] = (V)u;
          }
          if (!sync()) return false;
        }
        double nn[1] = {0.0};
        for (int i = tid; i < n; i += nthr) nn[0] += (double)U[i] * (double)U[i];
        if (!grid_wsum<1>(nn)) return false;
        const double be = sqrt(nn[0]);
        if (threadIdx.x == 0) lz_be[j] = be;
        kk = j + 1;
        FZ_MARK(PH_REFINE, step_bytes + (4.0 * (j + 1) + 4.0) * sizeof(V) * n);
        if (!(be > 1e-12 * fabs(al))) break;  // invariant subspace
        V *qn = Q + (size_t)(j + 1) * ld;
        const V ib = (V)(1.0 / be);
        for (int i = tid; i < n; i += nthr) qn[i] = U[i] * ib;
        if (!sync()) return false;
      }
      if (kk == 0) {  // the cap was reached at a cycle boundary
        capped = 1;
        break;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        const double th = tri_smallest(lz_al, lz_be, kk, lz_s, lz_w);
        bc[0] = th;
        bc[1] = lz_be[kk - 1] * fabs(lz_s[kk - 1]);
      }
      __syncthreads();
      const double theta = bc[0], est = bc[1];
      __syncthreads();
      // Ritz vector y = sum_t s_t Q_t into U, then deflated and normalised into Q_0
      double acc[2] = {0.0, 0.0};
      for (int i = tid; i < n; i += nthr) {
        double y = 0.0;
        for (int t = 0; t < kk; t++) y += lz_s[t] * (double)Q[(size_t)t * ld + i];
        const V v = (V)y;
        U[i] = v;
        acc[0] += (double)v;
        acc[1] += (double)v * (double)v;
      }
      if (!grid_wsum<2>(acc)) return false;
      const double my = acc[0] * inv_n, ny = 1.0 / sqrt(fmax(acc[1] - acc[0] * my, DBL_MIN));
      for (int i = tid; i < n; i += nthr) Q[i] = (V)(((double)U[i] - my) * ny);
      if (!sync()) return false;
      if (est <= tol * theta) break;
      if (total >= kmax) {
        capped = 1;
        break;
      }
    }
    if (lead()) {
      L->x = Q;
      L->y = U;
      L->mu = 0.0;
      L->s = 1.0;
      L->refine_iters = total;
      L->capped |= capped;
    }
    return sync();
  }

  // Row pass over level 0 in solve order: f(i, lv, d) with lv = sum_j w_ij
  // (u_i - u_j) and d = sum_j w_ij in V; light rows one thread each, heavy rows
  // a group of lanes each (f runs on the group's first lane).
  template <class V, class F>
  FZD void lap_rows(const Level *L, const V *u, F f) {
    const int n = L->n;
    const int *srp = L->srowptr, *scol = L->scol;
    const V *sw = (const V *)L->sw;
    const int nl = L->colstart[L->ncolors];
    const int lane = threadIdx.x & 31, gw = tid >> 5, nwarp = nthr >> 5;
    for (int i = tid; i < nl; i += nthr) {
      const V ui = u[i];
      V lv = (V)0, dv = (V)0;
      const int e1 = srp[i + 1];
      for (int e = srp[i]; e < e1; e++) {
        const V wv = sw[e];
        lv += wv * (ui - u[scol[e]]);
        dv += wv;
      }
      f(i, lv, dv);
    }
    with_group<GRID>(heavy_group(srp, nl, n), [&](auto gs) {
      constexpr int G = decltype(gs)::value, GW = 32 / G;
      const int gl = lane & (G - 1), gi = lane / G;
      for (int base = nl + gw * GW; base < n; base += nwarp * GW) {
        const int i = base + gi;
        V lv = (V)0, dv = (V)0;
        if (i < n) {
          const V ui = u[i];
          group_row<G>(srp[i], srp[i + 1], scol, sw, [&](int j, V wv) {
            lv += wv * (ui - u[j]);
            dv += wv;
          });
        }
        lv = group_sum<G>(lv);
        dv = group_sum<G>(dv);
        if (gl == 0 && i < n) f(i, lv, dv);
      }
    });
  }

  // ---- V-cycle preconditioner of the LOBPCG refinement ---------------------
  // One V-cycle of the cascade's own hierarchy on L e = r: per level one
  // forward Gauss-Seidel sweep from e = 0 (colour classes ascending; a class
  // has no internal edges, so rows update in place in any order), the
  // residual summed over each aggregate (members ascending, FP64 sums) as the
  // next level's right-hand side, 20 sweeps and the mean removed on the
  // coarsest level, the correction added to every member, one backward sweep
  // (classes descending).  Level l's vectors vb (rhs), ve (correction), vt
  // (residual) have the level's value type.
  template <class F>
  FZD void with_ltype(int l, F f) {
    if (vdbl(S->lv[l].n, S->lv[l].nnz)) f((double)0);
    else f((T)0);
  }

  template <class V>
  FZD void vc_class(const Level *L, int c, const V *b, V *e) {
    const int C = L->ncolors, n = L->n;
    const int *cst = L->colstart, *srp = L->srowptr, *scol = L->scol;
    const V *sw = (const V *)L->sw;
    const int nl = cst[C], cs = cst[c], ce = cst[c + 1], hs = cst[C + c], he = cst[C + c + 1];
    for (int i = cs + tid; i < ce; i += nthr) {
      V num = b[i], dsum = (V)0;
      const int e1 = srp[i + 1];
      for (int k = srp[i]; k < e1; k++) {
        const V wv = sw[k];
        num += wv * e[scol[k]];
        dsum += wv;
      }
      e[i] = num / dsum;
    }
    const int lane = threadIdx.x & 31, gw = tid >> 5, nwarp = nthr >> 5;
    with_group<GRID>(heavy_group(srp, nl, n), [&](auto gs) {
      constexpr int G = decltype(gs)::value, GW = 32 / G;
      const int gl = lane & (G - 1), gi = lane / G;
      for (int base = hs + gw * GW; base < he; base += nwarp * GW) {
        const int i = base + gi;
        V num = (V)0, dsum = (V)0;
        if (i < he)
          group_row<G>(srp[i], srp[i + 1], scol, sw, [&](int j, V wv) {
            num += wv * e[j];
            dsum += wv;
          });
        num = group_sum<G>(num);
        dsum = group_sum<G>(dsum);
        if (gl == 0 && i < he) e[i] = (b[i] + num) / dsum;
      }
    });
  }

  template <class V>
  FZN bool vc_sweeps(int l, bool forward, bool zero_first, int count) {
    const Level *L = &S->lv[l];
    const V *b = (const V *)L->vb;
    V *e = (V *)L->ve;
    const int C = L->ncolors;
    if (zero_first) {
      for (int i = tid; i < L->n; i += nthr) e[i] = (V)0;
      if (!sync()) return false;
    }
    for (int k = 0; k < count; k++)
      for (int q = 0; q < C; q++) {
        vc_class<V>(L, forward ? q : C - 1 - q, b, e);
        if (!sync()) return false;
      }
    return true;
  }

  template <class V>
  FZN bool vc_resid(int l) {
    const Level *L = &S->lv[l];
    const V *b = (const V *)L->vb;
    V *t = (V *)L->vt;
    lap_rows<V>(L, (const V *)L->ve, [&](int i, V lv, V dv) { t[i] = b[i] - lv; });
    return sync();
  }

  template <class VF, class VC>
  FZN bool vc_restrict(int l) {
    const Level *F = &S->lv[l];
    const Level *Cl = &S->lv[l + 1];
    const int nc = Cl->n;
    const int *mptr = F->mptr, *mem = F->mem, *ipf = F->iperm, *ipc = Cl->iperm;
    const VF *t = (const VF *)F->vt;
    VC *bc = (VC *)Cl->vb;
    for (int I = tid; I < nc; I += nthr) {
      double s = 0.0;
      for (int k = mptr[I]; k < mptr[I + 1]; k++) s += (double)t[ipf[mem[k]]];
      bc[ipc[I]] = (VC)s;
    }
    return sync();
  }

  template <class V>
  FZN bool vc_coarsest(int J) {
    const Level *L = &S->lv[J];
    if (!vc_sweeps<V>(J, true, true, 20)) return false;
    V *e = (V *)L->ve;
    double acc[1] = {0.0};
    for (int i = tid; i < L->n; i += nthr) acc[0] += (double)e[i];
    if (!grid_dsum<1>(acc)) return false;
    const V mu = (V)(acc[0] / (double)L->n);
    for (int i = tid; i < L->n; i += nthr) e[i] = e[i] - mu;
    return sync();
  }

  template <class VF, class VC>
  FZN bool vc_prolong(int l) {
    const Level *F = &S->lv[l];
    const Level *Cl = &S->lv[l + 1];
    VF *ef = (VF *)F->ve;
    const VC *ec = (const VC *)Cl->ve;
    const int *sagg = F->sagg;
    for (int k = tid; k < F->n; k += nthr) ef[k] = ef[k] + (VF)ec[sagg[k]];
    return sync();
  }

  // down-sweep over levels [a, b): pre-smoothing, residual, restriction to l + 1
  FZD bool vc_down(int a, int b) {
    bool ok = true;
    for (int l = a; l < b && ok; l++)
      with_ltype(l, [&](auto tf) {
        using VF = decltype(tf);
        ok = vc_sweeps<VF>(l, true, true, 1) && vc_resid<VF>(l);
        if (ok)
          with_ltype(l + 1, [&](auto tc) {
            using VC = decltype(tc);
            ok = vc_restrict<VF, VC>(l);
          });
      });
    return ok;
  }
  // up-sweep over levels a down to b: prolongation from l + 1, post-smoothing
  FZD bool vc_up(int a, int b) {
    bool ok = true;
    for (int l = a; l >= b && ok; l--)
      with_ltype(l, [&](auto tf) {
        using VF = decltype(tf);
        with_ltype(l + 1, [&](auto tc) {
          using VC = decltype(tc);
          ok = vc_prolong<VF, VC>(l);
        });
        if (ok) ok = vc_sweeps<VF>(l, false, false, 1);
      });
    return ok;
  }
  FZD bool vc_bottom(int J) {
    bool ok = true;
    with_ltype(J, [&](auto t) {
      using V = decltype(t);
      ok = vc_coarsest<V>(J);
    });
    return ok;
  }

  // e_0 = V(b_0): the right-hand side in level 0's vb, the result in its ve.
  // In the grid form the small levels (those the one-block engine sets up)
  // are cycled by block 0 alone with block barriers, while the other blocks
  // wait at one grid barrier: there a grid barrier per colour pass would cost
  // far more than the levels' work.
  FZN bool vcycle() {
    const int J = nlevels - 1;
    if (!GRID) return vc_down(0, J) && vc_bottom(J) && vc_up(J - 1, 0);
    int ls = 0;
    while (ls < J && !small(S->lv[ls].n, S->lv[ls].nnz)) ls++;
    if (!vc_down(0, ls)) return false;
    if (bid == 0) {
      const int stid = tid, snthr = nthr, snb = nb;
      local_ = true;
      tid = threadIdx.x;
      nthr = blockDim.x;
      nb = 1;
      vc_down(ls, J) && vc_bottom(J) && vc_up(J - 1, ls);
      local_ = false;
      tid = stid;
      nthr = snthr;
      nb = snb;
    }
    if (!sync()) return false;
    return vc_up(ls - 1, 0);
  }

  // the V-cycle's per-level vectors, from the arena
  FZN bool vc_alloc() {
    for (int l = 0; l < nlevels; l++) {
      Level *L = &S->lv[l];
      const unsigned long long vs = vdbl(L->n, L->nnz) ? 8ull : sizeof(T);
      void *b = aalloc(vs * L->n), *e = aalloc(vs * L->n), *t = aalloc(vs * L->n);
      if (!b || !e || !t) return false;
      if (lead()) {
        L->vb = b;
        L->ve = e;
        L->vt = t;
      }
    }
    return sync();
  }

  // LOBPCG (Knyazev 2001), one vector, on 1-perp with the preconditioner
  // D^-1.  Iterate X, preconditioned residual W = D^-1 (L X - theta X), search
  // direction P; the means of X, W and P are removed lazily (x = X - mu_x ...;
  // L 1 = 0, so L-products need no correction).  The products L X and L P are
  // computed afresh every iteration (a float recurrence for them drifts and
  // lets the iteration diverge).  Per iteration: a matvec pass (L X, L P, the
  // Rayleigh quotient and residual sums), a pass forming W, a matvec pass L W
  // with the Gram sums of [x, w, p], one FP64 Rayleigh-Ritz step, an update
  // pass.  Stops when ||L x - theta x|| <= refine_tol theta ||x||, after
  // kRefineFlat steps in a row without a new lowest theta (each Rayleigh-Ritz
  // step lowers it in exact arithmetic: this is the rounding floor of the
  // value type; float iterates reach it near a residual of 1e-3 theta with
  // lambda_2 exact to ~1e-8; such a step also restarts without p), or at
  // refine_max_iters.
  template <class V>
  FZN bool lobpcg_v() {
    Level *L = &S->lv[0];
    const int n = L->n, nnz = L->nnz;
    V *A = (V *)L->x;
    V *X = (V *)aalloc(sizeof(V) * (size_t)n);
    V *LX = (V *)aalloc(sizeof(V) * (size_t)n);
    V *W = (V *)aalloc(sizeof(V) * (size_t)n);
    V *LW = (V *)aalloc(sizeof(V) * (size_t)n);
    V *P = (V *)aalloc(sizeof(V) * (size_t)n);
    V *LP = (V *)aalloc(sizeof(V) * (size_t)n);
    V *DI = (V *)aalloc(sizeof(V) * (size_t)n);
    if (!X || !LX || !W || !LW || !P || !LP || !DI) return false;
    const bool vc = S->opt.refine_precond == 1;
    if (vc && !vc_alloc()) return false;
    V *VB = (V *)L->vb;  // level 0's V-cycle right-hand side (vc only)
    const double tol = S->opt.refine_tol;
    const int kmax = S->opt.refine_max_iters;
    const double inv_n = 1.0 / (double)n;
    const double it_bytes = 2.0 * (4.0 * (n + 1) + (4.0 + sizeof(V)) * nnz) + 16.0 * sizeof(V) * n;
    double *bc = sh_bc();
    {
      const V muT = (V)L->mu, sT = (V)L->s;
      for (int i = tid; i < n; i += nthr) X[i] = (A[i] - muT) * sT;
      if (!sync()) return false;
    }
    double mux = 0.0, mup = 0.0, theta_best = 0.0;
    bool pvalid = false;
    int iters = 0, capped = 0, flat = 0;
    for (;;) {
      // L X and L P afresh; sums for theta and the means (X's stored mean is
      // the update's rounding only: it is measured here, and L 1 = 0)
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      lap_rows<V>(L, X, [&](int i, V lv, V dv) {
        LX[i] = lv;
        if (iters == 0) DI[i] = (V)1 / dv;
        const double xv = (double)X[i], lx = (double)lv;
        acc[0] += xv * xv;
        acc[1] += xv * lx;
        acc[2] += xv;
      });
      if (pvalid)
        lap_rows<V>(L, P, [&](int i, V lv, V dv) {
          LP[i] = lv;
          acc[3] += (double)P[i];
        });
      if (!grid_wsum<4>(acc)) return false;
      mux = acc[2] * inv_n;
      mup = acc[3] * inv_n;
      const double xx = acc[0] - acc[2] * mux, theta = acc[1] / xx;
      // residual r = L x - theta x (its norm for the stop rule) and the
      // preconditioned W = D^-1 r, or r as the V-cycle's right-hand side;
      // W's mean mu_w is removed where W is read
      double racc[2] = {0.0, 0.0};
      {
        const V mx = (V)mux, th = (V)theta;
        for (int i = tid; i < n; i += nthr) {
          const V r = LX[i] - th * (X[i] - mx);
          racc[0] += (double)r * (double)r;
          if (vc) {
            VB[i] = r;
          } else {
            const V wv = DI[i] * r;
            W[i] = wv;
            racc[1] += (double)wv;
          }
        }
      }
      if (!grid_wsum<2>(racc)) return false;
      double muw = racc[1] * inv_n;
      if (racc[0] <= tol * tol * theta * theta * xx) break;
      if (iters == 0 || theta < theta_best) {
        theta_best = theta;
        flat = 0;
      } else {
        // no new lowest Rayleigh quotient (only rounding causes it): restart
        // without p; kRefineFlat such steps in a row are the rounding floor
        pvalid = false;
        if (++flat >= kRefineFlat) break;
      }
      if (iters >= kmax) {
        capped = 1;
        break;
      }
      if (vc) {  // W = V(r)
        if (!vcycle()) return false;
        const V *E = (const V *)L->ve;
        double wacc[1] = {0.0};
        for (int i = tid; i < n; i += nthr) {
          const V wv = E[i];
          W[i] = wv;
          wacc[0] += (double)wv;
        }
        if (!grid_wsum<1>(wacc)) return false;
        muw = wacc[0] * inv_n;
      }
      // L W and the Gram sums of [x, w, p]
      double g[12];
#pragma unroll
      for (int k = 0; k < 12; k++) g[k] = 0.0;
      {
        const V mx = (V)mux, mp = (V)mup, mw = (V)muw;
        lap_rows<V>(L, W, [&](int i, V lv, V dv) {
          LW[i] = lv;
          const double xh = (double)(X[i] - mx), wh = (double)(W[i] - mw), lx = (double)LX[i];
          const double lw = (double)lv;
          // x^T L w is taken as (L x)^T w: L x of the smooth iterate comes out of
          // the difference form nearly exact, while a float L w carries an error
          // of eps ||L|| ||w||, large beside x^T L w once the residual is small
          g[0] += xh * xh;
          g[1] += xh * wh;
          g[3] += wh * wh;
          g[6] += xh * lx;
          g[7] += lx * wh;
          g[9] += wh * lw;
          if (pvalid) {
            const double ph = (double)(P[i] - mp), lp = (double)LP[i];
            g[2] += xh * ph;
            g[4] += wh * ph;
            g[5] += ph * ph;
            g[8] += lx * ph;
            g[10] += wh * lp;
            g[11] += ph * lp;
          }
        });
      }
      if (!grid_wsum<12>(g)) return false;
      iters++;
      FZ_MARK(PH_REFINE, it_bytes);
      if (threadIdx.x == 0) {
        const double G[9] = {g[0], g[1], g[2], g[1], g[3], g[4], g[2], g[4], g[5]};
        const double H[9] = {g[6], g[7], g[8], g[7], g[9], g[10], g[8], g[10], g[11]};
        double c[3];
        const double piv = sizeof(V) == 4 ? kRrPivot32 : kRrPivot64;
        double th = rr3(G, H, true, pvalid, c, piv);
        if (!(th > 0.0) && pvalid) th = rr3(G, H, true, false, c, piv);  // again without p
        double nx = 0.0, np = 0.0;
        if (th > 0.0)
          for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
              nx += c[a] * G[a * 3 + b] * c[b];
              if (a > 0 && b > 0) np += c[a] * G[a * 3 + b] * c[b];
            }
        const bool ok = th > 0.0 && nx > 0.0;
        const double ix = ok ? 1.0 / sqrt(nx) : 0.0;
        const double ip = (ok && np > 1e-300) ? 1.0 / sqrt(np) : 0.0;
        bc[0] = ok ? 1.0 : 0.0;
        bc[1] = c[0] * ix;
        bc[2] = c[1] * ix;
        bc[3] = c[2] * ix;
        bc[4] = c[1] * ip;
        bc[5] = c[2] * ip;
        bc[6] = ip > 0.0 ? 1.0 : 0.0;
      }
      __syncthreads();
      const bool ok = bc[0] != 0.0;
      const V a0 = (V)bc[1], a1 = (V)bc[2], a2 = (V)bc[3], b1 = (V)bc[4], b2 = (V)bc[5];
      const bool pnext = bc[6] != 0.0;
      __syncthreads();
      if (!ok) break;  // no step left (w and p dependent on x): x is final
      // x <- a0 x + a1 w + a2 p,  p <- b1 w + b2 p  (means removed)
      {
        const V mx = (V)mux, mp = (V)mup, mw = (V)muw;
        for (int i = tid; i < n; i += nthr) {
          const V xh = X[i] - mx, wh = W[i] - mw, ph = pvalid ? P[i] - mp : (V)0;
          X[i] = a0 * xh + a1 * wh + a2 * ph;
          if (pnext) P[i] = b1 * wh + b2 * ph;
        }
        mux = 0.0;
        pvalid = pnext;
        if (!sync()) return false;
      }
    }
    if (lead()) {
      L->x = X;
      L->y = W;
      L->mu = mux;
      L->s = 1.0;
      L->refine_iters = iters;
      L->capped |= capped;
    }
    return sync();
  }

  // ---- A11: Rayleigh quotient, residual, orthogonality, sign, output --------
  FZD bool finalize() {
    const int n = S->lv[0].n, nnz = S->lv[0].nnz;
    if (GRID && vdbl(n, nnz) && sizeof(T) != 8) {  // see smooth()
      fail(ST_ENOTSUP);
      return false;
    }
    return (!GRID && vdbl(n, nnz)) ? finalize_v<double>() : finalize_v<T>();
  }

  template <class V>
  FZD bool finalize_v() {
    cur_level = 0;
    Level *L = &S->lv[0];
    const int n = L->n, nnz = L->nnz;
    const int *srp = L->srowptr, *scol = L->scol, *perm = L->perm, *iperm = L->iperm;
    const V *sw = (const V *)L->sw;
    const V *A = (const V *)L->x;
    const double mu = L->mu, s = L->s;
    // x_hat = (x - mu) * s.  The edge form needs only differences x_i - x_j,
    // in which mu cancels: per row, sum_j w (x_i - x_j) and sum_j w (x_i - x_j)^2
    // are taken in V (neighbouring values of a smooth vector are close, so
    // their difference is exact in V) and accumulated over rows in FP64, scaled
    // by s and s^2 at the end.
    // the row sums (L x)_k / s are kept in y for the residual pass below
    V *LXk = (V *)L->y;
    double acc[3] = {0.0, 0.0, 0.0};
    IRed big{0, 0, LLONG_MIN};
    auto row = [&](int k, V xi, V lx, V num) {
      const double xk = ((double)xi - mu) * s;
      acc[0] += xk * xk;
      acc[1] += xk;
      acc[2] += (double)num;
      LXk[k] = lx;
      big.mx = max(big.mx, (long long)__double_as_longlong(fabs(xk)));
    };
    const int nl = L->colstart[L->ncolors];  // light rows [0, nl), heavy rows [nl, n)
    const int lane = threadIdx.x & 31, gw = tid >> 5, nwarp = nthr >> 5;
    {
      for (int k = tid; k < nl; k += nthr) {
        const V xi = A[k];
        V lx = (V)0, num = (V)0;
        const int e1 = srp[k + 1];
        for (int e = srp[k]; e < e1; e++) {
          const V dl = xi - A[scol[e]];
          const V wd = sw[e] * dl;
          lx += wd;
          num += wd * dl;
        }
        row(k, xi, lx, num);
      }
      with_group<GRID>(heavy_group(srp, nl, n), [&](auto gs) {  // heavy rows: a group of lanes each
        constexpr int G = decltype(gs)::value, GW = 32 / G;
        const int gl = lane & (G - 1), gi = lane / G;
        for (int base = nl + gw * GW; base < n; base += nwarp * GW) {
          const int k = base + gi;
          V xi = (V)0, lx = (V)0, num = (V)0;
          if (k < n) {
            xi = A[k];
            group_row<G>(srp[k], srp[k + 1], scol, sw, [&](int j, V wv) {
              const V dl = xi - A[j];
              const V wd = wv * dl;
              lx += wd;
              num += wd * dl;
            });
          }
          lx = group_sum<G>(lx);
          num = group_sum<G>(num);
          if (gl == 0 && k < n) row(k, xi, lx, num);
        }
      });
    }
    if (!grid_dsum<3>(acc)) return false;
    acc[2] *= s * s;
    // residual ||L x - lambda x|| / ||x|| from its own sum of squares (a
    // difference of ||L x||^2 and lambda^2 ||x||^2 would cancel when the
    // residual is small)
    const double lam0 = acc[2] / (2.0 * acc[0]);
    double rac[1] = {0.0};
    for (int k = tid; k < n; k += nthr) {
      const double xk = ((double)A[k] - mu) * s;
      const double rk = s * (double)LXk[k] - lam0 * xk;
      rac[0] += rk * rk;
    }
    if (!grid_dsum<1>(rac)) return false;
    if (!grid_ired(big)) return false;
    // lowest original index among the entries of largest |x|
    const long long bits = big.mx;
    IRed low{0, 0, LLONG_MIN};
    for (int k = tid; k < n; k += nthr) {
      const double xk = ((double)A[k] - mu) * s;
      if ((long long)__double_as_longlong(fabs(xk)) == bits) low.mx = max(low.mx, -(long long)perm[k]);
    }
    if (!grid_ired(low)) return false;
    const int imax = (int)(-low.mx);
    const double xx = acc[0];
    const double lam = lam0;
    const double r2 = rac[0] / xx;
    const double xbig = ((double)A[iperm[imax]] - mu) * s;
    const double sign = xbig < 0.0 ? -1.0 : 1.0;
    const double inv = sign / sqrt(xx);
    double *out = S->xout;
    if (out)
      for (int k = tid; k < n; k += nthr) out[perm[k]] = ((double)A[k] - mu) * s * inv;
    int ptot = 0, gtot = 0, rtot = 0, cap = 0;
    for (int l = 0; l < nlevels; l++) {
      ptot += S->lv[l].pi_iters;
      gtot += S->lv[l].gs_sweeps;
      rtot += S->lv[l].refine_iters;
      cap |= S->lv[l].capped;
    }
    if (lead()) {
      S->lambda = lam;
      S->residual = sqrt(fmax(r2, 0.0));
      S->ortho = fabs(acc[1]) / (sqrt((double)n) * sqrt(xx));
      S->pi_total = ptot;
      S->gs_total = gtot;
      S->refine_total = rtot;
      S->capped = cap;
    }
    if (!sync()) return false;
    FZ_MARK(PH_FINAL, 4.0 * (n + 1) + (4.0 + sizeof(V)) * nnz + (4.0 * sizeof(V) + 8.0 + 8.0) * n);
    return true;
  }

  // ---- the walk over the hierarchy ------------------------------------------
  // mode 0: setup only; 1: everything eligible; 2: solve only
  FZD bool run(int mode) {
    if (status() != 0) return false;
    if (mode != 2) {
      if (nlevels == 0) {
        if (!elig(S->n0, S->nnz0)) return true;
        if (!ingest()) return false;
        nlevels = 1;
        persist();
      }
      while (!setup_done) {
        const int l = nlevels - 1;
        const int n = S->lv[l].n;
        if (!elig(n, S->lv[l].nnz)) return true;
        soff = 0;  // the level's scratch: colouring, matching, Galerkin
        if (!jp_start(l)) return false;
        bool last = n <= S->opt.coarse_max_n || nlevels >= S->opt.max_levels;
        GalerkinScratch G;
        int nc = -1;
        if (!last) {
          if (S->opt.hec_mode == 1) {
            if (!hec_paper(l, nc, G)) return false;
          } else {
            if (!match(l)) return false;
            if (!aggregate(l, nc, G)) return false;
          }
          last = nc < 0;
          if (!last && !galerkin(l, nc, G)) return false;
        }
        if (!jp_finish()) return false;
        if (!reorder(l)) return false;
        if (last) {
          setup_done = 1;
          coarsest = l;
          persist();
          break;
        }
        nlevels++;
        persist();
      }
    }
    if (mode == 0) return true;
    if (!setup_done) return true;
    if (!coarsest_solved) {
      if (!elig(S->lv[coarsest].n, S->lv[coarsest].nnz)) return true;
      if (!coarsest_solve(coarsest)) return false;
      coarsest_solved = 1;
      solved = coarsest;
      persist();
    }
    while (solved > 0) {
      const int l = solved - 1;
      if (!elig(S->lv[l].n, S->lv[l].nnz)) return true;
      if (!prolong(l)) return false;
      solved = l;
      persist();
    }
    if (S->opt.refine && !refined) {
      if (!refine()) return false;
      refined = 1;
      persist();
    }
    if (!finalized) {
      if (!finalize()) return false;
      finalized = 1;
      persist();
    }
    return true;
  }
};

// fault injection for the bounded-wait test: block 0 leaves before the first
// barrier, so every other block's wait runs out and reports ETIMEOUT
template <class T, bool GRID>
FZD void engine_entry(State *S, int mode) {
  if (GRID && S->opt.fault_inject == 1 && blockIdx.x == 0) return;
  Eng<T, GRID> E;
  E.init(S);
  E.run(mode);
  E.persist();
  E.flush_profile();
}

// Batched form: persistent blocks pull graph indices from a device counter
// and run the one-block engine on each graph's own state, with the block's
// private scratch slot.  A graph's computation does not depend on which block
// runs it or on the other graphs of the batch.
template <class T>
FZD void batch_entry(State *states, int count, int *next, char *scratch, unsigned long long slot_bytes) {
  __shared__ int s_g;
  for (;;) {
    if (threadIdx.x == 0) s_g = atomicAdd(next, 1);
    __syncthreads();
    const int g = s_g;
    __syncthreads();
    if (g >= count) return;
    State *S = states + g;
    if (threadIdx.x == 0) {
      S->scratch = scratch + (size_t)blockIdx.x * slot_bytes;
      S->scratch_size = slot_bytes;
    }
    __syncthreads();
    engine_entry<T, false>(S, 1);
    __syncthreads();
  }
}

// Serving form: resident blocks claim published tickets one at a time (each
// ticket's state carries its own arena and scratch) and flag each one as soon
// as it is finished, so a long solve holds only its own block.  A block with
// no work waits briefly (bounded by ring->idle_ns, checking the ring with
// backoff), then leaves and says so (block base + b flags exited[]); the host
// keeps as many blocks alive as there is work, launching more when needed.
template <class T>
FZD void serve_entry(ServeRing *ring, ServeDone *fin, unsigned long long base) {
  __shared__ long long s_k;
  for (;;) {
    if (threadIdx.x == 0) {
      long long got = -1;
      const uint64_t t0 = gtime();
      volatile ServeRing *vr = ring;
      for (;;) {
        const unsigned long long tail = vr->tail;
        const unsigned long long h = vr->head;
        if (h < tail) {
          if (atomicCAS(&ring->head, h, h + 1) == h) {
            got = (long long)h;
            break;
          }
          continue;
        }
        if (vr->stop || gtime() - t0 > vr->idle_ns) break;
        __nanosleep(2000);
      }
      s_k = got;
    }
    __syncthreads();
    const long long k = s_k;
    __syncthreads();
    if (k < 0) {
      if (threadIdx.x == 0) {
        const unsigned long long g = base + blockIdx.x;
        ((volatile unsigned long long *)fin->exited)[g % kExitRing] = g + 1ull;
      }
      return;
    }
    __threadfence();
    State *S = ((State *volatile *)ring->item)[k % kRing];
    engine_entry<T, false>(S, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence_system();  // the state's results before the flag
      ((volatile unsigned long long *)fin->done)[k % kRing] = (unsigned long long)k + 1ull;
    }
  }
}

}  // namespace fz
