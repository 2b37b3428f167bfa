// partition.cu -- device steps of the recursive spectral bisection: induced
// subgraphs, the sign cut of a Fiedler vector, connected components.
#include "partition.h"

namespace fz {
namespace {

constexpr int kT = 256;          // threads per block
constexpr int kItems = 4;        // scan items per thread
constexpr int kTile = kT * kItems;

__device__ __forceinline__ int warp_incl(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// exclusive scan of v over the block (kT threads); *tot = block sum
__device__ int block_excl(int v, int *tot) {
  __shared__ int ws[kT / 32 + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int inc = warp_incl(v);
  if (lane == 31) ws[w] = inc;
  __syncthreads();
  if (w == 0) {
    int t = lane < kT / 32 ? ws[lane] : 0;
    t = warp_incl(t);
    if (lane < kT / 32) ws[lane] = t;
  }
  __syncthreads();
  const int ex = inc - v + (w > 0 ? ws[w - 1] : 0);
  *tot = ws[kT / 32 - 1];
  __syncthreads();
  return ex;
}

// a[0, n) -> exclusive scan per tile; bsum[b] = tile total
__global__ void k_scan_tile(int *a, int64_t n, int *bsum) {
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
  int v[kItems], s = 0;
#pragma unroll
  for (int k = 0; k < kItems; k++) {
    v[k] = base + k < n ? a[base + k] : 0;
    s += v[k];
  }
  int tot;
  int run = block_excl(s, &tot);
#pragma unroll
  for (int k = 0; k < kItems; k++) {
    if (base + k < n) a[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// bsum[0, nb) -> exclusive scan, bsum[nb] = total (one block)
__global__ void k_scan_sums(int *bsum, int nb) {
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += kT) {
    const int b = b0 + threadIdx.x;
    const int v = b < nb ? bsum[b] : 0;
    int tot;
    const int ex = block_excl(v, &tot);
    if (b < nb) bsum[b] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void k_scan_add(int *a, int64_t n, const int *bsum, int nb) {
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i < n) a[i] += bsum[i / kTile];
  if (i == 0) a[n] = bsum[nb];
}

// exclusive scan of a[0, n) into a[0, n], a[n] = total
cudaError_t scan_excl(int *a, int64_t n, int *bsum, cudaStream_t st) {
  const int nb = (int)((n + kTile - 1) / kTile);
  if (nb > 0) k_scan_tile<<<nb, kT, 0, st>>>(a, n, bsum);
  k_scan_sums<<<1, kT, 0, st>>>(bsum, nb);
  k_scan_add<<<(unsigned)((n + kT) / kT), kT, 0, st>>>(a, n, bsum, nb);
  return cudaGetLastError();
}

__global__ void k_keep(const int32_t *label, int p, int64_t n, int *keep) {
  const int64_t v = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (v < n) keep[v] = label[v] == p;
}

// kept entries of every kept row, at the row's new id; map new id -> vertex
__global__ void k_rowcount(const int32_t *rowptr, const int32_t *col, const int32_t *label, int p, int64_t n,
                           const int *newid, int *cnt, int32_t *map) {
  const int64_t v = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (v >= n || label[v] != p) return;
  int c = 0;
  for (int e = rowptr[v]; e < rowptr[v + 1]; e++) c += label[col[e]] == p;
  cnt[newid[v]] = c;
  map[newid[v]] = (int32_t)v;
}

template <class W>
__global__ void k_fill(const int32_t *rowptr, const int32_t *col, const W *w, const int32_t *label, int p, int64_t n,
                       const int *newid, const int *subrp, int32_t *subcol, W *subw) {
  const int64_t v = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (v >= n || label[v] != p) return;
  int o = subrp[newid[v]];
  for (int e = rowptr[v]; e < rowptr[v + 1]; e++) {
    const int u = col[e];
    if (label[u] != p) continue;
    subcol[o] = newid[u];
    subw[o] = w[e];
    o++;
  }
}

__global__ void k_copy_int(const int *a, int32_t *b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i <= n) b[i] = a[i];
}

__global__ void k_split_sign(const double *x, int64_t m, const int32_t *map, int32_t *label, int newp, int *moved) {
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  int c = 0;
  if (i < m && x[i] < 0.0) {
    label[map[i]] = newp;
    c = 1;
  }
  c = __syncthreads_count(c);
  if (threadIdx.x == 0 && c) atomicAdd(moved, c);
}

__global__ void k_comp_init(int32_t *comp, int64_t m) {
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i < m) comp[i] = (int32_t)i;
}

// comp[i] = min(comp[i], comp of the neighbours), then one pointer jump
__global__ void k_comp_step(const int32_t *rp, const int32_t *ci, int64_t m, int32_t *comp, int *changed) {
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i >= m) return;
  int c = comp[i];
  for (int e = rp[i]; e < rp[i + 1]; e++) c = min(c, comp[ci[e]]);
  c = min(c, comp[c]);
  if (c < comp[i]) {
    comp[i] = c;
    *changed = 1;
  }
}

__global__ void k_split_comp(const int32_t *comp, int64_t m, const int32_t *map, int32_t *label, int newp,
                             int *moved) {
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  int c = 0;
  if (i < m && comp[i] != 0) {
    label[map[i]] = newp;
    c = 1;
  }
  c = __syncthreads_count(c);
  if (threadIdx.x == 0 && c) atomicAdd(moved, c);
}

unsigned blocks(int64_t n) { return (unsigned)((n + kT - 1) / kT > 0 ? (n + kT - 1) / kT : 1); }

}  // namespace

size_t part_scratch_ints(int64_t n) { return 2 * (size_t)(n + 1) + (size_t)(n / kTile + 2) + 2; }

cudaError_t part_extract(const int32_t *rowptr, const int32_t *col, const void *w, int w_f64, int64_t n,
                         const int32_t *label, int p, int32_t *sub_rowptr, int32_t *sub_col, void *sub_w,
                         int32_t *map, PartScratch &s, int *h_counts, cudaStream_t st) {
  k_keep<<<blocks(n), kT, 0, st>>>(label, p, n, s.keep);
  cudaError_t e = scan_excl(s.keep, n, s.bsum, st);
  if (e != cudaSuccess) return e;
  // s.keep[v] is now v's new id (for kept v), s.keep[n] the number kept
  k_rowcount<<<blocks(n), kT, 0, st>>>(rowptr, col, label, p, n, s.keep, s.cnt, map);
  if ((e = cudaMemcpyAsync(&h_counts[0], s.keep + n, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  const int64_t m = h_counts[0];
  if ((e = scan_excl(s.cnt, m, s.bsum, st)) != cudaSuccess) return e;
  k_copy_int<<<blocks(m + 1), kT, 0, st>>>(s.cnt, sub_rowptr, m);
  if (w_f64)
    k_fill<double><<<blocks(n), kT, 0, st>>>(rowptr, col, (const double *)w, label, p, n, s.keep, s.cnt, sub_col,
                                            (double *)sub_w);
  else
    k_fill<float><<<blocks(n), kT, 0, st>>>(rowptr, col, (const float *)w, label, p, n, s.keep, s.cnt, sub_col,
                                           (float *)sub_w);
  if ((e = cudaMemcpyAsync(&h_counts[1], s.cnt + m, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t part_split_sign(const double *x, int64_t m, const int32_t *map, int32_t *label, int newp, PartScratch &s,
                            int *h_moved, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(s.flag, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_split_sign<<<blocks(m), kT, 0, st>>>(x, m, map, label, newp, s.flag);
  if ((e = cudaMemcpyAsync(h_moved, s.flag, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t part_split_components(const int32_t *rp, const int32_t *ci, int64_t m, const int32_t *map, int32_t *label,
                                  int newp, int32_t *comp, PartScratch &s, int *h_moved, cudaStream_t st) {
  k_comp_init<<<blocks(m), kT, 0, st>>>(comp, m);
  cudaError_t e;
  // every step lowers some label or leaves all fixed; at most m steps
  for (int64_t it = 0; it <= m; it += 8) {
    if ((e = cudaMemsetAsync(s.flag, 0, sizeof(int), st)) != cudaSuccess) return e;
    for (int k = 0; k < 8; k++) k_comp_step<<<blocks(m), kT, 0, st>>>(rp, ci, m, comp, s.flag);
    if ((e = cudaMemcpyAsync(h_moved, s.flag, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if (*h_moved == 0) break;
  }
  if ((e = cudaMemsetAsync(s.flag + 1, 0, sizeof(int), st)) != cudaSuccess) return e;
  k_split_comp<<<blocks(m), kT, 0, st>>>(comp, m, map, label, newp, s.flag + 1);
  if ((e = cudaMemcpyAsync(h_moved, s.flag + 1, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace fz
