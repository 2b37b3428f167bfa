// partition.h -- device steps of the recursive spectral bisection
// (fiedler_partition): induced subgraphs of one part, the sign split of a
// Fiedler vector, connected components of a subgraph.  Every function queues
// kernels on `stream` and returns the first CUDA error; counts that the host
// needs are copied into pinned host memory given by the caller and are valid
// after the stream is synchronised.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fz {

// scratch of the partition steps for graphs of up to n vertices
struct PartScratch {
  int *keep;    // [n + 1] flags, then their exclusive scan (new ids)
  int *cnt;     // [n + 1] kept entries per kept row, then the sub rowptr
  int *bsum;    // [blocks + 1] block totals of the scans
  int *flag;    // [2] device counters
};
size_t part_scratch_ints(int64_t n);

// Induced subgraph of the vertices v with label[v] == p (kept vertices in
// ascending order; entries in the parent's order): sub rowptr/col/w (same
// weight type as the parent, w_f64) and map[i] = parent vertex of sub vertex
// i.  *h_counts receives {vertices, entries} of the subgraph.
cudaError_t part_extract(const int32_t *rowptr, const int32_t *col, const void *w, int w_f64, int64_t n,
                         const int32_t *label, int p, int32_t *sub_rowptr, int32_t *sub_col, void *sub_w,
                         int32_t *map, PartScratch &s, int *h_counts, cudaStream_t stream);

// label[map[i]] = newp for every sub vertex i with x[i] < 0 (the sign cut of
// the Fiedler vector); *h_moved receives their number.
cudaError_t part_split_sign(const double *x, int64_t m, const int32_t *map, int32_t *label, int newp,
                            PartScratch &s, int *h_moved, cudaStream_t stream);

// Connected components of the subgraph (min-label propagation with pointer
// jumping; comp[i] = the smallest vertex of i's component), then
// label[map[i]] = newp for every vertex outside the component of vertex 0;
// *h_moved receives their number.
cudaError_t part_split_components(const int32_t *sub_rowptr, const int32_t *sub_col, int64_t m,
                                  const int32_t *map, int32_t *label, int newp, int32_t *comp, PartScratch &s,
                                  int *h_moved, cudaStream_t stream);

}  // namespace fz
