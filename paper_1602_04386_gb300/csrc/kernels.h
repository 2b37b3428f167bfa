// kernels.h -- host-visible handles of the engine kernels (one set per value type)
#pragma once
#include "fz_state.h"

namespace fz {
struct KernelSet {
  const void *grid_setup;  // cooperative, kGridThreads per block: setup of the large levels
  const void *grid_solve;  // cooperative, kGridThreads per block: solve of the large levels
  const void *cta;         // one block of kCtaThreads: everything on the small levels
  const void *batch;       // persistent blocks of kCtaThreads, one graph at a time each
  const void *batch_v[3];  // the same with kBatchThreads[v] threads per block
  const void *serve_v[3];  // serving kernel (ring-fed), kBatchThreads[v] threads per block
  const char *names[4];    // profile slots: grid_setup, cta, grid_solve, batch
  const char *batch_names[3];
};
constexpr int kBatchThreads[3] = {512, 256, 128};
void kernels_f32(KernelSet *k);
void kernels_f64(KernelSet *k);
void grid_setup_kernel_f32(KernelSet *k);
void grid_solve_kernel_f32(KernelSet *k);
void cta_kernel_f32(KernelSet *k);
void grid_setup_kernel_f64(KernelSet *k);
void grid_solve_kernel_f64(KernelSet *k);
void cta_kernel_f64(KernelSet *k);
void batch_kernel512_f32(KernelSet *k);
void batch_kernel256_f32(KernelSet *k);
void batch_kernel128_f32(KernelSet *k);
void batch_kernel512_f64(KernelSet *k);
void batch_kernel256_f64(KernelSet *k);
void batch_kernel128_f64(KernelSet *k);
}  // namespace fz
