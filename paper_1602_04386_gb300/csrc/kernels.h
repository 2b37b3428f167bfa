// kernels.h -- host-visible handles of the engine kernels (one set per value type)
#pragma once
#include "fz_state.h"

namespace fz {
struct KernelSet {
  const void *grid_setup;  // cooperative, kGridThreads per block: setup of the large levels
  const void *grid_solve;  // cooperative, kGridThreads per block: solve of the large levels
  const void *cta;         // one block of kCtaThreads: everything on the small levels
  const void *batch;       // persistent blocks of kCtaThreads, one graph at a time each
  const char *names[4];    // profile slots: grid_setup, cta, grid_solve, batch
};
void kernels_f32(KernelSet *k);
void kernels_f64(KernelSet *k);
}  // namespace fz
