// engine_f32.cu -- float instantiation of the level engine.
#include "engine.cuh"
#include "kernels.h"

namespace fz {

__global__ void __launch_bounds__(kGridThreads, 2) fz_grid_setup_f32(State *S) { engine_entry<float, true>(S, 0); }
__global__ void __launch_bounds__(kGridThreads, 2) fz_grid_solve_f32(State *S) { engine_entry<float, true>(S, 2); }
__global__ void __launch_bounds__(kCtaThreads, 1) fz_cta_f32(State *S) { engine_entry<float, false>(S, 1); }
__global__ void __launch_bounds__(kCtaThreads, 1)
    fz_batch_f32(State *states, int count, int *next, char *scratch, unsigned long long slot_bytes) {
  batch_entry<float>(states, count, next, scratch, slot_bytes);
}

void kernels_f32(KernelSet *k) {
  k->grid_setup = (const void *)fz_grid_setup_f32;
  k->grid_solve = (const void *)fz_grid_solve_f32;
  k->cta = (const void *)fz_cta_f32;
  k->batch = (const void *)fz_batch_f32;
  k->names[0] = "fz_grid_setup_f32";
  k->names[1] = "fz_cta_f32";
  k->names[2] = "fz_grid_solve_f32";
  k->names[3] = "fz_batch_f32";
}

}  // namespace fz
