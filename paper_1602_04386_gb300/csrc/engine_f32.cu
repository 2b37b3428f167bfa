// engine_f32.cu -- float instantiation of the level engine.
#include "engine.cuh"
#include "kernels.h"

namespace fz {

__global__ void __launch_bounds__(kGridThreads, 2) fz_grid_setup_f32(State *S) { engine_entry<float, true>(S, 0); }
__global__ void __launch_bounds__(kGridThreads, 2) fz_grid_solve_f32(State *S) { engine_entry<float, true>(S, 2); }
__global__ void __launch_bounds__(kCtaThreads, 1) fz_cta_f32(State *S) { engine_entry<float, false>(S, 1); }

void kernels_f32(KernelSet *k) {
  k->grid_setup = (const void *)fz_grid_setup_f32;
  k->grid_solve = (const void *)fz_grid_solve_f32;
  k->cta = (const void *)fz_cta_f32;
  k->names[0] = "fz_grid_setup_f32";
  k->names[1] = "fz_cta_f32";
  k->names[2] = "fz_grid_solve_f32";
  batch_kernel512_f32(k);
  batch_kernel256_f32(k);
  batch_kernel128_f32(k);
  k->batch = k->batch_v[0];
  k->names[3] = k->batch_names[0];
}

}  // namespace fz
