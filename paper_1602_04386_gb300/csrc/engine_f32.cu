// engine_f32.cu -- float instantiation of the level engine: the kernel table (the
// kernels themselves are in engine_f32_setup.cu, engine_f32_solve.cu,
// engine_f32_cta.cu and engine_batch*_f32.cu).
#include "kernels.h"

namespace fz {

void kernels_f32(KernelSet *k) {
  grid_setup_kernel_f32(k);
  grid_solve_kernel_f32(k);
  cta_kernel_f32(k);
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
