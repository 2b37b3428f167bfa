// engine_f64.cu -- double instantiation of the level engine: the kernel table (the
// kernels themselves are in engine_f64_setup.cu, engine_f64_solve.cu,
// engine_f64_cta.cu and engine_batch*_f64.cu).
#include "kernels.h"

namespace fz {

void kernels_f64(KernelSet *k) {
  grid_setup_kernel_f64(k);
  grid_solve_kernel_f64(k);
  cta_kernel_f64(k);
  k->names[0] = "fz_grid_setup_f64";
  k->names[1] = "fz_cta_f64";
  k->names[2] = "fz_grid_solve_f64";
  batch_kernel512_f64(k);
  batch_kernel256_f64(k);
  batch_kernel128_f64(k);
  k->batch = k->batch_v[0];
  k->names[3] = k->batch_names[0];
}

}  // namespace fz
