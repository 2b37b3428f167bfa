// engine_f32_setup.cu -- float instantiation of the level engine: the grid setup kernel.
// Each kernel of the single-graph solve has a translation unit of its own, so
// that they compile in parallel.
#include "engine.cuh"
#include "kernels.h"

namespace fz {

__global__ void __launch_bounds__(kGridThreads, 1) fz_grid_setup_f32(State *S) { engine_entry<float, true>(S, 0); }

void grid_setup_kernel_f32(KernelSet *k) { k->grid_setup = (const void *)fz_grid_setup_f32; }

}  // namespace fz
