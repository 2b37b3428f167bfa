// engine_f32_solve.cu -- float instantiation of the level engine: the grid solve kernel.
// Each kernel of the single-graph solve has a translation unit of its own, so
// that they compile in parallel.
#include "engine.cuh"
#include "kernels.h"

namespace fz {

__global__ void __launch_bounds__(kGridThreads, 1) fz_grid_solve_f32(State *S) { engine_entry<float, true>(S, 2); }

void grid_solve_kernel_f32(KernelSet *k) { k->grid_solve = (const void *)fz_grid_solve_f32; }

}  // namespace fz
