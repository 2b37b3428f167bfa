// engine_f32_cta.cu -- float instantiation of the level engine: the cta kernel.
// Each kernel of the single-graph solve has a translation unit of its own, so
// that they compile in parallel.
#include "engine.cuh"
#include "kernels.h"

namespace fz {

__global__ void __launch_bounds__(kCtaThreads, 1) fz_cta_f32(State *S) { engine_entry<float, false>(S, 1); }

void cta_kernel_f32(KernelSet *k) { k->cta = (const void *)fz_cta_f32; }

}  // namespace fz
