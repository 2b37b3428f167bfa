// engine_f64_cta.cu -- double instantiation of the level engine: the cta kernel.
// Each kernel of the single-graph solve has a translation unit of its own, so
// that they compile in parallel.
#include "engine.cuh"
#include "kernels.h"

namespace fz {

__global__ void __launch_bounds__(kCtaThreads, 1) fz_cta_f64(State *S) { engine_entry<double, false>(S, 1); }

void cta_kernel_f64(KernelSet *k) { k->cta = (const void *)fz_cta_f64; }

}  // namespace fz
