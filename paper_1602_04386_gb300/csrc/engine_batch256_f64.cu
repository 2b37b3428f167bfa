// engine_batch256_f64.cu -- double batched and serving kernels with 256 threads per graph's block
// (4 graphs resident per SM); one translation unit per variant so that
// they compile in parallel.
#include "engine.cuh"
#include "kernels.h"

namespace fz {

__global__ void __launch_bounds__(256, 4)
    fz_batch256_f64(State *states, int count, int *next, char *scratch, unsigned long long slot_bytes) {
  batch_entry<double>(states, count, next, scratch, slot_bytes);
}
__global__ void __launch_bounds__(256, 4) fz_serve256_f64(ServeRing *ring, ServeDone *fin,
                                                              unsigned long long base) {
  serve_entry<double>(ring, fin, base);
}

void batch_kernel256_f64(KernelSet *k) {
  k->batch_v[1] = (const void *)fz_batch256_f64;
  k->serve_v[1] = (const void *)fz_serve256_f64;
  k->batch_names[1] = "fz_batch256_f64";
}

}  // namespace fz
