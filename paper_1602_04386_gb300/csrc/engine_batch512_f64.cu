// engine_batch512_f64.cu -- double batched and serving kernels with 512 threads per graph's block
// (2 graphs resident per SM); one translation unit per variant so that
// they compile in parallel.
#include "engine.cuh"
#include "kernels.h"

namespace fz {

__global__ void __launch_bounds__(512, 2)
    fz_batch_f64(State *states, int count, int *next, char *scratch, unsigned long long slot_bytes) {
  batch_entry<double>(states, count, next, scratch, slot_bytes);
}
__global__ void __launch_bounds__(512, 2) fz_serve512_f64(ServeRing *ring, ServeDone *fin,
                                                              unsigned long long base) {
  serve_entry<double>(ring, fin, base);
}

void batch_kernel512_f64(KernelSet *k) {
  k->batch_v[0] = (const void *)fz_batch_f64;
  k->serve_v[0] = (const void *)fz_serve512_f64;
  k->batch_names[0] = "fz_batch_f64";
}

}  // namespace fz
