// engine_batch512_f32.cu -- float batched and serving kernels with 512 threads per graph's block
// (2 graphs resident per SM); one translation unit per variant so that
// they compile in parallel.
#include "engine.cuh"
#include "kernels.h"

namespace fz {

__global__ void __launch_bounds__(512, 2)
    fz_batch_f32(State *states, int count, int *next, char *scratch, unsigned long long slot_bytes) {
  batch_entry<float>(states, count, next, scratch, slot_bytes);
}
__global__ void __launch_bounds__(512, 2) fz_serve512_f32(ServeRing *ring, ServeDone *fin,
                                                              unsigned long long base) {
  serve_entry<float>(ring, fin, base);
}

void batch_kernel512_f32(KernelSet *k) {
  k->batch_v[0] = (const void *)fz_batch_f32;
  k->serve_v[0] = (const void *)fz_serve512_f32;
  k->batch_names[0] = "fz_batch_f32";
}

}  // namespace fz
