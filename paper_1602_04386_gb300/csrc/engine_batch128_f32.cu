// engine_batch128_f32.cu -- float batched and serving kernels with 128 threads per graph's block
// (8 graphs resident per SM); one translation unit per variant so that
// they compile in parallel.
#include "engine.cuh"
#include "kernels.h"

namespace fz {

__global__ void __launch_bounds__(128, 8)
    fz_batch128_f32(State *states, int count, int *next, char *scratch, unsigned long long slot_bytes) {
  batch_entry<float>(states, count, next, scratch, slot_bytes);
}
__global__ void __launch_bounds__(128, 8) fz_serve128_f32(ServeRing *ring, ServeDone *fin,
                                                              unsigned long long base) {
  serve_entry<float>(ring, fin, base);
}

void batch_kernel128_f32(KernelSet *k) {
  k->batch_v[2] = (const void *)fz_batch128_f32;
  k->serve_v[2] = (const void *)fz_serve128_f32;
  k->batch_names[2] = "fz_batch128_f32";
}

}  // namespace fz
