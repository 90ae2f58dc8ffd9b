// lra_batched_k128.cu -- the batched C-A kernel for CTAs of 128 threads,
// 4 per SM (one translation unit per shape keeps the build parallel).
#include "lra_batched_kernel.cuh"

namespace lra {

void* batched_kernel_128(bool mixed) {
  return mixed ? reinterpret_cast<void*>(ca_batched_kernel<true, 128, 4>)
               : reinterpret_cast<void*>(ca_batched_kernel<false, 128, 4>);
}

}  // namespace lra
