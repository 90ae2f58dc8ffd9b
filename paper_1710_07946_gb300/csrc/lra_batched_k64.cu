// lra_batched_k64.cu -- the batched C-A kernel for CTAs of 64 threads,
// 8 per SM (one translation unit per shape keeps the build parallel).
#include "lra_batched_kernel.cuh"

namespace lra {

void* batched_kernel_64(bool mixed) {
  return mixed ? reinterpret_cast<void*>(ca_batched_kernel<true, 64, 8>)
               : reinterpret_cast<void*>(ca_batched_kernel<false, 64, 8>);
}

}  // namespace lra
