// lra_batched_k256.cu -- the batched C-A kernel for CTAs of 256 threads,
// 2 per SM (one translation unit per shape keeps the build parallel).
#include "lra_batched_kernel.cuh"

namespace lra {

void* batched_kernel_256(bool mixed, bool pairs) {
  if (pairs) return mixed ? nullptr : reinterpret_cast<void*>(ca_batched_kernel<false, 256, 2, true>);
  return mixed ? reinterpret_cast<void*>(ca_batched_kernel<true, 256, 2>)
               : reinterpret_cast<void*>(ca_batched_kernel<false, 256, 2>);
}

}  // namespace lra
