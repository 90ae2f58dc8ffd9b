// lra_batched_k512.cu -- the batched C-A kernel for CTAs of 512 threads,
// 1 per SM (one translation unit per shape keeps the build parallel).
#include "lra_batched_kernel.cuh"

namespace lra {

void* batched_kernel_512(bool mixed, bool pairs) {
  if (pairs) return mixed ? nullptr : reinterpret_cast<void*>(ca_batched_kernel<false, 512, 1, true>);
  return mixed ? reinterpret_cast<void*>(ca_batched_kernel<true, 512, 1>)
               : reinterpret_cast<void*>(ca_batched_kernel<false, 512, 1>);
}

}  // namespace lra
