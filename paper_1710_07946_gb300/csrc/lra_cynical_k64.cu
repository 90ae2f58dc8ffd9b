// lra_cynical_k64.cu -- the cynical CUR kernel for CTAs of 64 threads,
// 8 per SM (one translation unit per shape keeps the build parallel).
#include "lra_cynical_kernel.cuh"

namespace lra {

const void* cynical_kernel_64() { return reinterpret_cast<const void*>(cynical_batched_kernel<64, 8>); }

}  // namespace lra
