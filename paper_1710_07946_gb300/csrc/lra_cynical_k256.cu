// lra_cynical_k256.cu -- the cynical CUR kernel for CTAs of 256 threads,
// 2 per SM (one translation unit per shape keeps the build parallel).
#include "lra_cynical_kernel.cuh"

namespace lra {

const void* cynical_kernel_256() { return reinterpret_cast<const void*>(cynical_batched_kernel<256, 2>); }

}  // namespace lra
