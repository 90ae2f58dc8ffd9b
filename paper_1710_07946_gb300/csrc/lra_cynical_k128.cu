// lra_cynical_k128.cu -- the cynical CUR kernel for CTAs of 128 threads,
// 4 per SM (one translation unit per shape keeps the build parallel).
#include "lra_cynical_kernel.cuh"

namespace lra {

const void* cynical_kernel_128() { return reinterpret_cast<const void*>(cynical_batched_kernel<128, 4>); }

}  // namespace lra
