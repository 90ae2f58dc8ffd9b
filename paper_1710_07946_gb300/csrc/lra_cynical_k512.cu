// lra_cynical_k512.cu -- the cynical CUR kernel for CTAs of 512 threads,
// 1 per SM (one translation unit per shape keeps the build parallel).
#include "lra_cynical_kernel.cuh"

namespace lra {

const void* cynical_kernel_512() { return reinterpret_cast<const void*>(cynical_batched_kernel<512, 1>); }

}  // namespace lra
