// lra_profile.h -- RAII scope around each kernel launch of the library
// (launch counting; an NVTX range; CUDA-event timing when enabled).
#pragma once

#include <cuda_runtime.h>

namespace lra {

class LaunchScope {
 public:
  LaunchScope(cudaStream_t s, const char* name);
  ~LaunchScope();
  LaunchScope(const LaunchScope&) = delete;
  LaunchScope& operator=(const LaunchScope&) = delete;

 private:
  cudaStream_t stream_;
  const char* name_;
  cudaEvent_t a_, b_;
};

}  // namespace lra
