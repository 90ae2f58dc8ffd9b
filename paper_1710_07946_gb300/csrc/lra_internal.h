// lra_internal.h -- host-side pieces shared by the translation units of the
// library: the multiplier handle, problem validation and conversion to the
// device view, CUDA error mapping, device properties.
#pragma once

#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>

#include "lra.h"
#include "lra_device.cuh"

struct lra_multiplier_s {
  int32_t kind;
  int64_t n;
  int32_t param;        // depth d (ARHT) or nnz (sparse)
  int32_t* d_idx;       // ARHT perm (n) or sparse rows (n*nnz)
  int8_t* d_sign;       // ARHT diagonal (n) or sparse signs (n*nnz)
  double scale;         // 2^{-d/2} or 1/sqrt(nnz)
};

namespace lra {

inline lra_status cuda_status(cudaError_t e) { return e == cudaSuccess ? LRA_OK : LRA_ERR_CUDA; }

#define LRA_CUDA_TRY(expr)                              \
  do {                                                  \
    cudaError_t _e = (expr);                            \
    if (_e != cudaSuccess) return LRA_ERR_CUDA;         \
  } while (0)

// Validate a problem (and an optional multiplier) and fill the device view.
lra_status make_dev_problem(const lra_problem* p, lra_multiplier mult, DevProblem* out);

// Round the 3 x npts coordinates of X to FP32 into out (stream-ordered).
lra_status points_to_f32(const double* X, int64_t npts, float* out, cudaStream_t stream);

struct DeviceInfo {
  int device;
  int sms;
  size_t smem_optin;
};
lra_status current_device_info(DeviceInfo* info);

inline size_t align_up(size_t b, size_t a) { return (b + a - 1) / a * a; }

}  // namespace lra
