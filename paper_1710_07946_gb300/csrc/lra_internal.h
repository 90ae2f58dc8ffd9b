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
  int32_t side;         // LRA_SIDE_RIGHT (W' = W M) or LRA_SIDE_LEFT (W' = M^T W)
  int64_t n;
  int32_t param;        // depth d (ARHT), nnz (sparse) or the number of factors q (bidiagonal)
  int32_t width;        // bidiagonal: slots per column, min(2^q, n)
  int32_t* d_idx;       // ARHT perm (n), sparse rows (n*nnz) or bidiagonal rows (n*width)
  int8_t* d_sign;       // ARHT diagonal (n) or sparse signs (n*nnz)
  int32_t* d_val;       // bidiagonal integer weights (n*width)
  double* d_dense;      // bidiagonal with 2^q >= n: the integers of M as an n x n row-major matrix, else null
  double* d_wt;         // ARFT real form: 2n x 2^d real weights (rows in d_idx), else null
  double scale;         // 2^{-d/2}, 1/sqrt(nnz) or 2^{-q/2}
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

// Autotuner core: runs launch(i) reps times for each i < n (a launch returning
// LRA_ERR_INVALID_ARG marks shape i as unusable, time -1), timing each launch
// with CUDA events on the stream, and returns the fastest usable i in *best.
template <class Launch>
lra_status time_shapes(int n, int reps, cudaStream_t stream, Launch launch, float* ms, int* best) {
  cudaEvent_t e0, e1;
  LRA_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return LRA_ERR_CUDA; }
  lra_status st = LRA_OK;
  float bt = 0.f;
  int bi = -1;
  for (int i = 0; i < n && st == LRA_OK; ++i) {
    float fastest = -1.f;
    for (int r = 0; r < reps; ++r) {
      if (cudaEventRecord(e0, stream) != cudaSuccess) { st = LRA_ERR_CUDA; break; }
      const lra_status ls = launch(i);
      if (ls == LRA_ERR_INVALID_ARG) { fastest = -1.f; break; }
      if (ls != LRA_OK) { st = ls; break; }
      float t = 0.f;
      if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) { st = LRA_ERR_CUDA; break; }
      if (fastest < 0.f || t < fastest) fastest = t;
    }
    if (ms != nullptr) ms[i] = fastest;
    if (fastest >= 0.f && (bi < 0 || fastest < bt)) { bt = fastest; bi = i; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LRA_OK) return st;
  if (bi < 0) return LRA_ERR_INVALID_ARG;
  *best = bi;
  return LRA_OK;
}

// Staged generator sizes of lra_ca_params: none, or ascending sizes >= 1 that
// end at par->k, with a margin >= 0.
inline bool stages_valid(const lra_ca_params* par) {
  if (par->nstages == 0) return true;
  if (par->nstages < 0 || par->nstages > LRA_MAX_STAGES || par->rank_margin < 0) return false;
  for (int s = 0; s < par->nstages; ++s) {
    if (par->k_stages[s] < 1) return false;
    if (s > 0 && par->k_stages[s] <= par->k_stages[s - 1]) return false;
  }
  return par->k_stages[par->nstages - 1] == par->k;
}

// Inputs whose maxvol steps the certified FP32 mode handles: dense inputs and
// the FP64 Laplace kernel (its FP32 bounds are relative to the FP64 entries),
// without the bidiagonal-product multiplier.
inline bool mixed_supported(const DevProblem& P) {
  if (P.mkind == LRA_MULT_BIDIAG) return false;       // no FP32 bounds for integer-weighted sums
  if (P.mside != 0) return false;                     // FP32 gathers are written for right multipliers
  if (P.mkind == LRA_MULT_ARFT) return false;         // nor for the real-weighted Fourier columns
  return P.src == LRA_DENSE || (P.src == LRA_KERNEL_LAPLACE && P.dtype == LRA_F64);
}

}  // namespace lra
