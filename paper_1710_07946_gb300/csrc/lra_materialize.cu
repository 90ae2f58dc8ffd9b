// lra_materialize.cu -- the pre-processed input W' = W M written out densely,
// and the CUR's row factor R = W[I, :] gathered from the original input.
//
// The paper's bidiagonal pre-processing tests multiply the input by the
// factors before running C-A; with 20 factors every column of M is dense, so
// forming each entry of W' on the fly inside the C-A strips costs n terms per
// entry, strip after strip.  Written out once, W' feeds any number of C-A runs
// (or one batched launch over stacked copies) as a plain dense input.  Each
// entry is formed by the same device function the C-A gathers use (same terms,
// same order, same rounding), so the pivots of a C-A run on W' equal those of a
// run on (W, M); the CUR of W then takes R = W[I, :] (the original rows).
// Products of bidiagonal factors whose columns can all be full (2^q >= n) take
// a register-tiled dense product with the same per-entry fma chains.
#include <algorithm>

#include "lra_device.cuh"
#include "lra_internal.h"
#include "lra_profile.h"

namespace lra {

// One entry per thread: x over 32 consecutive columns (the rows of W they read
// are shared across the warp when the columns of M overlap), y over rows.
__global__ void __launch_bounds__(256) multiplier_apply_kernel(DevProblem P, double* __restrict__ Wp, int64_t ldwp) {
  const int64_t j = (int64_t)blockIdx.x * 32 + threadIdx.x;
  if (j >= pcols(P)) return;
  for (int64_t i = (int64_t)blockIdx.y * 8 + threadIdx.y; i < P.m; i += (int64_t)gridDim.y * 8)
    Wp[i * ldwp + j] = wp_entry(P, i, j);
}

// W' = scale (W Md) for a dense W (FP64, or FP32 widened exactly) and M's
// integers held densely (Md, n x n): CTA tile 32 rows x 64 columns, K steps of
// 16; thread (ty, tx) of 16 x 16 owns rows ty + 16a (a < 2) and columns
// tx + 16b (b < 4).  Every output is one fma chain over the rows r of M in
// ascending order, fma(M[r][j], W[i][r], acc), zero weights included: with W
// finite, an fma with a zero weight returns acc unchanged (acc starts at +0 and
// never becomes -0), so the chain equals the one over the nonzero terms that
// the gathers form; the scale is applied once at the end, as there.
template <typename T>
__global__ void __launch_bounds__(256) apply_dense_kernel(const T* __restrict__ W, int64_t ldw,
                                                          const double* __restrict__ Md, int64_t m, int64_t n,
                                                          double scale, double* __restrict__ Wp, int64_t ldwp) {
  __shared__ double Ws[32][17];
  __shared__ double Ms[16][64];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 64;
  double acc[2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int64_t r0 = 0; r0 < n; r0 += 16) {
    for (int e = threadIdx.x; e < 512; e += 256) {
      const int ii = e >> 4, rr = e & 15;
      const int64_t i = i0 + ii, r = r0 + rr;
      Ws[ii][rr] = (i < m && r < n) ? (double)W[i * ldw + r] : 0.0;
    }
    for (int e = threadIdx.x; e < 1024; e += 256) {
      const int rr = e >> 6, jj = e & 63;
      const int64_t r = r0 + rr, j = j0 + jj;
      Ms[rr][jj] = (r < n && j < n) ? Md[r * n + j] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
      double w[2], mv[4];
#pragma unroll
      for (int a = 0; a < 2; ++a) w[a] = Ws[ty + 16 * a][rr];
#pragma unroll
      for (int b = 0; b < 4; ++b) mv[b] = Ms[rr][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(mv[b], w[a], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
      if (i < m && j < n) Wp[i * ldwp + j] = acc[a][b] * scale;
    }
}

// R[a, c] = w_{I[a], c}; a row index outside [0, m) leaves NaN in its row and
// sets the status word.
__global__ void __launch_bounds__(256) gather_rows_kernel(DevProblem P, const int32_t* __restrict__ I, int32_t k,
                                                          double* __restrict__ R, int32_t* status) {
  const int64_t total = (int64_t)k * P.n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(t / P.n);
    const int64_t c = t - (int64_t)a * P.n;
    const int32_t r = I[a];
    if (r < 0 || r >= P.m) {
      R[t] = __longlong_as_double(0x7ff8000000000000ll);
      if (status != nullptr && c == 0) atomicMax(status, (int)LRA_ERR_INVALID_ARG);
      continue;
    }
    R[t] = w_entry(P, r, c);
  }
}

}  // namespace lra

using namespace lra;

extern "C" {

lra_status lra_multiplier_apply(const lra_problem* prob, lra_multiplier mult, double* Wp, int64_t ldwp,
                                lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  DevProblem P;
  lra_status st = make_dev_problem(prob, mult, &P);
  if (st != LRA_OK) return st;
  if (Wp == nullptr || ldwp < pcols(P) || P.m < 1 || P.n < 1) return LRA_ERR_INVALID_ARG;
  if (mult != nullptr && mult->kind == LRA_MULT_BIDIAG && mult->d_dense != nullptr && P.src == LRA_DENSE &&
      P.mside == 0 &&
      (P.m + 31) / 32 <= 65535 && (P.n + 63) / 64 <= INT32_MAX) {
    // every column of M can be full: the register-tiled product
    const dim3 grid((unsigned)((P.n + 63) / 64), (unsigned)((P.m + 31) / 32));
    LaunchScope ls(stream, "apply_dense_kernel");
    if (P.dtype == LRA_F32)
      apply_dense_kernel<float><<<grid, 256, 0, stream>>>(static_cast<const float*>(P.W), P.ldw, mult->d_dense, P.m,
                                                          P.n, P.mscale, Wp, ldwp);
    else
      apply_dense_kernel<double><<<grid, 256, 0, stream>>>(static_cast<const double*>(P.W), P.ldw, mult->d_dense,
                                                           P.m, P.n, P.mscale, Wp, ldwp);
    return cuda_status(cudaGetLastError());
  }
  const int64_t gx = (pcols(P) + 31) / 32;
  if (gx > INT32_MAX) return LRA_ERR_INVALID_ARG;
  const int64_t gy = std::min<int64_t>((P.m + 7) / 8, 65535);
  {
    LaunchScope ls(stream, "multiplier_apply_kernel");
    multiplier_apply_kernel<<<dim3((unsigned)gx, (unsigned)gy), dim3(32, 8), 0, stream>>>(P, Wp, ldwp);
  }
  return cuda_status(cudaGetLastError());
}

lra_status lra_gather_rows(const lra_problem* prob, const int32_t* I, int32_t k, double* R, int32_t* status_dev,
                           lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  DevProblem P;
  lra_status st = make_dev_problem(prob, nullptr, &P);
  if (st != LRA_OK) return st;
  if (I == nullptr || R == nullptr || k < 1 || P.n < 1) return LRA_ERR_INVALID_ARG;
  DeviceInfo dev;
  if ((st = current_device_info(&dev)) != LRA_OK) return st;
  const int64_t total = (int64_t)k * P.n;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)dev.sms * 8));
  {
    LaunchScope ls(stream, "gather_rows_kernel");
    gather_rows_kernel<<<grid, 256, 0, stream>>>(P, I, k, R, status_dev);
  }
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
