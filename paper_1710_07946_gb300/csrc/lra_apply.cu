// lra_apply.cu -- products with a CUR triple and the sampled a-posteriori
// residual, FP64.
//
// cur_apply:  Y = C (U (R X))   (paper: FMM / HSS stage (iii), multiplication
//   with the low-rank generators).  Stage 1 splits the n-long contraction R X
//   over CTAs (partial k x nrhs sums in the workspace), stage 2 adds the
//   partials in CTA order and applies U, stage 3 forms Y row by row.  All three
//   stages stream their operands once: the product is HBM-bound (about
//   k nrhs / (k + nrhs) flops per byte).
// residual_sample:  E[Q,S] = W[Q,S] - (C U)[Q,:] R[:,S] and its statistics
//   (paper: Section "Superfast a posteriori error estimation for LRA of a matrix
//   filled with i.i.d. values of a single variable").
#include <algorithm>

#include "lra_internal.h"
#include "lra_profile.h"

namespace lra {

constexpr int APPLY_ROWS_PER_CTA = 512;

// Stage 1: partial[b][a][c] = sum over this CTA's rows j of R[a][j] X[j][c].
__global__ void __launch_bounds__(NT) apply_rx_kernel(const double* __restrict__ R, const double* __restrict__ X,
                                                      int64_t n, int k, int nrhs, double* __restrict__ partial) {
  const int64_t j0 = (int64_t)blockIdx.x * APPLY_ROWS_PER_CTA;
  const int64_t j1 = min(n, j0 + APPLY_ROWS_PER_CTA);
  for (int it = threadIdx.x; it < k * nrhs; it += blockDim.x) {
    const int a = it / nrhs, c = it - a * nrhs;
    double s = 0.0;
    for (int64_t j = j0; j < j1; ++j) s = fma(__ldg(R + (int64_t)a * n + j), __ldg(X + j * nrhs + c), s);
    partial[((size_t)blockIdx.x * k + a) * nrhs + c] = s;
  }
}

// Stage 2: T2 = U (sum_b partial[b]).
__global__ void __launch_bounds__(NT) apply_u_kernel(const double* __restrict__ partial, int nb, const double* U,
                                                     int k, int nrhs, double* __restrict__ T1,
                                                     double* __restrict__ T2) {
  for (int it = threadIdx.x; it < k * nrhs; it += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s = s + partial[(size_t)b * k * nrhs + it];
    T1[it] = s;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < k * nrhs; it += blockDim.x) {
    const int a = it / nrhs, c = it - a * nrhs;
    double s = 0.0;
    for (int b = 0; b < k; ++b) s = fma(U[a * k + b], T1[b * nrhs + c], s);
    T2[it] = s;
  }
}

// Stage 3: Y[i][c] = sum_a C[i][a] T2[a][c].
__global__ void __launch_bounds__(NT) apply_c_kernel(const double* __restrict__ C, const double* __restrict__ T2,
                                                     int64_t m, int k, int nrhs, double* __restrict__ Y) {
  const int64_t total = m * nrhs;
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < total; it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = it / nrhs;
    const int c = (int)(it - i * nrhs);
    double s = 0.0;
    for (int a = 0; a < k; ++a) s = fma(__ldg(C + i * k + a), __ldg(T2 + a * nrhs + c), s);
    Y[it] = s;
  }
}

// Residual: rows of C U at the sampled rows, then E and its statistics.
// A sample index outside 0 <= Q[a] < m, 0 <= S[c] < n is never dereferenced:
// the kernels set *bad instead, and the statistics come out NaN.
__global__ void __launch_bounds__(NT) resid_cu_kernel(const double* __restrict__ C, const double* __restrict__ U,
                                                      const int32_t* __restrict__ Q, int q, int k, int64_t m,
                                                      double* __restrict__ CU, int* bad) {
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < (int64_t)q * k;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(it / k), b = (int)(it - (int64_t)a * k);
    const int64_t row = Q[a];
    if (row < 0 || row >= m) {
      atomicOr(bad, 1);
      CU[it] = __longlong_as_double(0x7ff8000000000000ll);
      continue;
    }
    double t = 0.0;
    for (int d = 0; d < k; ++d) t = fma(C[row * k + d], U[d * k + b], t);
    CU[it] = t;
  }
}

__global__ void __launch_bounds__(NT) resid_e_kernel(DevProblem P, const double* __restrict__ CU,
                                                     const double* __restrict__ R, const int32_t* __restrict__ Q,
                                                     const int32_t* __restrict__ S, int q, int s, int k,
                                                     double* __restrict__ E, double* __restrict__ W2, int* bad) {
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < (int64_t)q * s;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(it / s), c = (int)(it - (int64_t)a * s);
    const int64_t col = S[c], row = Q[a];
    if (row < 0 || row >= P.m || col < 0 || col >= P.n) {
      atomicOr(bad, 1);
      E[it] = __longlong_as_double(0x7ff8000000000000ll);
      W2[it] = 0.0;
      continue;
    }
    double t = 0.0;
    for (int b = 0; b < k; ++b) t = fma(CU[(int64_t)a * k + b], R[(int64_t)b * P.n + col], t);
    const double w = w_entry(P, row, col);
    E[it] = w - t;
    W2[it] = w * w;
  }
}

// Fixed-order block sum of per-thread values (deterministic for a fixed blockDim).
__device__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += red[w];
    red[32] = r;
  }
  __syncthreads();
  r = red[32];
  __syncthreads();
  return r;
}

__device__ double block_max(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
    red[32] = r;
  }
  __syncthreads();
  double r = red[32];
  __syncthreads();
  return r;
}

// Sample statistics over K = q s errors in three grid passes: per-CTA partial
// sums (sum e, sum |e|, max |e|, sum e^2, sum w^2), then each CTA folds the
// partial sums into the mean and adds its share of sum (e - mean)^2, then one
// CTA folds the partials in CTA order into the five statistics.
constexpr int RESID_MAX_PARTS = 1024;

__global__ void __launch_bounds__(NT) resid_part_kernel(const double* __restrict__ E, const double* __restrict__ W2,
                                                        int64_t K, double* __restrict__ part) {
  __shared__ double red[33];
  double s = 0.0, sa = 0.0, mx = 0.0, se2 = 0.0, sw2 = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < K; t += (int64_t)gridDim.x * blockDim.x) {
    const double e = E[t];
    s += e;
    sa += fabs(e);
    mx = fmax(mx, fabs(e));
    se2 = fma(e, e, se2);
    sw2 += W2[t];
  }
  s = block_sum(s, red);
  sa = block_sum(sa, red);
  mx = block_max(mx, red);
  se2 = block_sum(se2, red);
  sw2 = block_sum(sw2, red);
  if (threadIdx.x == 0) {
    double* o = part + 6 * (size_t)blockIdx.x;
    o[0] = s; o[1] = sa; o[2] = mx; o[3] = se2; o[4] = sw2;
  }
}

__global__ void __launch_bounds__(NT) resid_var_kernel(const double* __restrict__ E, int64_t K,
                                                       double* __restrict__ part) {
  __shared__ double red[33];
  __shared__ double s_mean;
  const int nparts = gridDim.x;
  if (threadIdx.x < 32) {          // every CTA folds the partial sums in the same order
    double s = 0.0;
    for (int b = threadIdx.x; b < nparts; b += 32) s += part[6 * (size_t)b];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) s_mean = s / (double)K;
  }
  __syncthreads();
  const double mean = s_mean;
  double v = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < K; t += (int64_t)gridDim.x * blockDim.x) {
    const double d = E[t] - mean;
    v = fma(d, d, v);
  }
  v = block_sum(v, red);
  if (threadIdx.x == 0) part[6 * (size_t)blockIdx.x + 5] = v;
}

__global__ void resid_final_kernel(const double* __restrict__ part, int nparts, int64_t K, const int* bad,
                                   double* __restrict__ stats) {
  // one warp: lane l folds the partials l, l + 32, ..., then a butterfly
  const int lane = threadIdx.x;
  double s = 0.0, sa = 0.0, mx = 0.0, se2 = 0.0, sw2 = 0.0, v = 0.0;
  for (int b = lane; b < nparts; b += 32) {
    const double* o = part + 6 * (size_t)b;
    s += o[0]; sa += o[1]; mx = fmax(mx, o[2]); se2 += o[3]; sw2 += o[4]; v += o[5];
  }
  for (int off = 16; off > 0; off >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, off);
    sa += __shfl_xor_sync(0xffffffffu, sa, off);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    se2 += __shfl_xor_sync(0xffffffffu, se2, off);
    sw2 += __shfl_xor_sync(0xffffffffu, sw2, off);
    v += __shfl_xor_sync(0xffffffffu, v, off);
  }
  if (lane == 0) {
    stats[0] = s / (double)K;
    stats[1] = v / (double)K;
    stats[2] = sa / (double)K;
    stats[3] = mx;
    stats[4] = sw2 > 0.0 ? sqrt(se2) / sqrt(sw2) : 0.0;
    if (*bad)
      for (int e = 0; e < 5; ++e) stats[e] = __longlong_as_double(0x7ff8000000000000ll);
  }
}

}  // namespace lra

using namespace lra;

namespace lra {
static size_t apply_ws_bytes(int64_t n, int32_t k, int32_t nrhs) {
  const int64_t nb = (n + APPLY_ROWS_PER_CTA - 1) / APPLY_ROWS_PER_CTA;
  return align_up(sizeof(double) * (size_t)nb * k * nrhs, 256) + 2 * align_up(sizeof(double) * (size_t)k * nrhs, 256);
}
}  // namespace lra

extern "C" {

lra_status lra_cur_apply_workspace_size(int64_t n, int32_t k, int32_t nrhs, size_t* bytes) {
  if (bytes == nullptr || n < 1 || k < 1 || k > KMAX || nrhs < 1 || nrhs > 1024) return LRA_ERR_INVALID_ARG;
  *bytes = apply_ws_bytes(n, k, nrhs);
  return LRA_OK;
}

lra_status lra_cur_apply(const double* C, const double* U, const double* R, int64_t m, int64_t n, int32_t k,
                         const double* X, int32_t nrhs, double* Y, void* workspace, size_t workspace_bytes,
                         lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (!C || !U || !R || !X || !Y || m < 1 || n < 1 || k < 1 || k > KMAX || nrhs < 1 || nrhs > 1024)
    return LRA_ERR_INVALID_ARG;
  const size_t need = apply_ws_bytes(n, k, nrhs);
  if (workspace == nullptr || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return LRA_ERR_WORKSPACE;
  const int nb = (int)((n + APPLY_ROWS_PER_CTA - 1) / APPLY_ROWS_PER_CTA);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  double* partial = reinterpret_cast<double*>(ws);
  double* T1 = reinterpret_cast<double*>(ws + align_up(sizeof(double) * (size_t)nb * k * nrhs, 256));
  double* T2 = T1 + align_up(sizeof(double) * (size_t)k * nrhs, 256) / sizeof(double);
  { LaunchScope ls(stream, "apply_rx_kernel"); apply_rx_kernel<<<nb, NT, 0, stream>>>(R, X, n, k, nrhs, partial); }
  { LaunchScope ls(stream, "apply_u_kernel"); apply_u_kernel<<<1, NT, 0, stream>>>(partial, nb, U, k, nrhs, T1, T2); }
  DeviceInfo dev;
  lra_status st = current_device_info(&dev);
  if (st != LRA_OK) return st;
  const int64_t tot = m * nrhs;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((tot + NT - 1) / NT, (int64_t)dev.sms * 8));
  { LaunchScope ls(stream, "apply_c_kernel"); apply_c_kernel<<<grid, NT, 0, stream>>>(C, T2, m, k, nrhs, Y); }
  return cuda_status(cudaGetLastError());
}

lra_status lra_residual_sample_workspace_size(int32_t k, int32_t q, int32_t s, size_t* bytes) {
  if (bytes == nullptr || k < 1 || k > KMAX || q < 1 || s < 1) return LRA_ERR_INVALID_ARG;
  *bytes = align_up(sizeof(double) * (size_t)q * k, 256) + 2 * align_up(sizeof(double) * (size_t)q * s, 256) +
           align_up(sizeof(double) * 6 * RESID_MAX_PARTS, 256) + 256;
  return LRA_OK;
}

lra_status lra_residual_sample(const lra_problem* prob, const double* C, const double* U, const double* R,
                               int32_t k, const int32_t* Q, int32_t q, const int32_t* S, int32_t s, double* stats,
                               double* E, void* workspace, size_t workspace_bytes, lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  DevProblem P;
  lra_status st = make_dev_problem(prob, nullptr, &P);
  if (st != LRA_OK) return st;
  if (!C || !U || !R || !Q || !S || !stats || k < 1 || k > KMAX || k > std::min(P.m, P.n) || q < 1 || s < 1)
    return LRA_ERR_INVALID_ARG;
  size_t need = 0;
  lra_residual_sample_workspace_size(k, q, s, &need);
  if (workspace == nullptr || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return LRA_ERR_WORKSPACE;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  double* CU = reinterpret_cast<double*>(ws);
  double* Ews = reinterpret_cast<double*>(ws + align_up(sizeof(double) * (size_t)q * k, 256));
  double* W2 = Ews + align_up(sizeof(double) * (size_t)q * s, 256) / sizeof(double);
  double* part = W2 + align_up(sizeof(double) * (size_t)q * s, 256) / sizeof(double);
  int* bad = reinterpret_cast<int*>(part + align_up(sizeof(double) * 6 * RESID_MAX_PARTS, 256) / sizeof(double));
  double* Eout = E ? E : Ews;
  DeviceInfo dev;
  if ((st = current_device_info(&dev)) != LRA_OK) return st;
  LRA_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), stream));
  const int g1 = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)q * k + NT - 1) / NT, dev.sms * 4));
  { LaunchScope ls(stream, "resid_cu_kernel"); resid_cu_kernel<<<g1, NT, 0, stream>>>(C, U, Q, q, k, P.m, CU, bad); }
  const int g2 = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)q * s + NT - 1) / NT, dev.sms * 8));
  { LaunchScope ls(stream, "resid_e_kernel"); resid_e_kernel<<<g2, NT, 0, stream>>>(P, CU, R, Q, S, q, s, k, Eout, W2, bad); }
  const int64_t K = (int64_t)q * s;
  const int g3 = (int)std::max<int64_t>(1, std::min<int64_t>((K + 4 * NT - 1) / (4 * NT),
                                                             std::min<int64_t>(RESID_MAX_PARTS, dev.sms * 4)));
  { LaunchScope ls(stream, "resid_part_kernel"); resid_part_kernel<<<g3, NT, 0, stream>>>(Eout, W2, K, part); }
  { LaunchScope ls(stream, "resid_var_kernel"); resid_var_kernel<<<g3, NT, 0, stream>>>(Eout, K, part); }
  { LaunchScope ls(stream, "resid_final_kernel"); resid_final_kernel<<<1, 32, 0, stream>>>(part, g3, K, bad, stats); }
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
