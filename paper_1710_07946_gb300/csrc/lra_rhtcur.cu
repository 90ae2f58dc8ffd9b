// lra_rhtcur.cu -- CUR LRA with Gaussian sampling (paper: Algorithm algrhtcur),
// with lbar = l = k:
//   1. the sketch S = W Hbar (m x k) for the caller's n x k Gaussian Hbar,
//      written transposed (k x m), one ascending fma chain per entry;
//   2. rows I: a one-loop C-A run on S^T from all k rows -- its cold first
//      column step is the maxvol (LU with column pivoting, then dominance swaps)
//      on S^T, i.e. the GE96-style selection of k rows of S;
//   3. columns J: a one-loop C-A run on the row strip W[I, :] from all k rows
//      -- its cold column step picks J, its row step orders the rows, and its
//      nucleus is the CUR's U = pinv of the rank-r truncation of W[I, J];
//   4. C = W[:, J], R = W[I, :].
// Steps 2 and 3 are lra_ca_run calls on the two small dense problems, so their
// arithmetic is the C-A path's, operation for operation.
#include <algorithm>
#include <cstring>

#include "lra_device.cuh"
#include "lra_internal.h"
#include "lra_profile.h"

namespace lra {

// S^T = (W Hbar)^T: CTA tile 32 rows of W x 16 KB sketch columns (KB =
// ceil(k / 16)), 16-deep steps over the columns j of W; thread (ty, tx) of
// 16 x 16 owns rows ty + 16a (a < 2) and sketch columns tx + 16b (b < KB).
// S[i][c] = sum over j ascending of fma(Hbar[j][c], w_ij, .); the zero padding
// past n adds exact zeros.
template <int KB>
__global__ void __launch_bounds__(256) sketch_kernel(DevProblem P, const double* __restrict__ Hbar, int k,
                                                     double* __restrict__ ST) {
  __shared__ double Ws[32][17];
  __shared__ double Hs[16][16 * KB];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  double acc[2][KB];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < KB; ++b) acc[a][b] = 0.0;
  for (int64_t j0 = 0; j0 < P.n; j0 += 16) {
    for (int e = threadIdx.x; e < 512; e += 256) {
      const int ii = e >> 4, jj = e & 15;
      const int64_t i = i0 + ii, j = j0 + jj;
      Ws[ii][jj] = (i < P.m && j < P.n) ? w_entry(P, i, j) : 0.0;
    }
    for (int e = threadIdx.x; e < 256 * KB; e += 256) {
      const int jj = e / (16 * KB), c = e - jj * (16 * KB);
      const int64_t j = j0 + jj;
      Hs[jj][c] = (j < P.n && c < k) ? Hbar[j * k + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
      double w[2], hv[KB];
#pragma unroll
      for (int a = 0; a < 2; ++a) w[a] = Ws[ty + 16 * a][rr];
#pragma unroll
      for (int b = 0; b < KB; ++b) hv[b] = Hs[rr][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < KB; ++b) acc[a][b] = fma(hv[b], w[a], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < KB; ++b) {
      const int64_t i = i0 + ty + 16 * a;
      const int c = tx + 16 * b;
      if (i < P.m && c < k) ST[(int64_t)c * P.m + i] = acc[a][b];
    }
}

__global__ void iota_kernel(int32_t* v, int k) {
  for (int a = threadIdx.x; a < k; a += blockDim.x) v[a] = a;
}

// Rows (dir 0: R[a][c] = w_{idx[a], c}, k x n) or columns (dir 1: C[i][a] =
// w_{i, idx[a]}, m x k) of W; an index out of range leaves NaN and sets *status.
__global__ void __launch_bounds__(256) rht_gather_kernel(DevProblem P, const int32_t* __restrict__ idx, int k,
                                                         int dir, double* __restrict__ out, int32_t* status) {
  const int64_t len = dir == 0 ? P.n : P.m;
  const int64_t lim = dir == 0 ? P.m : P.n;
  const int64_t total = (int64_t)k * len;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int a;
    int64_t c;
    if (dir == 0) { a = (int)(t / len); c = t - (int64_t)a * len; }
    else { c = t / k; a = (int)(t - c * k); }
    const int32_t r = idx[a];
    if (r < 0 || r >= lim) {
      out[t] = __longlong_as_double(0x7ff8000000000000ll);
      atomicMax(status, (int)LRA_ERR_INVALID_ARG);
      continue;
    }
    out[t] = dir == 0 ? w_entry(P, r, c) : w_entry(P, c, r);
  }
}

// I = J1[I2]; info from the two runs: rank of the second, swaps summed, loops
// 2, the worst status (an error of either run first), FP64 steps summed, k, k
// (after an error of the first run: rank 0, its swaps, loops 1).
__global__ void rht_finish_kernel(const int32_t* __restrict__ J1, const int32_t* __restrict__ I2, int k,
                                  const int32_t* __restrict__ info1, const int32_t* __restrict__ info2,
                                  const int32_t* __restrict__ gstatus, int32_t* __restrict__ I,
                                  int32_t* __restrict__ info) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    const int32_t t = I2[a];
    if (t < 0 || t >= k) { bad = 1; I[a] = -1; }
    else I[a] = J1[t];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int s1 = info1[3], s2 = info2[3];
    int st;
    if (s1 != LRA_OK && s1 < 16) st = s1;
    else if (s2 != LRA_OK && s2 < 16) st = s2;
    else if (*gstatus != 0 || bad) st = LRA_ERR_INVALID_ARG;
    else st = max(s1, s2);
    const bool first_failed = s1 != LRA_OK && s1 < 16;     // the second run's results are then void
    info[0] = first_failed ? 0 : info2[0];
    info[1] = first_failed ? info1[1] : info1[1] + info2[1];
    info[2] = first_failed ? 1 : 2;
    info[3] = st;
    info[4] = 0;
    info[5] = info1[5] + info2[5];
    info[6] = k;
    info[7] = k;
  }
}

struct RhtLayout {
  size_t off_ST, off_R0, off_iota, off_I1, off_J1, off_C1, off_U1, off_R1, off_lv1, off_info1, off_I2, off_C2, off_lv2,
      off_info2, off_status, off_ws, ws_bytes, bytes;
};

static lra_status rht_layout(const DevProblem& P, const lra_problem* prob, const lra_ca_params* par, RhtLayout* L,
                             lra_problem* ps, lra_problem* pr, lra_ca_params* p1) {
  const int k = par->k;
  size_t o = 256;
  auto take = [&o](size_t bytes) { const size_t at = o; o = align_up(o + bytes, 256); return at; };
  L->off_ST = take(sizeof(double) * (size_t)k * P.m);
  L->off_R0 = take(sizeof(double) * (size_t)k * P.n);
  L->off_iota = take(sizeof(int32_t) * k);
  L->off_I1 = take(sizeof(int32_t) * k);
  L->off_J1 = take(sizeof(int32_t) * k);
  L->off_C1 = take(sizeof(double) * (size_t)k * k);
  L->off_U1 = take(sizeof(double) * (size_t)k * k);
  L->off_R1 = take(sizeof(double) * (size_t)k * P.m);
  L->off_lv1 = take(sizeof(double) * 2);
  L->off_info1 = take(sizeof(int32_t) * LRA_INFO_LEN);
  L->off_I2 = take(sizeof(int32_t) * k);
  L->off_C2 = take(sizeof(double) * (size_t)k * k);
  L->off_lv2 = take(sizeof(double) * 2);
  L->off_info2 = take(sizeof(int32_t) * LRA_INFO_LEN);
  L->off_status = take(sizeof(int32_t));
  *p1 = *par;
  p1->sweeps = 1;
  p1->mode = LRA_MODE_FP64;
  p1->nstages = 0;
  std::memset(ps, 0, sizeof(*ps));
  ps->src = LRA_DENSE;
  ps->dtype = LRA_F64;
  ps->m = k;
  ps->n = P.m;
  ps->ldw = P.m;
  ps->W = reinterpret_cast<const void*>(uintptr_t(256));   // placeholder: sizes only
  *pr = *ps;
  pr->n = P.n;
  pr->ldw = P.n;
  size_t w1 = 0, w2 = 0;
  lra_status st = lra_ca_workspace_size(ps, p1, nullptr, &w1);
  if (st != LRA_OK) return st;
  if ((st = lra_ca_workspace_size(pr, p1, nullptr, &w2)) != LRA_OK) return st;
  L->ws_bytes = align_up(std::max(w1, w2), 256);
  L->off_ws = take(L->ws_bytes);
  L->bytes = o;
  (void)prob;
  return LRA_OK;
}

static lra_status rht_check(const lra_problem* prob, const lra_ca_params* par, DevProblem* P) {
  lra_status st = make_dev_problem(prob, nullptr, P);
  if (st != LRA_OK) return st;
  if (par == nullptr || par->k < 1 || par->k > KMAX || par->k > std::min(P->m, P->n)) return LRA_ERR_INVALID_ARG;
  if (!(par->h >= 1.0) || !(par->h < 1e300) || !(par->rank_tol >= 0.0) || !(par->rank_tol < 1.0) ||
      par->max_swaps < 0 || par->nstages != 0)
    return LRA_ERR_INVALID_ARG;
  return LRA_OK;
}

}  // namespace lra

using namespace lra;

extern "C" {

lra_status lra_rhtcur_workspace_size(const lra_problem* prob, const lra_ca_params* par, size_t* bytes) {
  if (bytes == nullptr) return LRA_ERR_INVALID_ARG;
  DevProblem P;
  lra_status st = rht_check(prob, par, &P);
  if (st != LRA_OK) return st;
  RhtLayout L;
  lra_problem ps, pr;
  lra_ca_params p1;
  if ((st = rht_layout(P, prob, par, &L, &ps, &pr, &p1)) != LRA_OK) return st;
  *bytes = L.bytes;
  return LRA_OK;
}

lra_status lra_rhtcur_run(const lra_problem* prob, const double* Hbar, const lra_ca_params* par, const lra_cur* out,
                          void* workspace, size_t workspace_bytes, lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  DevProblem P;
  lra_status st = rht_check(prob, par, &P);
  if (st != LRA_OK) return st;
  if (Hbar == nullptr || out == nullptr || !out->I || !out->J || !out->C || !out->U || !out->R || !out->logvol ||
      !out->info)
    return LRA_ERR_INVALID_ARG;
  RhtLayout L;
  lra_problem ps, pr;
  lra_ca_params p1;
  if ((st = rht_layout(P, prob, par, &L, &ps, &pr, &p1)) != LRA_OK) return st;
  if (workspace == nullptr || workspace_bytes < L.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return LRA_ERR_WORKSPACE;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  const int k = par->k;
  double* ST = reinterpret_cast<double*>(ws + L.off_ST);
  double* R0 = reinterpret_cast<double*>(ws + L.off_R0);
  int32_t* iota = reinterpret_cast<int32_t*>(ws + L.off_iota);
  int32_t* gstatus = reinterpret_cast<int32_t*>(ws + L.off_status);
  ps.W = ST;
  pr.W = R0;
  DeviceInfo dev;
  if ((st = current_device_info(&dev)) != LRA_OK) return st;
  LRA_CUDA_TRY(cudaMemsetAsync(gstatus, 0, sizeof(int32_t), stream));
  {
    LaunchScope ls(stream, "sketch_kernel");
    const unsigned grid = (unsigned)((P.m + 31) / 32);
    switch ((k + 15) / 16) {
      case 1: sketch_kernel<1><<<grid, 256, 0, stream>>>(P, Hbar, k, ST); break;
      case 2: sketch_kernel<2><<<grid, 256, 0, stream>>>(P, Hbar, k, ST); break;
      case 3: sketch_kernel<3><<<grid, 256, 0, stream>>>(P, Hbar, k, ST); break;
      default: sketch_kernel<4><<<grid, 256, 0, stream>>>(P, Hbar, k, ST); break;
    }
  }
  {
    LaunchScope ls(stream, "iota_kernel");
    iota_kernel<<<1, 64, 0, stream>>>(iota, k);
  }
  LRA_CUDA_TRY(cudaGetLastError());
  // step 2: rows of S from the cold column step of a one-loop C-A run on S^T
  lra_cur c1;
  c1.I = reinterpret_cast<int32_t*>(ws + L.off_I1);
  c1.J = reinterpret_cast<int32_t*>(ws + L.off_J1);
  c1.C = reinterpret_cast<double*>(ws + L.off_C1);
  c1.U = reinterpret_cast<double*>(ws + L.off_U1);
  c1.R = reinterpret_cast<double*>(ws + L.off_R1);
  c1.logvol = reinterpret_cast<double*>(ws + L.off_lv1);
  c1.info = reinterpret_cast<int32_t*>(ws + L.off_info1);
  if ((st = lra_ca_run(&ps, &p1, nullptr, iota, &c1, ws + L.off_ws, L.ws_bytes, stream_)) != LRA_OK) return st;
  // step 3: the row strip W[I, :] and a one-loop C-A run on it
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)k * std::max(P.m, P.n) + 255) / 256,
                                                           (int64_t)dev.sms * 8));
  {
    LaunchScope ls(stream, "rht_gather_kernel");
    rht_gather_kernel<<<g, 256, 0, stream>>>(P, c1.J, k, 0, R0, gstatus);
  }
  LRA_CUDA_TRY(cudaGetLastError());
  lra_cur c2;
  c2.I = reinterpret_cast<int32_t*>(ws + L.off_I2);
  c2.J = out->J;
  c2.C = reinterpret_cast<double*>(ws + L.off_C2);
  c2.U = out->U;
  c2.R = out->R;
  c2.logvol = out->logvol;
  c2.info = reinterpret_cast<int32_t*>(ws + L.off_info2);
  if ((st = lra_ca_run(&pr, &p1, nullptr, iota, &c2, ws + L.off_ws, L.ws_bytes, stream_)) != LRA_OK) return st;
  // step 4: C = W[:, J]; I = J1[I2]; info
  {
    LaunchScope ls(stream, "rht_gather_kernel");
    rht_gather_kernel<<<g, 256, 0, stream>>>(P, out->J, k, 1, out->C, gstatus);
  }
  {
    LaunchScope ls(stream, "rht_finish_kernel");
    rht_finish_kernel<<<1, 64, 0, stream>>>(c1.J, c2.I, k, c1.info, c2.info, gstatus, out->I, out->info);
  }
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
