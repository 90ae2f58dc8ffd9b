// lra_hmatvec.cu -- y = M x for a kernel matrix held as far blocks with C-A
// generators plus a dense near field (the FMM's stage (iii): generators and
// diagonal blocks times subvectors).  Three passes, each deterministic:
//   1. per far block, t_b = U_b (R_b x[cols]);
//   2. per (level, target box), each row's fma chain over the box's blocks in
//      order, C_b[i][:] . t_b, into the level's partial vector; per target
//      leaf, the near field's sums over the source leaves in order;
//   3. y = y_near + y_2 + ... + y_L, in that order.
// Rows outside every group of a level keep the 0 the partial vector starts with.
// Blocks whose generator run ended in an error (info status 1..15) and block or
// group entries outside the matrix contribute nothing.
#include <algorithm>

#include "lra_device.cuh"
#include "lra_internal.h"
#include "lra_profile.h"

namespace lra {

// Generator size of far block b; 0 for a block whose run ended in an error.
__device__ __forceinline__ int hm_kf(const lra_hmatrix& H, int64_t b) {
  const int32_t* inf = H.info + LRA_INFO_LEN * (size_t)b;
  if (inf[3] != LRA_OK && inf[3] < 16) return 0;
  return max(0, min(inf[6], H.kmax));
}

// Pass 1: one CTA per far block (grid-stride): t1 = R_b x[cols], a warp per row
// of R_b (lane-strided fma partial sums, then a fixed butterfly), then t = U_b t1
// with a thread per entry (an ascending fma chain).  MF (matrix-free: the
// batch kept only I, J, U): R_b[a][c] = w(r0 + I_b[a], c0 + c) is evaluated from
// the points as the batch's gathers evaluated it, so the sums are those of the
// stored form, bit for bit.
template <bool MF>
__global__ void __launch_bounds__(256) hm_t_kernel(DevProblem P, lra_hmatrix H, const double* __restrict__ x,
                                                   double* __restrict__ t) {
  __shared__ double t1[KMAX];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = blockIdx.x; b < H.nfar; b += gridDim.x) {
    const int64_t r0 = H.far[4 * (size_t)b], nr = H.far[4 * (size_t)b + 1];
    const int64_t nc = H.far[4 * (size_t)b + 3], c0 = H.far[4 * (size_t)b + 2];
    const int kf = (c0 < 0 || nc < 0 || c0 + nc > H.n || (MF && (r0 < 0 || nr < 1 || r0 + nr > H.n))) ? 0
                                                                                                       : hm_kf(H, b);
    const double* R = MF ? nullptr : H.R + H.far_offsets[2 * (size_t)b + 1];
    const int32_t* Ib = MF ? H.I + (size_t)b * H.kmax : nullptr;
    const double* U = H.U + (size_t)b * H.kmax * H.kmax;
    // a warp per row of R_b: lane-strided partial sums (coalesced), then a fixed butterfly
    for (int a = warp; a < kf; a += nw) {
      double acc = 0.0;
      const int64_t ia = MF ? r0 + min((int64_t)max(Ib[a], 0), nr - 1) : 0;
      for (int64_t c = lane; c < nc; c += 32) {
        const double r = MF ? w_entry(P, ia, c0 + c) : R[(int64_t)a * nc + c];
        acc = fma(r, x[c0 + c], acc);
      }
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (lane == 0) t1[a] = acc;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < kf; a += blockDim.x) {
      double acc = 0.0;
      for (int c = 0; c < kf; ++c) acc = fma(U[a * kf + c], t1[c], acc);
      t[(size_t)b * H.kmax + a] = acc;
    }
    __syncthreads();
  }
}

// Pass 2a: one CTA per (level, target box) group, a thread per row.  MF: C_b[i][a]
// = w(r0 + i, c0 + J_b[a]) from the points (the batch's gathered value).
template <bool MF>
__global__ void __launch_bounds__(256) hm_far_kernel(DevProblem P, lra_hmatrix H, const double* __restrict__ t,
                                                     double* __restrict__ ylev) {
  for (int g = blockIdx.x; g < H.nfar_groups; g += gridDim.x) {
    const int64_t* G = H.far_groups + 5 * (size_t)g;
    const int lev = (int)G[0];
    const int64_t r0 = G[1], nr = G[2], first = G[3], cnt = G[4];
    if (lev < 2 || lev > H.levels || r0 < 0 || nr < 0 || r0 + nr > H.n || first < 0 || cnt < 0 ||
        first + cnt > H.nfar)
      continue;
    double* yl = ylev + (size_t)(lev - 2) * H.n;
    for (int64_t i = threadIdx.x; i < nr; i += blockDim.x) {
      double acc = 0.0;
      for (int64_t b = first; b < first + cnt; ++b) {
        const int64_t br0 = H.far[4 * (size_t)b], bnr = H.far[4 * (size_t)b + 1];
        if (br0 != r0 || bnr != nr) continue;             // a block of another box: not this group's
        const int kf = hm_kf(H, b);
        const double* tb = t + (size_t)b * H.kmax;
        if (MF) {
          const int64_t bc0 = H.far[4 * (size_t)b + 2], bnc = H.far[4 * (size_t)b + 3];
          if (bc0 < 0 || bnc < 1 || bc0 + bnc > H.n) continue;
          const int32_t* Jb = H.J + (size_t)b * H.kmax;
          for (int a = 0; a < kf; ++a)
            acc = fma(w_entry(P, r0 + i, bc0 + min((int64_t)max(Jb[a], 0), bnc - 1)), tb[a], acc);
        } else {
          const double* C = H.C + H.far_offsets[2 * (size_t)b];
          for (int a = 0; a < kf; ++a) acc = fma(C[i * kf + a], tb[a], acc);
        }
      }
      yl[r0 + i] = acc;
    }
  }
}

// Pass 2b: one CTA of 256 threads per target leaf: thread t takes row
// t mod 128 (and every 128th after it) over the first (t < 128) or the second
// half of the leaf's source blocks; entries on the fly as rsqrt(r2) (the FP64
// reciprocal square root, within an ulp of 1/sqrt(r2)), the source points in
// order with two interleaved accumulators; the row's value is (first half's
// acc0 + acc1) + (second half's acc0 + acc1).
__global__ void __launch_bounds__(256) hm_near_kernel(DevProblem P, lra_hmatrix H, const double* __restrict__ x,
                                                      double* __restrict__ ynear) {
  __shared__ double part[128];
  const int half = threadIdx.x >> 7, tr = threadIdx.x & 127;
  for (int g = blockIdx.x; g < H.nnear_groups; g += gridDim.x) {
    const int64_t* G = H.near_groups + 4 * (size_t)g;
    const int64_t r0 = G[0], nr = G[1], first = G[2], cnt = G[3];
    if (r0 < 0 || nr < 0 || r0 + nr > H.n || first < 0 || cnt < 0 || first + cnt > H.nnear) continue;
    const int64_t mid = first + (cnt + 1) / 2;
    const int64_t bl = half == 0 ? first : mid, bh = half == 0 ? mid : first + cnt;
    for (int64_t i0 = 0; i0 < nr; i0 += 128) {
      const int64_t i = i0 + tr;
      double acc0 = 0.0, acc1 = 0.0;
      if (i < nr) {
        const int64_t gi = r0 + i;
        const double xi = P.X[3 * gi], yi = P.X[3 * gi + 1], zi = P.X[3 * gi + 2];
        int par = 0;
        for (int64_t b = bl; b < bh; ++b) {
          const int64_t c0 = H.near[4 * (size_t)b + 2], nc = H.near[4 * (size_t)b + 3];
          if (c0 < 0 || nc < 0 || c0 + nc > H.n) continue;
          for (int64_t j = c0; j < c0 + nc; ++j, par ^= 1) {
            const double dx = xi - P.Y[3 * j], dy = yi - P.Y[3 * j + 1], dz = zi - P.Y[3 * j + 2];
            const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
            const double w = (j == gi) ? 0.0 : rsqrt(r2);
            if (par) acc1 = fma(w, x[j], acc1);
            else acc0 = fma(w, x[j], acc0);
          }
        }
      }
      __syncthreads();
      if (half == 1) part[tr] = acc0 + acc1;
      __syncthreads();
      if (half == 0 && i < nr) ynear[r0 + i] = (acc0 + acc1) + part[tr];
    }
  }
}

// Pass 3: y = y_near + y_2 + ... + y_L.
__global__ void hm_sum_kernel(const double* __restrict__ parts, int nparts, int64_t n, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = parts[i];
    for (int p = 1; p < nparts; ++p) acc = acc + parts[(size_t)p * n + i];
    y[i] = acc;
  }
}

static lra_status hm_check(const lra_hmatrix* H) {
  if (H == nullptr || H->n < 1 || H->levels < 2 || H->kmax < 1 || H->kmax > KMAX || H->nfar < 0 ||
      H->nfar_groups < 0 || H->nnear < 0 || H->nnear_groups < 0)
    return LRA_ERR_INVALID_ARG;
  if (H->nfar > 0 && (!H->far || !H->far_offsets || !H->U || !H->info || !H->far_groups)) return LRA_ERR_INVALID_ARG;
  // stored factors, or matrix-free from the generators' rows and columns
  if (H->nfar > 0 && !((H->C && H->R) || (!H->C && !H->R && H->I && H->J))) return LRA_ERR_INVALID_ARG;
  if (H->nnear > 0 && (!H->near || !H->near_groups)) return LRA_ERR_INVALID_ARG;
  return LRA_OK;
}

static size_t hm_bytes(const lra_hmatrix* H) {
  return align_up(sizeof(double) * (size_t)std::max(H->nfar, 1) * H->kmax, 256) +
         align_up(sizeof(double) * (size_t)H->levels * H->n, 256);
}

}  // namespace lra

using namespace lra;

extern "C" {

lra_status lra_hmatvec_workspace_size(const lra_hmatrix* H, size_t* bytes) {
  if (bytes == nullptr) return LRA_ERR_INVALID_ARG;
  lra_status st = hm_check(H);
  if (st != LRA_OK) return st;
  *bytes = hm_bytes(H);
  return LRA_OK;
}

lra_status lra_hmatvec(const lra_problem* prob, const lra_hmatrix* H, const double* x, double* y, void* workspace,
                       size_t workspace_bytes, lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  DevProblem P;
  lra_status st = make_dev_problem(prob, nullptr, &P);
  if (st != LRA_OK) return st;
  if ((st = hm_check(H)) != LRA_OK) return st;
  if (P.src != LRA_KERNEL_LAPLACE || P.m != H->n || P.n != H->n || x == nullptr || y == nullptr)
    return LRA_ERR_INVALID_ARG;
  const size_t need = hm_bytes(H);
  if (workspace == nullptr || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return LRA_ERR_WORKSPACE;
  DeviceInfo dev;
  if ((st = current_device_info(&dev)) != LRA_OK) return st;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  double* t = reinterpret_cast<double*>(ws);
  double* parts = reinterpret_cast<double*>(ws + align_up(sizeof(double) * (size_t)std::max(H->nfar, 1) * H->kmax,
                                                          256));
  // parts[0] = y_near, parts[1 + lev - 2] = y_lev
  LRA_CUDA_TRY(cudaMemsetAsync(parts, 0, sizeof(double) * (size_t)H->levels * H->n, stream));
  const lra_hmatrix Hv = *H;
  const int cap = dev.sms * 8;
  if (H->nfar > 0) {
    const bool mf = H->C == nullptr;
    {
      LaunchScope ls(stream, "hm_t_kernel");
      if (mf) hm_t_kernel<true><<<std::min(H->nfar, cap), 256, 0, stream>>>(P, Hv, x, t);
      else hm_t_kernel<false><<<std::min(H->nfar, cap), 256, 0, stream>>>(P, Hv, x, t);
    }
    {
      LaunchScope ls(stream, "hm_far_kernel");
      const int grid = std::max(1, std::min(H->nfar_groups, cap));
      if (mf) hm_far_kernel<true><<<grid, 256, 0, stream>>>(P, Hv, t, parts + H->n);
      else hm_far_kernel<false><<<grid, 256, 0, stream>>>(P, Hv, t, parts + H->n);
    }
  }
  if (H->nnear_groups > 0) {
    LaunchScope ls(stream, "hm_near_kernel");
    hm_near_kernel<<<std::min(H->nnear_groups, dev.sms * 8), 256, 0, stream>>>(P, Hv, x, parts);
  }
  {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((H->n + 255) / 256, cap));
    LaunchScope ls(stream, "hm_sum_kernel");
    hm_sum_kernel<<<grid, 256, 0, stream>>>(parts, H->levels, H->n, y);
  }
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
