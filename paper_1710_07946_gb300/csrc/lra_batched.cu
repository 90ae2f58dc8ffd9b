// lra_batched.cu -- many independent C-A CUR approximations (the generators of
// the neutered block columns of an HSS / FMM matrix) in one persistent launch.
//
// Each CTA takes blocks from a device work queue (one atomic counter; the
// caller's processing order, largest blocks first for a balanced tail) and
// runs the whole C-A loop of a block, then its nucleus, on its own: the block's
// strips sit in the CTA's shared memory when they fit, otherwise in the CTA's
// slice of a global scratch area.  The per-block arithmetic is the single-CTA
// path of lra_ca_run, operation for operation.  A second kernel draws the
// a-posteriori residual sample of every block.
#include <algorithm>
#include <cstring>

#include "lra_ca_loop.cuh"
#include "lra_internal.h"
#include "lra_nucleus.cuh"
#include "lra_profile.h"

namespace lra {

struct BatchArgs {
  DevProblem base;
  const int64_t* blocks;    // nb x 4: row0, nrows, col0, ncols
  const int64_t* offs;      // nb x 2: offsets (in doubles) of C_b and R_b
  const int32_t* order;     // processing order (nb) or null
  int32_t nb, kmax, sweeps, max_swaps;
  double h, rank_tol;
  const int32_t* I0;        // nb x kmax initial rows (block-local)
  int32_t* I;               // nb x kmax
  int32_t* J;               // nb x kmax
  double* C;                // packed
  double* R;                // packed
  double* U;                // nb x kmax x kmax (k_b x k_b at the start of each slot)
  double* logvol;           // nb x 2 sweeps
  int32_t* info;            // nb x LRA_INFO_LEN
  unsigned int* counter;    // work queue head
  double* scratch;          // per CTA: G (kmax^2) then, if needed, a strip (kmax x max_len)
  size_t scratch_stride;    // doubles per CTA
  int32_t cap_ldm;          // largest strip length kept in shared memory
  int64_t max_len;          // largest block dimension the scratch was sized for
  int32_t mixed;
  int32_t nstages, margin;  // staged generator sizes (0: one run of size k_b)
  int32_t stages[LRA_MAX_STAGES];
};

template <bool MIXED>
__global__ void __launch_bounds__(NT) ca_batched_kernel(BatchArgs B) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_b;
  __shared__ int32_t s_I0[KMAX];
  double* G = B.scratch + (size_t)blockIdx.x * B.scratch_stride;
  double* gstrip = G + (size_t)B.kmax * B.kmax;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned int q = atomicAdd(B.counter, 1u);
      s_b = (q < (unsigned)B.nb) ? (B.order ? B.order[q] : (int)q) : -1;
    }
    __syncthreads();
    const int b = s_b;
    __syncthreads();
    if (b < 0) break;
    int32_t* info = B.info + LRA_INFO_LEN * (size_t)b;
    const int64_t r0 = B.blocks[4 * (size_t)b], nr = B.blocks[4 * (size_t)b + 1];
    const int64_t c0 = B.blocks[4 * (size_t)b + 2], nc = B.blocks[4 * (size_t)b + 3];
    if (r0 < 0 || c0 < 0 || nr < 1 || nc < 1 || r0 + nr > B.base.m || c0 + nc > B.base.n || nr > B.max_len ||
        nc > B.max_len) {
      for (int e = threadIdx.x; e < LRA_INFO_LEN; e += blockDim.x) info[e] = (e == 3) ? LRA_ERR_INVALID_ARG : 0;
      continue;
    }
    CaArgs A;
    A.P = B.base;
    A.P.m = nr;
    A.P.n = nc;
    if (A.P.src == LRA_DENSE) {
      const size_t esz = (A.P.dtype == LRA_F32) ? 4 : 8;
      A.P.W = static_cast<const unsigned char*>(B.base.W) + (size_t)(r0 * B.base.ldw + c0) * esz;
    } else {
      A.P.X = B.base.X + 3 * r0;
      A.P.Y = B.base.Y + 3 * c0;
    }
    const int kb = (int)min((int64_t)B.kmax, min(nr, nc));
    A.sweeps = B.sweeps;
    A.max_swaps = B.max_swaps;
    A.h = B.h;
    A.I0 = B.I0 + (size_t)b * B.kmax;
    A.I = B.I + (size_t)b * B.kmax;
    A.J = B.J + (size_t)b * B.kmax;
    A.C = B.C + B.offs[2 * (size_t)b];
    A.R = B.R + B.offs[2 * (size_t)b + 1];
    A.logvol = B.logvol + (size_t)b * 2 * B.sweeps;
    A.info = info;
    A.G = G;
    A.chunk_n = (int)nc;
    A.chunk_m = (int)nr;
    A.ldm = (int)max(nr, nc);
    A.strip_in_smem = A.ldm <= B.cap_ldm;
    A.mixed = B.mixed;
    if (B.mixed && A.P.src == LRA_KERNEL_LAPLACE) {
      A.P.X32 = B.base.X32 + 3 * r0;
      A.P.Y32 = B.base.Y32 + 3 * c0;
    }
    A.gstrip = A.strip_in_smem ? nullptr : gstrip;
    // Generator sizes: the caller's stages clipped to kb (one run of size kb
    // without stages).  Each stage is a complete C-A run and nucleus; the next
    // stage starts from this stage's rows, then the block's unused initial rows.
    const int32_t* I0b = B.I0 + (size_t)b * B.kmax;
    int stage = 0, k = B.nstages > 0 ? min(B.stages[0], kb) : kb;
    int swaps = 0, loops = 0, n32 = 0, n64 = 0, nrun = 0, r = 0, st = LRA_OK;
    for (;;) {
      A.k = k;
      A.I0 = (nrun == 0) ? I0b : s_I0;
      const CaSmem S = ca_smem_carve(smem, k, A.ldm, A.strip_in_smem ? nullptr : gstrip);
      ca_loop<SoloGroup, MIXED>(SoloGroup{}, A, S);
      __syncthreads();
      ++nrun;
      st = info[3];
      swaps += info[1]; loops += info[2]; n32 += info[4]; n64 += info[5];
      if (st != LRA_OK && st < 16) break;
      r = nucleus_cta(G, k, B.rank_tol, B.U + (size_t)b * B.kmax * B.kmax, smem);
      if (r < k && st == LRA_OK) st = LRA_WARN_RANK_DEFICIENT;
      if (k >= kb || r < k - B.margin) break;
      int kn = k;
      while (stage + 1 < B.nstages && kn <= k) kn = min(B.stages[++stage], kb);
      if (kn <= k) break;
      if (threadIdx.x == 0) {           // next initial rows: I, then unused I0b rows in order
        for (int a = 0; a < k; ++a) s_I0[a] = A.I[a];
        int c = k;
        for (int t = 0; t < kb && c < kn; ++t) {
          const int32_t v = I0b[t];
          bool in = false;
          for (int a = 0; a < k; ++a) in |= (s_I0[a] == v);
          if (!in) s_I0[c++] = v;
        }
      }
      __syncthreads();
      k = kn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      info[0] = (st != LRA_OK && st < 16) ? 0 : r;
      info[1] = swaps; info[2] = loops; info[3] = st;
      info[4] = n32; info[5] = n64; info[6] = k; info[7] = nrun;
    }
    __syncthreads();
  }
}

// Residual sample of every block: E_b[Q_b, S_b] = W_b[Q_b, S_b] - (C_b U_b)[Q_b, :] R_b[:, S_b]
// and its statistics (mean, variance, mean |e|, max |e|, Frobenius ratio).
__global__ void __launch_bounds__(256) resid_batched_kernel(DevProblem base, const int64_t* blocks,
                                                            const int64_t* offs, int32_t nb, int32_t kmax,
                                                            const double* C, const double* U, const double* R,
                                                            const int32_t* info, const int32_t* Qs, int32_t q,
                                                            const int32_t* Ss, int32_t s, double* stats) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* CU = reinterpret_cast<double*>(smem);                  // q x k
  double* E = CU + (size_t)q * kmax;                              // q x s
  double* W2 = E + (size_t)q * s;                                 // q x s
  __shared__ double red[33];
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    double* st = stats + 5 * (size_t)b;
    const int status = info[LRA_INFO_LEN * (size_t)b + 3];
    const int64_t r0 = blocks[4 * (size_t)b], nr = blocks[4 * (size_t)b + 1];
    const int64_t c0 = blocks[4 * (size_t)b + 2], nc = blocks[4 * (size_t)b + 3];
    if (status != LRA_OK && status < 16) {
      if (threadIdx.x < 5) st[threadIdx.x] = __longlong_as_double(0x7ff8000000000000ll);
      continue;
    }
    const int kf = info[LRA_INFO_LEN * (size_t)b + 6];
    const int k = (kf > 0) ? kf : (int)min((int64_t)kmax, min(nr, nc));
    const double* Cb = C + offs[2 * (size_t)b];
    const double* Rb = R + offs[2 * (size_t)b + 1];
    const double* Ub = U + (size_t)b * kmax * kmax;
    const int32_t* Q = Qs + (size_t)b * q;
    const int32_t* S = Ss + (size_t)b * s;
    DevProblem P = base;
    P.m = nr;
    P.n = nc;
    if (P.src == LRA_DENSE) {
      const size_t esz = (P.dtype == LRA_F32) ? 4 : 8;
      P.W = static_cast<const unsigned char*>(base.W) + (size_t)(r0 * base.ldw + c0) * esz;
    } else {
      P.X = base.X + 3 * r0;
      P.Y = base.Y + 3 * c0;
    }
    for (int it = threadIdx.x; it < q * k; it += blockDim.x) {
      const int a = it / k, bb = it - a * k;
      const int64_t row = min((int64_t)Q[a], nr - 1);
      double t = 0.0;
      for (int d = 0; d < k; ++d) t = fma(Cb[row * k + d], Ub[d * k + bb], t);
      CU[it] = t;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < q * s; it += blockDim.x) {
      const int a = it / s, c = it - a * s;
      const int64_t col = min((int64_t)S[c], nc - 1);
      double t = 0.0;
      for (int bb = 0; bb < k; ++bb) t = fma(CU[a * k + bb], Rb[(int64_t)bb * nc + col], t);
      const double w = w_entry(P, min((int64_t)Q[a], nr - 1), col);
      E[it] = w - t;
      W2[it] = w * w;
    }
    __syncthreads();
    double sm = 0.0, sa = 0.0, mx = 0.0, se2 = 0.0, sw2 = 0.0;
    for (int it = threadIdx.x; it < q * s; it += blockDim.x) {
      const double e = E[it];
      sm += e; sa += fabs(e); mx = fmax(mx, fabs(e)); se2 = fma(e, e, se2); sw2 += W2[it];
    }
    auto bsum = [&](double v) {
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += red[w];
        red[32] = r;
      }
      __syncthreads();
      const double r = red[32];
      __syncthreads();
      return r;
    };
    auto bmax = [&](double v) {
      for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
        red[32] = r;
      }
      __syncthreads();
      const double r = red[32];
      __syncthreads();
      return r;
    };
    sm = bsum(sm); sa = bsum(sa); mx = bmax(mx); se2 = bsum(se2); sw2 = bsum(sw2);
    const double K = (double)q * (double)s;
    const double mean = sm / K;
    double v = 0.0;
    for (int it = threadIdx.x; it < q * s; it += blockDim.x) {
      const double d = E[it] - mean;
      v = fma(d, d, v);
    }
    v = bsum(v);
    if (threadIdx.x == 0) {
      st[0] = mean; st[1] = v / K; st[2] = sa / K; st[3] = mx;
      st[4] = sw2 > 0.0 ? sqrt(se2) / sqrt(sw2) : 0.0;
    }
    __syncthreads();
  }
}

struct BatchPlan {
  int grid;
  int cap_ldm;
  size_t smem;
  size_t scratch_stride;
  size_t off_pts;
  size_t bytes;
};

static size_t ca_need(int k, int ldm, bool strip) {
  return ca_smem_fixed(k, ldm) + (strip ? sizeof(double) * (size_t)k * ldm : 0);
}

static lra_status batch_plan(const DevProblem& P, const lra_ca_params* par, int64_t max_len, BatchPlan* pl) {
  const int32_t kmax = par->k;
  DeviceInfo dev;
  lra_status st = current_device_info(&dev);
  if (st != LRA_OK) return st;
  const size_t budget = dev.smem_optin - 4096;
  int cap = 0;
  {
    int lo = 0, hi = (int)std::min<int64_t>(max_len, 1 << 20);
    while (lo < hi) {                       // largest ldm whose strip fits in shared memory
      const int mid = (lo + hi + 1) / 2;
      if (ca_need(kmax, mid, true) <= budget) lo = mid; else hi = mid - 1;
    }
    cap = lo;
  }
  size_t smem = std::max(ca_need(kmax, cap, true), nucleus_smem_bytes(kmax));
  if (max_len > cap) smem = std::max(smem, ca_need(kmax, (int)max_len, false));
  if (smem > budget) return LRA_ERR_INVALID_ARG;
  const bool mixed = par->mode == LRA_MODE_MIXED && mixed_supported(P);
  auto kern = mixed ? ca_batched_kernel<true> : ca_batched_kernel<false>;
  LRA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  LRA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem));
  if (occ < 1) return LRA_ERR_INVALID_ARG;
  pl->grid = occ * dev.sms;
  pl->cap_ldm = cap;
  pl->smem = smem;
  pl->scratch_stride = (size_t)kmax * kmax + (max_len > cap ? (size_t)kmax * max_len : 0);
  pl->scratch_stride = align_up(pl->scratch_stride, 32);
  pl->off_pts = align_up(256 + sizeof(double) * pl->scratch_stride * pl->grid, 256);
  pl->bytes = pl->off_pts;
  if (mixed && P.src == LRA_KERNEL_LAPLACE)
    pl->bytes = align_up(pl->off_pts + sizeof(float) * 3 * (size_t)(P.m + P.n), 256);
  return LRA_OK;
}

}  // namespace lra

using namespace lra;

extern "C" {

lra_status lra_ca_batched_workspace_size(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                                         size_t* bytes) {
  if (bytes == nullptr || batch == nullptr || par == nullptr) return LRA_ERR_INVALID_ARG;
  DevProblem P;
  lra_status st = make_dev_problem(base, nullptr, &P);
  if (st != LRA_OK) return st;
  if (par->k < 1 || par->k > KMAX || batch->nb < 1 || batch->max_len < 1) return LRA_ERR_INVALID_ARG;
  BatchPlan pl;
  if ((st = batch_plan(P, par, batch->max_len, &pl)) != LRA_OK) return st;
  *bytes = pl.bytes;
  return LRA_OK;
}

lra_status lra_ca_run_batched(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                              const int32_t* I0, const lra_cur_batch* out, void* workspace, size_t workspace_bytes,
                              lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  DevProblem P;
  lra_status st = make_dev_problem(base, nullptr, &P);
  if (st != LRA_OK) return st;
  if (batch == nullptr || par == nullptr || out == nullptr || I0 == nullptr) return LRA_ERR_INVALID_ARG;
  if (batch->blocks == nullptr || batch->offsets == nullptr || batch->nb < 1 || batch->max_len < 1)
    return LRA_ERR_INVALID_ARG;
  if (par->k < 1 || par->k > KMAX || par->sweeps < 1 || par->max_swaps < 0 || !(par->h >= 1.0) ||
      !(par->h < 1e300) || !(par->rank_tol >= 0.0) || !(par->rank_tol < 1.0) ||
      (par->mode != LRA_MODE_FP64 && par->mode != LRA_MODE_MIXED) || !stages_valid(par))
    return LRA_ERR_INVALID_ARG;
  if (!out->I || !out->J || !out->C || !out->U || !out->R || !out->logvol || !out->info) return LRA_ERR_INVALID_ARG;
  BatchPlan pl;
  if ((st = batch_plan(P, par, batch->max_len, &pl)) != LRA_OK) return st;
  if (workspace == nullptr || workspace_bytes < pl.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return LRA_ERR_WORKSPACE;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  BatchArgs A;
  std::memset(&A, 0, sizeof(A));
  A.base = P;
  A.blocks = batch->blocks;
  A.offs = batch->offsets;
  A.order = batch->order;
  A.nb = batch->nb;
  A.kmax = par->k;
  A.sweeps = par->sweeps;
  A.max_swaps = par->max_swaps;
  A.h = par->h;
  A.rank_tol = par->rank_tol;
  A.I0 = I0;
  A.I = out->I;
  A.J = out->J;
  A.C = out->C;
  A.R = out->R;
  A.U = out->U;
  A.logvol = out->logvol;
  A.info = out->info;
  A.counter = reinterpret_cast<unsigned int*>(ws);
  A.scratch = reinterpret_cast<double*>(ws + 256);
  A.scratch_stride = pl.scratch_stride;
  A.cap_ldm = pl.cap_ldm;
  A.max_len = batch->max_len;
  A.mixed = (par->mode == LRA_MODE_MIXED && mixed_supported(P)) ? 1 : 0;
  A.nstages = par->nstages;
  A.margin = par->rank_margin;
  for (int s = 0; s < par->nstages; ++s) A.stages[s] = par->k_stages[s];
  if (A.mixed && P.src == LRA_KERNEL_LAPLACE) {
    float* X32 = reinterpret_cast<float*>(ws + pl.off_pts);
    A.base.X32 = X32;
    A.base.Y32 = X32 + 3 * P.m;
    if ((st = points_to_f32(P.X, P.m, X32, stream)) != LRA_OK) return st;
    if ((st = points_to_f32(P.Y, P.n, X32 + 3 * P.m, stream)) != LRA_OK) return st;
  }
  LRA_CUDA_TRY(cudaMemsetAsync(ws, 0, 256, stream));
  {
    LaunchScope ls(stream, "ca_batched_kernel");
    if (A.mixed) ca_batched_kernel<true><<<pl.grid, NT, pl.smem, stream>>>(A);
    else ca_batched_kernel<false><<<pl.grid, NT, pl.smem, stream>>>(A);
  }
  return cuda_status(cudaGetLastError());
}

lra_status lra_residual_sample_batched(const lra_problem* base, const lra_batch* batch, int32_t kmax,
                                       const lra_cur_batch* cur, const int32_t* Q, int32_t q, const int32_t* S,
                                       int32_t s, double* stats, lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  DevProblem P;
  lra_status st = make_dev_problem(base, nullptr, &P);
  if (st != LRA_OK) return st;
  if (batch == nullptr || cur == nullptr || !Q || !S || !stats || q < 1 || s < 1 || kmax < 1 || kmax > KMAX ||
      batch->nb < 1 || !cur->C || !cur->U || !cur->R || !cur->info)
    return LRA_ERR_INVALID_ARG;
  const size_t smem = sizeof(double) * ((size_t)q * kmax + 2 * (size_t)q * s);
  DeviceInfo dev;
  if ((st = current_device_info(&dev)) != LRA_OK) return st;
  if (smem > dev.smem_optin - 1024) return LRA_ERR_INVALID_ARG;
  LRA_CUDA_TRY(cudaFuncSetAttribute(resid_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = std::min(batch->nb, dev.sms * 8);
  {
    LaunchScope ls(stream, "resid_batched_kernel");
    resid_batched_kernel<<<grid, 256, smem, stream>>>(P, batch->blocks, batch->offsets, batch->nb, kmax, cur->C,
                                                      cur->U, cur->R, cur->info, Q, q, S, s, stats);
  }
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
