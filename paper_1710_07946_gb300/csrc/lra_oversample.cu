// lra_oversample.cu -- rectangular k x l generators for a batch of blocks
// (paper: Algorithm algrup, greedy expansions of a k x k submatrix to k x l;
// Theorem th3 bounds the CUR error of such generators), one CTA per block from a
// work queue, after a batched C-A run has produced each block's square
// generator (rows I, columns J).
//
// Per block: X = B^{-1} W'[I, :] is the C matrix of a maxvol step on the row
// strip warm-started at J with no swaps (the single-CTA maxvol arithmetic);
// then p times the column outside the generator with the largest s_j =
// ||X[:, j]||^2 joins it (the squared volume grows by 1 + s_j) and every other
// column is whitened again, X[:, q] -= gamma (x . X[:, q]) x with gamma =
// (1 - 1/sqrt(1 + sigma)) / sigma (Sherman-Morrison for (C C^T)^{-1}); the
// columns are independent, one thread each.  Outputs C = W'[:, J'], the
// rectangular nucleus U of W'[I, J'] and R = W[I, :].
#include <algorithm>
#include <cstring>

#include "lra_ca_core.cuh"
#include "lra_internal.h"
#include "lra_nucleus.cuh"
#include "lra_profile.h"

namespace lra {

struct OvArgs {
  DevProblem base;
  const int64_t* blocks;      // nb x 4
  const int64_t* offs;        // nb x 2: offsets of C_b (nrows x l_b) and R_b (k_b x ncols) in the outputs
  const int32_t* order;
  int32_t nb, kmax, pextra, lmax;
  double h, rank_tol;
  const int32_t* Iin;         // nb x kmax
  const int32_t* Jin;         // nb x kmax
  const int32_t* info_in;     // nb x LRA_INFO_LEN (k used = info[6], status = info[3])
  int32_t* I;                 // nb x kmax
  int32_t* J;                 // nb x lmax
  double* C;
  double* R;
  double* U;                  // nb x lmax x kmax
  int32_t* info;              // nb x LRA_INFO_LEN
  unsigned int* counter;
  double* scratch;            // per CTA: G (kmax x lmax) then, if needed, a strip (kmax x max_len)
  size_t scratch_stride;
  size_t smem_bytes;
  int64_t max_len;
};

__global__ void __launch_bounds__(NT) oversample_kernel(OvArgs B) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_b;
  __shared__ double s_x[KMAX];
  __shared__ double s_g[2];
  double* G = B.scratch + (size_t)blockIdx.x * B.scratch_stride;
  double* gstrip = G + (size_t)B.kmax * B.lmax;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (;;) {
    if (tid == 0) {
      const unsigned int qh = atomicAdd(B.counter, 1u);
      s_b = (qh < (unsigned)B.nb) ? (B.order ? B.order[qh] : (int)qh) : -1;
    }
    __syncthreads();
    const int b = s_b;
    __syncthreads();
    if (b < 0) break;
    int32_t* info = B.info + LRA_INFO_LEN * (size_t)b;
    const int32_t* inf0 = B.info_in + LRA_INFO_LEN * (size_t)b;
    const int64_t r0 = B.blocks[4 * (size_t)b], nr = B.blocks[4 * (size_t)b + 1];
    const int64_t c0 = B.blocks[4 * (size_t)b + 2], nc = B.blocks[4 * (size_t)b + 3];
    const int st_in = inf0[3];
    const int k = inf0[6];
    if (r0 < 0 || c0 < 0 || nr < 1 || nc < 1 || r0 + nr > B.base.m || c0 + nc > B.base.n || nr > B.max_len ||
        nc > B.max_len || (st_in != LRA_OK && st_in < 16) || k < 1 || k > B.kmax || k > min(nr, nc)) {
      for (int e = tid; e < LRA_INFO_LEN; e += nt)
        info[e] = (e == 3) ? ((st_in != LRA_OK && st_in < 16) ? st_in : LRA_ERR_INVALID_ARG) : 0;
      continue;
    }
    const int lb = (int)min((int64_t)(k + B.pextra), nc);
    CaArgs A;
    std::memset(&A, 0, sizeof(A));
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
    A.k = k;
    A.max_swaps = 0;
    A.h = B.h;
    A.chunk_n = (int)nc;
    A.chunk_m = (int)nr;
    A.ldm = (int)max(nr, nc);
    A.strip_in_smem = ca_smem_fixed(k, A.ldm) + sizeof(double) * (size_t)k * A.ldm <= B.smem_bytes;
    A.gstrip = A.strip_in_smem ? nullptr : gstrip;
    int32_t* Jb = B.J + (size_t)b * B.lmax;
    int l = k, st = LRA_OK;
    {
      const CaSmem S = ca_smem_carve(smem, k, A.ldm, A.gstrip);
      for (int a = tid; a < k; a += nt) {
        S.Is[a] = B.Iin[(size_t)b * B.kmax + a];
        S.Js[a] = B.Jin[(size_t)b * B.kmax + a];
      }
      __syncthreads();
      unsigned long long seq = 0;
      const StepResult sr = maxvol_step(SoloGroup{}, A, S, 0, false, S.Js, seq, true);
      __syncthreads();
      st = (sr.status == LRA_WARN_NOT_CONVERGED) ? LRA_OK : sr.status;
      if (st != LRA_OK && st < 16) {
        if (tid == 0) {
          info[0] = 0; info[1] = 0; info[2] = 0; info[3] = st; info[4] = 0; info[5] = 0; info[6] = k; info[7] = k;
        }
        __syncthreads();
        continue;
      }
      if (st == LRA_WARN_RANK_DEFICIENT) {
        // zero pivot: no expansion, the square generator as given
        for (int a = tid; a < k; a += nt) Jb[a] = B.Jin[(size_t)b * B.kmax + a];
      } else {
        for (int a = tid; a < k; a += nt) Jb[a] = S.Js[a];
        double* M = S.M;
        double* s = S.tq;                        // per-column s_j (ldm doubles)
        // s_j of the columns outside the generator, ascending rows
        for (int c = tid; c < nc; c += nt) {
          if (S.pos[c]) continue;
          double v = 0.0;
          for (int i = 0; i < k; ++i) v = fma(M[(int64_t)i * A.ldm + c], M[(int64_t)i * A.ldm + c], v);
          s[c] = v;
        }
        __syncthreads();
        for (int g = 0; g < B.pextra && l < lb; ++g) {
          Cand mine = cand_none();
          for (int c = tid; c < nc; c += nt)
            if (!S.pos[c]) cand_consider(mine, mag_key(s[c]), 0, c);
          unsigned long long fl = 0;
          const Cand w = block_best(mine, fl, S.red);
          if (w.key == 0ull || w.key == mag_key(0.0)) break;     // nothing left, or no volume gain
          const int js = w.j;
          if (tid == 0) {
            const double sigma = s[js];
            s_g[0] = (1.0 - 1.0 / sqrt(1.0 + sigma)) / sigma;
            S.pos[js] = l + 1;
            Jb[l] = js;
          }
          for (int i = tid; i < k; i += nt) s_x[i] = M[(int64_t)i * A.ldm + js];
          __syncthreads();
          ++l;
          const double gamma = s_g[0];
          for (int c = tid; c < nc; c += nt) {
            if (S.pos[c]) continue;
            double t = 0.0;
            for (int i = 0; i < k; ++i) t = fma(s_x[i], M[(int64_t)i * A.ldm + c], t);
            const double cc = gamma * t;
            double v = 0.0;
            for (int i = 0; i < k; ++i) {
              const double x = fma(-cc, s_x[i], M[(int64_t)i * A.ldm + c]);
              M[(int64_t)i * A.ldm + c] = x;
              v = fma(x, x, v);
            }
            s[c] = v;
          }
          __syncthreads();
        }
      }
    }
    __syncthreads();
    // outputs at l: C = W'[:, J'] (nr x l), R = W[I, :] (k x nc), G = W'[I, J'] -> U
    const int32_t* Ib = B.Iin + (size_t)b * B.kmax;
    double* Cb = B.C + B.offs[2 * (size_t)b];
    double* Rb = B.R + B.offs[2 * (size_t)b + 1];
    for (int64_t it = tid; it < nr * l; it += nt) {
      const int64_t i = it / l;
      const int a = (int)(it - i * l);
      Cb[it] = wp_entry(A.P, i, Jb[a]);
    }
    for (int64_t it = tid; it < (int64_t)k * nc; it += nt) {
      const int a = (int)(it / nc);
      const int64_t c = it - (int64_t)a * nc;
      Rb[it] = w_entry(A.P, Ib[a], c);
    }
    for (int it = tid; it < k * l; it += nt) {
      const int a = it / l, c = it - a * l;
      G[it] = wp_entry(A.P, Ib[a], Jb[c]);
    }
    for (int a = tid; a < k; a += nt) B.I[(size_t)b * B.kmax + a] = Ib[a];
    __syncthreads();
    const int rank = nucleus_rect_cta(G, k, l, B.rank_tol, B.U + (size_t)b * B.lmax * B.kmax, smem);
    if (tid == 0) {
      if (rank < k && st == LRA_OK) st = LRA_WARN_RANK_DEFICIENT;
      info[0] = rank; info[1] = 0; info[2] = 0; info[3] = st; info[4] = 0; info[5] = 0; info[6] = k; info[7] = l;
    }
    __syncthreads();
  }
}

struct OvPlan {
  int grid;
  size_t smem, scratch_stride, bytes;
};

static lra_status ov_plan(int kmax, int lmax, int64_t max_len, OvPlan* pl) {
  DeviceInfo dev;
  lra_status st = current_device_info(&dev);
  if (st != LRA_OK) return st;
  const size_t budget = dev.smem_optin - 4096;
  const int ldm = (int)max_len;
  const size_t fixed = ca_smem_fixed(kmax, ldm), strip = sizeof(double) * (size_t)kmax * ldm;
  size_t need = std::max(fixed, nucleus_rect_smem_bytes(kmax, lmax));
  bool gstrip = true;
  if (std::max(fixed + strip, need) <= budget) { need = std::max(fixed + strip, need); gstrip = false; }
  if (need > budget) return LRA_ERR_INVALID_ARG;
  LRA_CUDA_TRY(cudaFuncSetAttribute(oversample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
  int occ = 0;
  LRA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, oversample_kernel, NT, need));
  if (occ < 1) return LRA_ERR_INVALID_ARG;
  pl->grid = occ * dev.sms;
  pl->smem = need;
  pl->scratch_stride = align_up((size_t)kmax * lmax + (gstrip ? (size_t)kmax * max_len : 0), 32);
  pl->bytes = align_up(256 + sizeof(double) * pl->scratch_stride * pl->grid, 256);
  return LRA_OK;
}

static lra_status ov_check(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par, int32_t pextra,
                           DevProblem* P) {
  lra_status st = make_dev_problem(base, nullptr, P);
  if (st != LRA_OK) return st;
  if (batch == nullptr || par == nullptr || batch->blocks == nullptr || batch->offsets == nullptr || batch->nb < 1 ||
      batch->max_len < 1)
    return LRA_ERR_INVALID_ARG;
  if (par->k < 1 || par->k > KMAX || pextra < 0 || pextra > KMAX || !(par->h >= 1.0) || !(par->h < 1e300) ||
      !(par->rank_tol >= 0.0) || !(par->rank_tol < 1.0))
    return LRA_ERR_INVALID_ARG;
  return LRA_OK;
}

}  // namespace lra

using namespace lra;

extern "C" {

lra_status lra_oversample_batched_workspace_size(const lra_problem* base, const lra_batch* batch,
                                                 const lra_ca_params* par, int32_t pextra, size_t* bytes) {
  if (bytes == nullptr) return LRA_ERR_INVALID_ARG;
  DevProblem P;
  lra_status st = ov_check(base, batch, par, pextra, &P);
  if (st != LRA_OK) return st;
  OvPlan pl;
  if ((st = ov_plan(par->k, par->k + pextra, batch->max_len, &pl)) != LRA_OK) return st;
  *bytes = pl.bytes;
  return LRA_OK;
}

lra_status lra_oversample_batched(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                                  int32_t pextra, const lra_cur_batch* in, const lra_cur_batch* out, void* workspace,
                                  size_t workspace_bytes, lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  DevProblem P;
  lra_status st = ov_check(base, batch, par, pextra, &P);
  if (st != LRA_OK) return st;
  if (in == nullptr || out == nullptr || !in->I || !in->J || !in->info || !out->I || !out->J || !out->C || !out->U ||
      !out->R || !out->info)
    return LRA_ERR_INVALID_ARG;
  OvPlan pl;
  if ((st = ov_plan(par->k, par->k + pextra, batch->max_len, &pl)) != LRA_OK) return st;
  if (workspace == nullptr || workspace_bytes < pl.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return LRA_ERR_WORKSPACE;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  OvArgs A;
  std::memset(&A, 0, sizeof(A));
  A.base = P;
  A.blocks = batch->blocks;
  A.offs = batch->offsets;
  A.order = batch->order;
  A.nb = batch->nb;
  A.kmax = par->k;
  A.pextra = pextra;
  A.lmax = par->k + pextra;
  A.h = par->h;
  A.rank_tol = par->rank_tol;
  A.Iin = in->I;
  A.Jin = in->J;
  A.info_in = in->info;
  A.I = out->I;
  A.J = out->J;
  A.C = out->C;
  A.R = out->R;
  A.U = out->U;
  A.info = out->info;
  A.counter = reinterpret_cast<unsigned int*>(ws);
  A.scratch = reinterpret_cast<double*>(ws + 256);
  A.scratch_stride = pl.scratch_stride;
  A.smem_bytes = pl.smem;
  A.max_len = batch->max_len;
  LRA_CUDA_TRY(cudaMemsetAsync(ws, 0, 256, stream));
  {
    LaunchScope ls(stream, "oversample_kernel");
    oversample_kernel<<<pl.grid, NT, pl.smem, stream>>>(A);
  }
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
