// lra_batched.cu -- many independent C-A CUR approximations (the generators of
// the neutered block columns of an HSS / FMM matrix) in one persistent launch:
// the launch plan per CTA shape (with or without CTA pairs for the largest
// blocks), the autotuners over the shapes and over the staged generator sizes,
// and the batched residual sample.  The kernel itself is in
// lra_batched_kernel.cuh.
#include <algorithm>
#include <cstring>
#include <vector>

#include "lra_batched_kernel.cuh"
#include "lra_internal.h"
#include "lra_profile.h"

namespace lra {

// Residual sample of every block: E_b[Q_b, S_b] = W_b[Q_b, S_b] - (C_b U_b)[Q_b, :] R_b[:, S_b]
// and its statistics (mean, variance, mean |e|, max |e|, Frobenius ratio).
__global__ void __launch_bounds__(256) resid_batched_kernel(DevProblem base, const int64_t* blocks,
                                                            const int64_t* offs, int32_t nb, int32_t kmax,
                                                            int32_t lmax,
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
    // generator rows k (R, U columns) and columns l (C, U rows); l = k when square
    const int kf = info[LRA_INFO_LEN * (size_t)b + 6], lf = info[LRA_INFO_LEN * (size_t)b + 7];
    const int k = min(kmax, (kf > 0) ? kf : (int)min((int64_t)kmax, min(nr, nc)));
    const int l = min(lmax, (lf > 0) ? lf : k);
    const double* Cb = C + offs[2 * (size_t)b];
    const double* Rb = R + offs[2 * (size_t)b + 1];
    const double* Ub = U + (size_t)b * lmax * kmax;
    const int32_t* Q = Qs + (size_t)b * q;
    const int32_t* S = Ss + (size_t)b * s;
    {
      // sample positions outside the block are not read: the block's stats are NaN
      int bad = 0;
      for (int a = threadIdx.x; a < q; a += blockDim.x) bad |= (Q[a] < 0) | ((int64_t)Q[a] >= nr);
      for (int c = threadIdx.x; c < s; c += blockDim.x) bad |= (S[c] < 0) | ((int64_t)S[c] >= nc);
      if (__syncthreads_or(bad)) {
        if (threadIdx.x < 5) st[threadIdx.x] = __longlong_as_double(0x7ff8000000000000ll);
        continue;
      }
    }
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
      const int64_t row = Q[a];
      double t = 0.0;
      for (int d = 0; d < l; ++d) t = fma(Cb[row * l + d], Ub[d * k + bb], t);
      CU[it] = t;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < q * s; it += blockDim.x) {
      const int a = it / s, c = it - a * s;
      const int64_t col = S[c];
      double t = 0.0;
      for (int bb = 0; bb < k; ++bb) t = fma(CU[a * k + bb], Rb[(int64_t)bb * nc + col], t);
      const double w = w_entry(P, Q[a], col);
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
  int threads, ctas;        // CTA shape and CTAs per SM
  int grid;
  size_t smem;
  size_t scratch_stride;
  size_t off_pairs;         // CTA pairs' exchange slots and abort words (pairs only)
  size_t pairs_bytes;
  size_t off_pts;
  size_t bytes;
};

// CTA shapes of the batched kernel: NTB threads x MINB CTAs per SM, 16 warps
// per SM in each case (128 registers a thread fill the register file; 64
// threads is the smallest CTA the k x k elimination's layout allows).  Fewer
// threads per block and more blocks per SM trade the parallelism inside one
// block for overlap between blocks (their barriers and FP64 latencies).
struct BatchShape { int threads, ctas; };
constexpr BatchShape kShapes[] = {{512, 1}, {256, 2}, {128, 4}, {64, 8}};
constexpr int kNumShapes = 4;

static size_t ca_need(int k, int ldm, bool strip, bool mixed) {
  return ca_smem_fixed(k, ldm, mixed) + (strip ? sizeof(double) * (size_t)k * ldm : 0);
}

static void* batched_kernel_ptr(bool mixed, int threads, bool pairs = false) {
  if (threads == 512) return batched_kernel_512(mixed, pairs);
  if (threads == 256) return batched_kernel_256(mixed, pairs);
  if (pairs) return nullptr;
  if (threads == 128) return batched_kernel_128(mixed);
  return batched_kernel_64(mixed);
}

static bool shape_known(int threads, int ctas) {
  for (int i = 0; i < kNumShapes; ++i)
    if (kShapes[i].threads == threads && kShapes[i].ctas == ctas) return true;
  return false;
}

// Whether a launch of this shape runs the batch's first pair_blocks blocks on CTA
// pairs: the 512- and 256-thread shapes in FP64 mode.
static bool use_pairs(const DevProblem& P, const lra_batch* batch, const lra_ca_params* par, int threads) {
  const bool mixed = par->mode == LRA_MODE_MIXED && mixed_supported(P);
  return batch->pair_blocks > 0 && !mixed && (threads == 512 || threads == 256);
}

static lra_status batch_plan(const DevProblem& P, const lra_ca_params* par, int64_t max_len, int threads, int ctas,
                             BatchPlan* pl, bool pairs = false) {
  const int32_t kmax = par->k;
  DeviceInfo dev;
  lra_status st = current_device_info(&dev);
  if (st != LRA_OK) return st;
  int per_sm = 0;
  LRA_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev.device));
  // per CTA: its share of the SM's shared memory, less the 1 KiB the hardware
  // reserves per CTA and the kernel's static arrays
  const size_t budget = std::min(dev.smem_optin, (size_t)per_sm / ctas - 1024) - 512;
  const int ldm = (int)std::min<int64_t>(max_len, 1 << 30);
  const bool mixed = par->mode == LRA_MODE_MIXED && mixed_supported(P);
  size_t smem = std::max(ca_need(kmax, ldm, true, mixed), nucleus_smem_bytes(kmax));
  if (smem > budget) smem = budget;
  if (ca_need(kmax, ldm, false, mixed) > smem || nucleus_smem_bytes(kmax) > smem) return LRA_ERR_INVALID_ARG;
  const void* kern = batched_kernel_ptr(mixed, threads, pairs);
  if (kern == nullptr) return LRA_ERR_INVALID_ARG;       // no pair variant of this shape or mode
  LRA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  LRA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem));
  if (occ < 1) return LRA_ERR_INVALID_ARG;
  pl->threads = threads;
  pl->ctas = ctas;                                  // the shape
  pl->grid = std::min(occ, ctas) * dev.sms;         // resident CTAs of the persistent launch
  pl->smem = smem;
  // global strip scratch when the largest strip does not fit beside the fixed part
  pl->scratch_stride = (size_t)kmax * kmax + (ca_need(kmax, ldm, true, mixed) > smem ? (size_t)kmax * max_len : 0);
  pl->scratch_stride = align_up(pl->scratch_stride, 32);
  pl->off_pairs = align_up(256 + sizeof(double) * pl->scratch_stride * pl->grid, 256);
  pl->pairs_bytes = pairs ? align_up(sizeof(double) * 4 * SLOT * (size_t)(pl->grid / 2) +
                                     sizeof(unsigned int) * (size_t)(pl->grid / 2), 256) : 0;
  if (pairs && (pl->grid & 1)) return LRA_ERR_INVALID_ARG;
  pl->off_pts = pl->off_pairs + pl->pairs_bytes;
  pl->bytes = pl->off_pts;
  if (mixed && P.src == LRA_KERNEL_LAPLACE)
    pl->bytes = align_up(pl->off_pts + sizeof(float) * 3 * (size_t)(P.m + P.n), 256);
  return LRA_OK;
}

// The CTA shape a batch asks for (0, 0: the default, 512 x 1, which measured
// fastest on the octree Laplace batch: the largest blocks keep the most threads).
static void batch_shape(const lra_batch* batch, int* threads, int* ctas) {
  *threads = batch->cta_threads;
  *ctas = batch->ctas_per_sm;
  if (*threads == 0 && *ctas == 0) { *threads = 512; *ctas = 1; }
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
  // enough for every CTA shape that can hold the batch (a shape whose shared
  // memory share is too small for the largest block is left out), so that one
  // workspace serves the tuner and any choice
  size_t most = 0;
  lra_status first = LRA_ERR_INVALID_ARG;
  for (int i = 0; i < kNumShapes; ++i) {
    BatchPlan pl;
    st = batch_plan(P, par, batch->max_len, kShapes[i].threads, kShapes[i].ctas, &pl,
                    use_pairs(P, batch, par, kShapes[i].threads));
    if (st == LRA_ERR_INVALID_ARG) continue;
    if (st != LRA_OK) return st;
    first = LRA_OK;
    most = std::max(most, pl.bytes);
  }
  if (first != LRA_OK) return first;
  *bytes = most;
  return LRA_OK;
}

namespace {

lra_status batched_check(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par, const int32_t* I0,
                         const lra_cur_batch* out, DevProblem* P) {
  lra_status st = make_dev_problem(base, nullptr, P);
  if (st != LRA_OK) return st;
  if (batch == nullptr || par == nullptr || out == nullptr || I0 == nullptr) return LRA_ERR_INVALID_ARG;
  if (batch->blocks == nullptr || batch->offsets == nullptr || batch->nb < 1 || batch->max_len < 1 ||
      batch->pair_blocks < 0 || batch->pair_blocks > batch->nb)
    return LRA_ERR_INVALID_ARG;
  if (par->k < 1 || par->k > KMAX || par->sweeps < 1 || par->max_swaps < 0 || !(par->h >= 1.0) ||
      !(par->h < 1e300) || !(par->rank_tol >= 0.0) || !(par->rank_tol < 1.0) ||
      (par->mode != LRA_MODE_FP64 && par->mode != LRA_MODE_MIXED) || !stages_valid(par))
    return LRA_ERR_INVALID_ARG;
  if (!out->I || !out->J || !out->U || !out->logvol || !out->info) return LRA_ERR_INVALID_ARG;
  if ((out->C == nullptr) != (out->R == nullptr)) return LRA_ERR_INVALID_ARG;   // both factors, or neither
  return LRA_OK;
}

lra_status batched_launch(const DevProblem& P, const lra_batch* batch, const lra_ca_params* par, const int32_t* I0,
                          const lra_cur_batch* out, void* workspace, size_t workspace_bytes, cudaStream_t stream,
                          int threads, int ctas) {
  if (!shape_known(threads, ctas)) return LRA_ERR_INVALID_ARG;
  BatchPlan pl;
  lra_status st;
  const bool pairs = use_pairs(P, batch, par, threads);
  if ((st = batch_plan(P, par, batch->max_len, threads, ctas, &pl, pairs)) != LRA_OK) return st;
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
  A.work = out->work;
  A.U = out->U;
  A.logvol = out->logvol;
  A.info = out->info;
  A.counter = reinterpret_cast<unsigned int*>(ws);
  A.scratch = reinterpret_cast<double*>(ws + 256);
  A.scratch_stride = pl.scratch_stride;
  A.smem_bytes = pl.smem;
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
  if (pairs) {
    // the pairs' exchange slots and abort words start at zero in every launch
    A.nteam = batch->pair_blocks;
    A.tslots = reinterpret_cast<double*>(ws + pl.off_pairs);
    A.tabort = reinterpret_cast<unsigned int*>(ws + pl.off_pairs + sizeof(double) * 4 * SLOT * (size_t)(pl.grid / 2));
    LRA_CUDA_TRY(cudaMemsetAsync(ws + pl.off_pairs, 0, pl.pairs_bytes, stream));
  }
  {
    LaunchScope ls(stream, "ca_batched_kernel");
    const void* kern = batched_kernel_ptr(A.mixed != 0, pl.threads, pairs);
    void* args[] = {&A};
    if (pairs) {
      // the two CTAs of a pair wait for each other: a cooperative launch makes the
      // whole grid resident at once
      cudaLaunchConfig_t cfg;
      std::memset(&cfg, 0, sizeof(cfg));
      cfg.gridDim = dim3(pl.grid);
      cfg.blockDim = dim3(pl.threads);
      cfg.dynamicSmemBytes = pl.smem;
      cfg.stream = stream;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      LRA_CUDA_TRY(cudaLaunchKernelExC(&cfg, kern, args));
    } else {
      LRA_CUDA_TRY(cudaLaunchKernel(kern, dim3(pl.grid), dim3(pl.threads), args, pl.smem, stream));
    }
  }
  return cuda_status(cudaGetLastError());
}

}  // namespace

lra_status lra_ca_run_batched(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                              const int32_t* I0, const lra_cur_batch* out, void* workspace, size_t workspace_bytes,
                              lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  DevProblem P;
  lra_status st = batched_check(base, batch, par, I0, out, &P);
  if (st != LRA_OK) return st;
  int threads, ctas;
  batch_shape(batch, &threads, &ctas);
  return batched_launch(P, batch, par, I0, out, workspace, workspace_bytes, stream, threads, ctas);
}

lra_status lra_ca_batched_tune(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                               const int32_t* I0, const lra_cur_batch* out, void* workspace, size_t workspace_bytes,
                               lra_stream_t stream_, int32_t reps, int32_t* cta_threads, int32_t* ctas_per_sm,
                               float* ms) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  DevProblem P;
  lra_status st = batched_check(base, batch, par, I0, out, &P);
  if (st != LRA_OK) return st;
  if (cta_threads == nullptr || ctas_per_sm == nullptr || reps < 1) return LRA_ERR_INVALID_ARG;
  int bi = -1;
  st = time_shapes(kNumShapes, reps, stream, [&](int i) {
    BatchPlan pl;
    const lra_status fit = batch_plan(P, par, batch->max_len, kShapes[i].threads, kShapes[i].ctas, &pl,
                                      use_pairs(P, batch, par, kShapes[i].threads));
    if (fit != LRA_OK) return fit;
    return batched_launch(P, batch, par, I0, out, workspace, workspace_bytes, stream, kShapes[i].threads,
                          kShapes[i].ctas);
  }, ms, &bi);
  if (st != LRA_OK) return st;
  *cta_threads = kShapes[bi].threads;
  *ctas_per_sm = kShapes[bi].ctas;
  return LRA_OK;
}

lra_status lra_ca_batched_tune_stages(const lra_problem* base, const lra_problem* exact, const lra_batch* batch,
                                      const lra_ca_params* par, const int32_t* I0, const lra_cur_batch* out,
                                      void* workspace, size_t workspace_bytes, const int32_t* Q, int32_t q,
                                      const int32_t* S, int32_t s, double* stats, double tol,
                                      const int32_t* schedules, int32_t nsched, int32_t reps, lra_stream_t stream_,
                                      int32_t* best, float* ms, double* err) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (par == nullptr || batch == nullptr || schedules == nullptr || best == nullptr || stats == nullptr ||
      nsched < 1 || reps < 1 || !(tol >= 0.0) || out == nullptr || out->C == nullptr || out->R == nullptr)
    return LRA_ERR_INVALID_ARG;
  const lra_problem* ex = exact ? exact : base;
  const int nb = batch->nb;
  // every schedule well formed (host checks, before any CUDA call)
  for (int i = 0; i < nsched; ++i) {
    const int32_t* sc = schedules + (size_t)i * (2 + LRA_MAX_STAGES);
    lra_ca_params pi = *par;
    pi.nstages = sc[0];
    pi.rank_margin = sc[1];
    if (pi.nstages < 1 || pi.nstages > LRA_MAX_STAGES) return LRA_ERR_INVALID_ARG;
    for (int t = 0; t < LRA_MAX_STAGES; ++t) pi.k_stages[t] = t < pi.nstages ? sc[2 + t] : 0;
    if (!stages_valid(&pi)) return LRA_ERR_INVALID_ARG;
  }
  int threads, ctas;
  batch_shape(batch, &threads, &ctas);
  std::vector<double> hst((size_t)nb * 5);
  std::vector<int32_t> hinfo((size_t)nb * LRA_INFO_LEN);
  cudaEvent_t e0, e1;
  LRA_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return LRA_ERR_CUDA; }
  lra_status st = LRA_OK;
  int bi = -1, last = -1;
  float bt = 0.f;
  for (int i = 0; i < nsched && st == LRA_OK; ++i) {
    const int32_t* sc = schedules + (size_t)i * (2 + LRA_MAX_STAGES);
    lra_ca_params pi = *par;
    pi.nstages = sc[0];
    pi.rank_margin = sc[1];
    if (pi.nstages < 1 || pi.nstages > LRA_MAX_STAGES) { st = LRA_ERR_INVALID_ARG; break; }
    for (int t = 0; t < LRA_MAX_STAGES; ++t) pi.k_stages[t] = t < pi.nstages ? sc[2 + t] : 0;
    DevProblem P;
    if ((st = batched_check(base, batch, &pi, I0, out, &P)) != LRA_OK) break;
    float fastest = -1.f;
    for (int r = 0; r < reps && st == LRA_OK; ++r) {
      float t = 0.f;
      if (cudaEventRecord(e0, stream) != cudaSuccess) { st = LRA_ERR_CUDA; break; }
      if ((st = batched_launch(P, batch, &pi, I0, out, workspace, workspace_bytes, stream, threads, ctas)) != LRA_OK)
        break;
      if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) { st = LRA_ERR_CUDA; break; }
      if (fastest < 0.f || t < fastest) fastest = t;
    }
    if (st != LRA_OK) break;
    last = i;
    // every block: a usable status and a sampled error within tol
    if ((st = lra_residual_sample_batched(ex, batch, par->k, out, Q, q, S, s, stats, stream_)) != LRA_OK) break;
    if (cudaMemcpyAsync(hst.data(), stats, sizeof(double) * hst.size(), cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(hinfo.data(), out->info, sizeof(int32_t) * hinfo.size(), cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) { st = LRA_ERR_CUDA; break; }
    double emax = 0.0;
    bool ok = true;
    for (int b = 0; b < nb; ++b) {
      const double e = hst[(size_t)b * 5 + 4];
      const int32_t bs = hinfo[(size_t)b * LRA_INFO_LEN + 3];
      if (!(e <= tol) || (bs != LRA_OK && bs < 16)) ok = false;
      if (!(e <= emax)) emax = e;           // NaN propagates
    }
    if (ms != nullptr) ms[i] = fastest;
    if (err != nullptr) err[i] = emax;
    if (ok && (bi < 0 || fastest < bt)) { bt = fastest; bi = i; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LRA_OK) return st;
  if (bi < 0) return LRA_ERR_INVALID_ARG;
  *best = bi;
  if (last != bi) {                          // leave the chosen schedule's results in out
    const int32_t* sc = schedules + (size_t)bi * (2 + LRA_MAX_STAGES);
    lra_ca_params pb = *par;
    pb.nstages = sc[0];
    pb.rank_margin = sc[1];
    for (int t = 0; t < LRA_MAX_STAGES; ++t) pb.k_stages[t] = t < pb.nstages ? sc[2 + t] : 0;
    DevProblem P;
    if ((st = batched_check(base, batch, &pb, I0, out, &P)) != LRA_OK) return st;
    return batched_launch(P, batch, &pb, I0, out, workspace, workspace_bytes, stream, threads, ctas);
  }
  return LRA_OK;
}

int32_t lra_ca_batched_shapes(int32_t* threads, int32_t* ctas, int32_t cap) {
  for (int i = 0; i < kNumShapes && i < cap; ++i) {
    if (threads) threads[i] = kShapes[i].threads;
    if (ctas) ctas[i] = kShapes[i].ctas;
  }
  return kNumShapes;
}

lra_status lra_residual_sample_batched(const lra_problem* base, const lra_batch* batch, int32_t kmax,
                                       const lra_cur_batch* cur, const int32_t* Q, int32_t q, const int32_t* S,
                                       int32_t s, double* stats, lra_stream_t stream_) {
  return lra_residual_sample_batched_rect(base, batch, kmax, kmax, cur, Q, q, S, s, stats, stream_);
}

lra_status lra_residual_sample_batched_rect(const lra_problem* base, const lra_batch* batch, int32_t kmax,
                                            int32_t lmax, const lra_cur_batch* cur, const int32_t* Q, int32_t q,
                                            const int32_t* S, int32_t s, double* stats, lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  DevProblem P;
  lra_status st = make_dev_problem(base, nullptr, &P);
  if (st != LRA_OK) return st;
  if (batch == nullptr || cur == nullptr || !Q || !S || !stats || q < 1 || s < 1 || kmax < 1 || kmax > KMAX ||
      lmax < kmax || lmax > 2 * KMAX || batch->nb < 1 || !cur->C || !cur->U || !cur->R || !cur->info)
    return LRA_ERR_INVALID_ARG;
  const size_t smem = sizeof(double) * ((size_t)q * kmax + 2 * (size_t)q * s);
  DeviceInfo dev;
  if ((st = current_device_info(&dev)) != LRA_OK) return st;
  if (smem > dev.smem_optin - 1024) return LRA_ERR_INVALID_ARG;
  LRA_CUDA_TRY(cudaFuncSetAttribute(resid_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = std::min(batch->nb, dev.sms * 8);
  {
    LaunchScope ls(stream, "resid_batched_kernel");
    resid_batched_kernel<<<grid, 256, smem, stream>>>(P, batch->blocks, batch->offsets, batch->nb, kmax, lmax,
                                                      cur->C, cur->U, cur->R, cur->info, Q, q, S, s, stats);
  }
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
