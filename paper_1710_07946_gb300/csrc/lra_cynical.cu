// lra_cynical.cu -- the cynical CUR algorithms (paper: section "CUR LRA;
// primitive, cynical, and cross-approximation algorithms"; the tests' Tests 3
// and Tests 4) over a batch of blocks: launch plan per CTA shape, autotuner and
// C ABI entry points.  The kernel is in lra_cynical_kernel.cuh.
#include <algorithm>
#include <cstring>

#include "lra_cynical_kernel.cuh"
#include "lra_internal.h"
#include "lra_profile.h"

namespace lra {

struct CynPlan {
  int threads, ctas, grid;
  size_t smem, scratch_stride, bytes;
};

// CTA shapes (the batched C-A kernel's): a sketch C-A has little work per
// barrier, so small CTAs, many per SM, are the default.
struct CynShape { int threads, ctas; };
constexpr CynShape kCynShapes[] = {{512, 1}, {256, 2}, {128, 4}, {64, 8}};
constexpr int kNumCynShapes = 4;

static const void* cyn_kernel(int threads) {
  if (threads == 512) return cynical_kernel_512();
  if (threads == 256) return cynical_kernel_256();
  if (threads == 128) return cynical_kernel_128();
  return cynical_kernel_64();
}

// The batch's shape, or -1 for the default (0, 0).
static int cyn_shape_index(const lra_batch* batch) {
  if (batch->cta_threads == 0 && batch->ctas_per_sm == 0) return -1;
  for (int i = 0; i < kNumCynShapes; ++i)
    if (kCynShapes[i].threads == batch->cta_threads && kCynShapes[i].ctas == batch->ctas_per_sm) return i;
  return -2;
}

static lra_status cyn_plan(int r, int q, int64_t max_len, int kind, int shape, CynPlan* pl) {
  DeviceInfo dev;
  lra_status st = current_device_info(&dev);
  if (st != LRA_OK) return st;
  int per_sm = 0;
  LRA_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev.device));
  const int threads = kCynShapes[shape].threads, ctas = kCynShapes[shape].ctas;
  const size_t budget = std::min(dev.smem_optin, (size_t)per_sm / ctas - 1024) - 512;
  const int ldm = (int)max_len;
  // Tests 4 steps: the fixed part at k = q (strip in shared memory when it fits);
  // the sketch C-A at k = r, ldm = q; the nucleus at r
  size_t need = std::max(ca_smem_fixed(r, q) + sizeof(double) * (size_t)r * q, nucleus_smem_bytes(r));
  bool gstrip = false;
  if (kind == 1) {
    const size_t fixed = ca_smem_fixed(q, ldm), strip = sizeof(double) * (size_t)q * ldm;
    if (fixed + strip <= budget) need = std::max(need, fixed + strip);
    else { need = std::max(need, fixed); gstrip = true; }
  }
  if (need > budget) return LRA_ERR_INVALID_ARG;
  const void* kern = cyn_kernel(threads);
  LRA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
  int occ = 0;
  LRA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, need));
  if (occ < 1) return LRA_ERR_INVALID_ARG;
  pl->threads = threads;
  pl->ctas = ctas;
  pl->grid = std::min(occ, ctas) * dev.sms;
  pl->smem = need;
  pl->scratch_stride = align_up(cyn_fixed_doubles(r, q) + (gstrip ? (size_t)q * max_len : 0), 32);
  pl->bytes = align_up(256 + sizeof(double) * pl->scratch_stride * pl->grid, 256);
  return LRA_OK;
}

static lra_status cyn_check(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par, int32_t kind,
                            int32_t q, DevProblem* P) {
  lra_status st = make_dev_problem(base, nullptr, P);
  if (st != LRA_OK) return st;
  if (batch == nullptr || par == nullptr || batch->blocks == nullptr || batch->offsets == nullptr || batch->nb < 1 ||
      batch->max_len < 1)
    return LRA_ERR_INVALID_ARG;
  if (kind != 0 && kind != 1) return LRA_ERR_INVALID_ARG;
  if (par->k < 1 || q < par->k || q > KMAX || par->sweeps < 1 || par->max_swaps < 0 || !(par->h >= 1.0) ||
      !(par->h < 1e300) || !(par->rank_tol >= 0.0) || !(par->rank_tol < 1.0) || par->mode != LRA_MODE_FP64 ||
      par->nstages != 0)
    return LRA_ERR_INVALID_ARG;
  return LRA_OK;
}

}  // namespace lra

using namespace lra;

extern "C" {

lra_status lra_cynical_batched_workspace_size(const lra_problem* base, const lra_batch* batch,
                                              const lra_ca_params* par, int32_t kind, int32_t q, size_t* bytes) {
  if (bytes == nullptr) return LRA_ERR_INVALID_ARG;
  DevProblem P;
  lra_status st = cyn_check(base, batch, par, kind, q, &P);
  if (st != LRA_OK) return st;
  size_t most = 0;
  bool any = false;
  for (int i = 0; i < kNumCynShapes; ++i) {        // enough for every shape that fits
    CynPlan pl;
    st = cyn_plan(par->k, q, batch->max_len, kind, i, &pl);
    if (st == LRA_ERR_INVALID_ARG) continue;
    if (st != LRA_OK) return st;
    any = true;
    most = std::max(most, pl.bytes);
  }
  if (!any) return LRA_ERR_INVALID_ARG;
  *bytes = most;
  return LRA_OK;
}

static lra_status cyn_launch(const DevProblem& P, const lra_batch* batch, const lra_ca_params* par, int32_t kind,
                             int32_t q, int32_t* K, int32_t* L, const int32_t* I0s, const lra_cur_batch* out,
                             void* workspace, size_t workspace_bytes, cudaStream_t stream, int shape) {
  CynPlan pl;
  lra_status st;
  if ((st = cyn_plan(par->k, q, batch->max_len, kind, shape, &pl)) != LRA_OK) return st;
  if (workspace == nullptr || workspace_bytes < pl.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return LRA_ERR_WORKSPACE;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  CynArgs A;
  std::memset(&A, 0, sizeof(A));
  A.base = P;
  A.blocks = batch->blocks;
  A.offs = batch->offsets;
  A.order = batch->order;
  A.nb = batch->nb;
  A.kind = kind;
  A.r = par->k;
  A.q = q;
  A.sweeps = par->sweeps;
  A.max_swaps = par->max_swaps;
  A.h = par->h;
  A.rank_tol = par->rank_tol;
  A.K = K;
  A.L = L;
  A.I0s = I0s;
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
  A.smem_bytes = pl.smem;
  A.max_len = batch->max_len;
  LRA_CUDA_TRY(cudaMemsetAsync(ws, 0, 256, stream));
  {
    LaunchScope ls(stream, "cynical_batched_kernel");
    void* args[] = {&A};
    LRA_CUDA_TRY(cudaLaunchKernel(cyn_kernel(pl.threads), dim3(pl.grid), dim3(pl.threads), args, pl.smem, stream));
  }
  return cuda_status(cudaGetLastError());
}

static lra_status cyn_args_ok(int32_t kind, int32_t* K, int32_t* L, const int32_t* I0s, const lra_cur_batch* out) {
  if (L == nullptr || I0s == nullptr || K == nullptr || out == nullptr || !out->I || !out->J || !out->C ||
      !out->U || !out->R || !out->logvol || !out->info || (kind != 0 && kind != 1))
    return LRA_ERR_INVALID_ARG;
  return LRA_OK;
}

lra_status lra_cynical_run_batched(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                                   int32_t kind, int32_t q, int32_t* K, int32_t* L, const int32_t* I0s,
                                   const lra_cur_batch* out, void* workspace, size_t workspace_bytes,
                                   lra_stream_t stream_) {
  DevProblem P;
  lra_status st = cyn_check(base, batch, par, kind, q, &P);
  if (st != LRA_OK) return st;
  if ((st = cyn_args_ok(kind, K, L, I0s, out)) != LRA_OK) return st;
  int shape = cyn_shape_index(batch);
  if (shape == -2) return LRA_ERR_INVALID_ARG;
  if (shape == -1 && kind == 1) shape = 0;   // Tests 4: its q-wide maxvol steps prefer 512 x 1, as C-A does
  if (shape == -1) {
    // Tests 3: the smallest CTAs whose shared-memory share holds the run
    for (int i = kNumCynShapes - 1; i >= 0 && shape < 0; --i) {
      CynPlan pl;
      st = cyn_plan(par->k, q, batch->max_len, kind, i, &pl);
      if (st == LRA_OK) shape = i;
      else if (st != LRA_ERR_INVALID_ARG) return st;
    }
    if (shape < 0) return LRA_ERR_INVALID_ARG;
  }
  return cyn_launch(P, batch, par, kind, q, K, L, I0s, out, workspace, workspace_bytes,
                    reinterpret_cast<cudaStream_t>(stream_), shape);
}

lra_status lra_cynical_batched_tune(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                                    int32_t kind, int32_t q, int32_t* K, int32_t* L, const int32_t* I0s,
                                    const lra_cur_batch* out, void* workspace, size_t workspace_bytes,
                                    lra_stream_t stream_, int32_t reps, int32_t* cta_threads, int32_t* ctas_per_sm,
                                    float* ms) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  DevProblem P;
  lra_status st = cyn_check(base, batch, par, kind, q, &P);
  if (st != LRA_OK) return st;
  if ((st = cyn_args_ok(kind, K, L, I0s, out)) != LRA_OK) return st;
  if (cta_threads == nullptr || ctas_per_sm == nullptr || reps < 1 || kind != 0) return LRA_ERR_INVALID_ARG;
  int bi = -1;
  st = time_shapes(kNumCynShapes, reps, stream, [&](int i) {
    return cyn_launch(P, batch, par, kind, q, K, L, I0s, out, workspace, workspace_bytes, stream, i);
  }, ms, &bi);
  if (st != LRA_OK) return st;
  *cta_threads = kCynShapes[bi].threads;
  *ctas_per_sm = kCynShapes[bi].ctas;
  return LRA_OK;
}

}  // extern "C"
