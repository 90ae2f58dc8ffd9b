// lra_ca.cu -- cross-approximation CUR for one input: launch planning,
// workspace layout, the persistent C-A kernel and the nucleus kernel.
//
// One C-A run is one persistent launch.  Small inputs (at most 64 strip columns
// per step) run on a single CTA.  Larger ones run on a cooperative grid of up
// to one CTA per SM: each CTA owns a contiguous chunk of every strip and the
// CTAs meet only in the pivot exchanges (lra_device.cuh), so the sweep loop
// never returns to the host.  The nucleus (one k x k QRP) follows as a
// single-CTA kernel on the same stream.
#include <algorithm>
#include <cstring>

#include "lra_ca_loop.cuh"
#include "lra_internal.h"
#include "lra_nucleus.cuh"
#include "lra_profile.h"

namespace lra {

template <class Group, bool MIXED = false>
__global__ void __launch_bounds__(NT) ca_kernel(CaArgs A, Group grp) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* gchunk = A.strip_in_smem ? nullptr : A.gstrip + (size_t)grp.rank() * A.k * A.ldm;
  CaSmem S = ca_smem_carve(smem, A.k, A.ldm, gchunk);
  ca_loop<Group, MIXED>(grp, A, S);
}

__global__ void __launch_bounds__(NT) nucleus_kernel(const double* G, int k, double tol, double* U, int32_t* info) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int st = info[3];
  if (st != LRA_OK && st < 16) return;      // the C-A loop failed; U stays undefined
  const int r = nucleus_cta(G, k, tol, U, smem);
  if (threadIdx.x == 0) {
    info[0] = r;
    if (r < k && st == LRA_OK) info[3] = LRA_WARN_RANK_DEFICIENT;
  }
}

constexpr size_t STATIC_SMEM_RESERVE = 4096;   // the exchange / reduction arrays
constexpr int MIN_COLS_PER_CTA = 32;
constexpr int64_t MIXED_SOLO_MAX = 2048;

struct CaPlan {
  int nblk;
  int chunk_n, chunk_m, ldm;
  int strip_in_smem;
  size_t smem;
  size_t off_hdr, off_G, off_slots, off_strip, off_pts, bytes;
  int mixed;
};

static lra_status validate_params(const DevProblem& P, const lra_ca_params* par) {
  if (par == nullptr) return LRA_ERR_INVALID_ARG;
  const int64_t kmax = std::min<int64_t>(std::min<int64_t>(P.m, P.n), KMAX);
  if (par->k < 1 || par->k > kmax) return LRA_ERR_INVALID_ARG;
  if (par->sweeps < 1 || par->max_swaps < 0) return LRA_ERR_INVALID_ARG;
  if (!(par->h >= 1.0) || !(par->h < 1e300)) return LRA_ERR_INVALID_ARG;
  if (!(par->rank_tol >= 0.0) || !(par->rank_tol < 1.0)) return LRA_ERR_INVALID_ARG;
  if (par->mode != LRA_MODE_FP64 && par->mode != LRA_MODE_MIXED) return LRA_ERR_INVALID_ARG;
  if (par->nstages != 0) return LRA_ERR_INVALID_ARG;      // staged sizes: batched runs only
  if (par->ctas < 0) return LRA_ERR_INVALID_ARG;
  return LRA_OK;
}

static lra_status make_plan(const DevProblem& P, const lra_ca_params* par, CaPlan* pl) {
  DeviceInfo dev;
  lra_status st = current_device_info(&dev);
  if (st != LRA_OK) return st;
  const int k = par->k;
  const int64_t maxlen = std::max(P.m, pcols(P));
  int nblk = (int)std::min<int64_t>((maxlen + MIN_COLS_PER_CTA - 1) / MIN_COLS_PER_CTA, dev.sms);
  nblk = std::max(nblk, 1);
  if (par->ctas > 0) nblk = std::min(par->ctas, dev.sms);     // the caller's (or the tuner's) choice
  // mixed mode runs its certified FP32 steps on one CTA: take the single-CTA plan
  // for strips up to MIXED_SOLO_MAX columns (larger runs stay on the FP64 grid)
  if (par->mode == LRA_MODE_MIXED && mixed_supported(P) && maxlen <= MIXED_SOLO_MAX) nblk = 1;
  const size_t budget = dev.smem_optin - STATIC_SMEM_RESERVE;
  for (;;) {
    const int cn = (int)((pcols(P) + nblk - 1) / nblk);      // columns of W' (R has P.n <= pcols)
    const int cm = (int)((P.m + nblk - 1) / nblk);
    const int ldm = std::max(cn, cm);
    const size_t fixed = ca_smem_fixed(k, ldm);
    const size_t strip = sizeof(double) * (size_t)k * ldm;
    pl->nblk = nblk;
    pl->chunk_n = cn;
    pl->chunk_m = cm;
    pl->ldm = ldm;
    pl->strip_in_smem = (fixed + strip <= budget) ? 1 : 0;
    pl->smem = pl->strip_in_smem ? fixed + strip : fixed;
    if (pl->smem <= budget) break;
    // the per-CTA scratch alone does not fit: only possible for enormous chunks
    if (nblk >= dev.sms) return LRA_ERR_INVALID_ARG;
    nblk = std::min(dev.sms, nblk * 2);
  }
  if (pl->nblk > 256) return LRA_ERR_INVALID_ARG;      // the grid exchange polls at most 8 slots a lane
  if (pl->nblk > 1) {
    int occ = 0;
    LRA_CUDA_TRY(cudaFuncSetAttribute(ca_kernel<GridGroup>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)pl->smem));
    LRA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ca_kernel<GridGroup>, NT, pl->smem));
    if (occ < 1) return LRA_ERR_INVALID_ARG;
    if (pl->nblk > occ * dev.sms) return LRA_ERR_INVALID_ARG;
  }
  size_t o = 0;
  pl->off_hdr = o; o += 256;
  pl->off_G = o; o = align_up(o + sizeof(double) * (size_t)k * k, 256);
  pl->off_slots = o; o = align_up(o + sizeof(double) * 2 * (size_t)pl->nblk * SLOT, 256);
  pl->off_strip = o;
  if (!pl->strip_in_smem) o = align_up(o + sizeof(double) * (size_t)pl->nblk * k * pl->ldm, 256);
  // mixed mode: single-CTA runs of dense or Laplace inputs (Laplace needs FP32 points)
  pl->mixed = (par->mode == LRA_MODE_MIXED && pl->nblk == 1 && mixed_supported(P) && maxlen <= MIXED_SOLO_MAX) ? 1 : 0;
  pl->off_pts = o;
  if (pl->mixed && P.src == LRA_KERNEL_LAPLACE) o = align_up(o + sizeof(float) * 3 * (size_t)(P.m + P.n), 256);
  pl->bytes = o;
  return LRA_OK;
}

}  // namespace lra

using namespace lra;

extern "C" {

lra_status lra_ca_workspace_size(const lra_problem* prob, const lra_ca_params* par, lra_multiplier mult,
                                 size_t* bytes) {
  if (bytes == nullptr) return LRA_ERR_INVALID_ARG;
  DevProblem P;
  lra_status st = make_dev_problem(prob, mult, &P);
  if (st != LRA_OK) return st;
  if ((st = validate_params(P, par)) != LRA_OK) return st;
  CaPlan pl;
  if ((st = make_plan(P, par, &pl)) != LRA_OK) return st;
  *bytes = pl.bytes;
  return LRA_OK;
}

lra_status lra_ca_run(const lra_problem* prob, const lra_ca_params* par, lra_multiplier mult, const int32_t* I0,
                      const lra_cur* out, void* workspace, size_t workspace_bytes, lra_stream_t stream_) {
  return lra_ca_run_warm(prob, par, mult, I0, nullptr, out, workspace, workspace_bytes, stream_);
}

lra_status lra_ca_run_warm(const lra_problem* prob, const lra_ca_params* par, lra_multiplier mult, const int32_t* I0,
                           const int32_t* J0, const lra_cur* out, void* workspace, size_t workspace_bytes,
                           lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  DevProblem P;
  lra_status st = make_dev_problem(prob, mult, &P);
  if (st != LRA_OK) return st;
  if ((st = validate_params(P, par)) != LRA_OK) return st;
  if (I0 == nullptr || out == nullptr || out->I == nullptr || out->J == nullptr || out->C == nullptr ||
      out->U == nullptr || out->R == nullptr || out->logvol == nullptr || out->info == nullptr)
    return LRA_ERR_INVALID_ARG;
  CaPlan pl;
  if ((st = make_plan(P, par, &pl)) != LRA_OK) return st;
  if (workspace == nullptr || workspace_bytes < pl.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
    return LRA_ERR_WORKSPACE;
  unsigned char* ws = static_cast<unsigned char*>(workspace);

  CaArgs A;
  std::memset(&A, 0, sizeof(A));
  A.P = P;
  A.k = par->k;
  A.sweeps = par->sweeps;
  A.max_swaps = par->max_swaps;
  A.h = par->h;
  A.I0 = I0;
  A.J0 = J0;
  A.I = out->I;
  A.J = out->J;
  A.C = out->C;
  A.R = out->R;
  A.logvol = out->logvol;
  A.info = out->info;
  A.G = reinterpret_cast<double*>(ws + pl.off_G);
  A.gstrip = pl.strip_in_smem ? nullptr : reinterpret_cast<double*>(ws + pl.off_strip);
  A.chunk_n = pl.chunk_n;
  A.chunk_m = pl.chunk_m;
  A.ldm = pl.ldm;
  A.strip_in_smem = pl.strip_in_smem;
  A.mixed = pl.mixed;
  if (pl.mixed && P.src == LRA_KERNEL_LAPLACE) {
    float* X32 = reinterpret_cast<float*>(ws + pl.off_pts);
    A.P.X32 = X32;
    A.P.Y32 = X32 + 3 * P.m;
    if ((st = points_to_f32(P.X, P.m, X32, stream)) != LRA_OK) return st;
    if ((st = points_to_f32(P.Y, P.n, X32 + 3 * P.m, stream)) != LRA_OK) return st;
  }

  // exchange tags and the abort word start at zero in every run
  LRA_CUDA_TRY(cudaMemsetAsync(ws + pl.off_hdr, 0, 256, stream));
  if (pl.nblk > 1) LRA_CUDA_TRY(cudaMemsetAsync(ws + pl.off_slots, 0, pl.off_strip - pl.off_slots, stream));

  if (pl.nblk == 1) {
    auto kern = pl.mixed ? ca_kernel<SoloGroup, true> : ca_kernel<SoloGroup, false>;
    LRA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem));
    LaunchScope ls(stream, "ca_kernel");
    kern<<<1, NT, pl.smem, stream>>>(A, SoloGroup{});
    LRA_CUDA_TRY(cudaGetLastError());
  } else {
    GridGroup grp;
    grp.slots = reinterpret_cast<double*>(ws + pl.off_slots);
    grp.abort = reinterpret_cast<unsigned int*>(ws + pl.off_hdr);
    grp.nblk = pl.nblk;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(pl.nblk);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = pl.smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    LaunchScope ls(stream, "ca_kernel");
    LRA_CUDA_TRY(cudaLaunchKernelEx(&cfg, ca_kernel<GridGroup>, A, grp));
  }
  const size_t nsm = nucleus_smem_bytes(par->k);
  LRA_CUDA_TRY(cudaFuncSetAttribute(nucleus_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nsm));
  {
    LaunchScope ls(stream, "nucleus_kernel");
    nucleus_kernel<<<1, NT, nsm, stream>>>(A.G, par->k, par->rank_tol, out->U, out->info);
  }
  LRA_CUDA_TRY(cudaGetLastError());
  return LRA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// lra_ca_run_noalloc: the same C-A run for callers that cannot allocate device
// memory.  Its scratch is one file-scope device array of NOALLOC_SCRATCH_BYTES,
// resident on every device that loads the library until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace lra {

constexpr size_t NOALLOC_SCRATCH_BYTES = 256 * 1024;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of g_noalloc_scratch on the current device, looked up once per
// device (the host-side name of the array is not a device address).
static lra_status noalloc_scratch(void** addr) {
  int dev = 0;
  LRA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return LRA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return LRA_ERR_CUDA;
    g_noalloc_addr[dev] = p;
  }
  *addr = g_noalloc_addr[dev];
  return LRA_OK;
}

}  // namespace lra

extern "C" lra_status lra_ca_run_noalloc(const lra_problem* prob, const lra_ca_params* par, lra_multiplier mult,
                                         const int32_t* I0, const lra_cur* out, lra_stream_t stream) {
  size_t need = 0;
  lra_status st = lra_ca_workspace_size(prob, par, mult, &need);
  if (st != LRA_OK) return st;
  if (need > NOALLOC_SCRATCH_BYTES) return LRA_ERR_WORKSPACE;
  void* scratch = nullptr;
  if ((st = noalloc_scratch(&scratch)) != LRA_OK) return st;
  st = lra_ca_run(prob, par, mult, I0, out, scratch, NOALLOC_SCRATCH_BYTES, stream);
  if (st == LRA_ERR_CUDA) {
    // a failed CUDA call may mean the context was torn down: look the array up
    // again on the next call instead of trusting the cached address
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < NOALLOC_MAX_DEVICES) {
      std::lock_guard<std::mutex> lk(g_noalloc_mu);
      g_noalloc_addr[dev] = nullptr;
    }
  }
  return st;
}
