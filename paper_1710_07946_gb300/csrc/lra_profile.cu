// lra_profile.cu -- launch counting, NVTX ranges and optional per-launch
// CUDA-event timing.
//
// Every kernel launch of the library goes through LaunchScope: it counts the
// launch, opens an NVTX range named after the kernel around the launch call
// (free when no tracing tool is attached), and, when timing is enabled,
// brackets it with two CUDA events recorded on the launch's own stream.
// lra_profile_collect() waits for the recorded events and returns per-kernel
// totals.  Timing is meant for benchmarks; leave it off while capturing a CUDA
// graph.
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lra_internal.h"
#include "lra_profile.h"

namespace lra {

static std::atomic<long long> g_launches{0};
static std::atomic<int> g_timing{0};
static std::mutex g_mu;
struct Rec {
  const char* name;
  cudaEvent_t a, b;
};
static std::vector<Rec> g_recs;

LaunchScope::LaunchScope(cudaStream_t s, const char* name) : stream_(s), name_(name), a_(nullptr), b_(nullptr) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  nvtxRangePushA(name);
  if (g_timing.load(std::memory_order_relaxed)) {
    if (cudaEventCreate(&a_) == cudaSuccess && cudaEventCreate(&b_) == cudaSuccess) {
      cudaEventRecord(a_, stream_);
    } else {
      if (a_) cudaEventDestroy(a_);
      a_ = b_ = nullptr;
    }
  }
}

LaunchScope::~LaunchScope() {
  if (a_ != nullptr) {
    cudaEventRecord(b_, stream_);
    std::lock_guard<std::mutex> lk(g_mu);
    g_recs.push_back(Rec{name_, a_, b_});
  }
  nvtxRangePop();
}

}  // namespace lra

extern "C" {

int64_t lra_launch_count(void) { return lra::g_launches.load(); }

lra_status lra_profile_enable(int32_t on) {
  lra::g_timing.store(on ? 1 : 0);
  return LRA_OK;
}

lra_status lra_profile_collect(int32_t max_kernels, char* names, double* total_ms, int64_t* launches,
                               int32_t* n_out) {
  if (max_kernels < 0 || n_out == nullptr) return LRA_ERR_INVALID_ARG;
  std::vector<lra::Rec> recs;
  {
    std::lock_guard<std::mutex> lk(lra::g_mu);
    recs.swap(lra::g_recs);
  }
  std::vector<std::string> nm;
  std::vector<double> ms;
  std::vector<long long> cnt;
  lra_status st = LRA_OK;
  for (auto& r : recs) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
      st = LRA_ERR_CUDA;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
    size_t i = 0;
    while (i < nm.size() && nm[i] != r.name) ++i;
    if (i == nm.size()) { nm.emplace_back(r.name); ms.push_back(0.0); cnt.push_back(0); }
    ms[i] += t;
    cnt[i] += 1;
  }
  const int n = (int)std::min<size_t>(nm.size(), (size_t)max_kernels);
  for (int i = 0; i < n; ++i) {
    if (names) {
      std::strncpy(names + (size_t)i * LRA_PROFILE_NAME_LEN, nm[i].c_str(), LRA_PROFILE_NAME_LEN - 1);
      names[(size_t)i * LRA_PROFILE_NAME_LEN + LRA_PROFILE_NAME_LEN - 1] = 0;
    }
    if (total_ms) total_ms[i] = ms[i];
    if (launches) launches[i] = cnt[i];
  }
  *n_out = (int32_t)nm.size();
  return st;
}

}  // extern "C"
