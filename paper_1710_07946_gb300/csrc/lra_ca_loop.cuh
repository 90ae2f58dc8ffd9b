// lra_ca_loop.cuh -- the whole C-A loop for one problem (Tests 2 schedule:
// random initial rows, a column step then a row step per loop, warm starts,
// early stop), then the outputs C, R, I, J, the core G and the volume trace.
// Each maxvol step tries the FP32 certified path first when the group is one
// CTA and the run is in mixed mode, and otherwise (or on a fallback) the FP64
// path; after a fallback the run's remaining steps go straight to FP64.
#pragma once

#include <type_traits>

#include "lra_ca_core.cuh"
#include "lra_mixed.cuh"

namespace lra {

template <class Group, bool MIXED>
__device__ StepResult run_step(const Group& grp, const CaArgs& A, const CaSmem& S, int phase, bool cold,
                               int32_t* Jsel, unsigned long long& seq, bool lead, int& n32, int& n64) {
  if constexpr (MIXED && std::is_same<Group, SoloGroup>::value) {
    // every FP64 step of a mixed run is a fallback: after the first one the run
    // stays in FP64 (the FP32 attempt would only add its cost)
    if (n64 == 0) {
      const MixedStep m = maxvol_step_mixed(A, S, phase, cold, Jsel, lead);
      if (!m.fallback) {
        ++n32;
        return StepResult{m.status, m.nswaps, m.logdet};
      }
    }
  }
  ++n64;
  return maxvol_step(grp, A, S, phase, cold, Jsel, seq, lead);
}

// The whole C-A loop for one problem, then the outputs C, R, I, J, G, logvol.
template <class Group, bool MIXED = false>
__device__ void ca_loop(const Group& grp, const CaArgs& A, const CaSmem& S) {
  const DevProblem& P = A.P;
  const int k = A.k, tid = threadIdx.x, nt = blockDim.x;
  const bool lead = grp.rank() == 0;
  // initial rows (and warm-start columns); every CTA validates them identically
  if (tid == 0) {
    int bad = 0;
    for (int a = 0; a < k; ++a) {
      int32_t v = A.I0[a];
      S.Is[a] = v;
      if (v < 0 || v >= P.m) bad = 1;
      for (int b = 0; b < a; ++b) if (S.Is[b] == v) bad = 1;
    }
    if (A.J0 != nullptr)
      for (int a = 0; a < k; ++a) {
        int32_t v = A.J0[a];
        S.Js[a] = v;
        if (v < 0 || v >= pcols(P)) bad = 1;
        for (int b = 0; b < a; ++b) if (S.Js[b] == v) bad = 1;
      }
    S.ctl[4] = bad;
  }
  if (lead) for (int s = tid; s < 2 * A.sweeps; s += nt) A.logvol[s] = __longlong_as_double(0x7ff8000000000000ll);
  __syncthreads();
  if (S.ctl[4]) {
    if (lead) for (int e = tid; e < LRA_INFO_LEN; e += nt) A.info[e] = (e == 3) ? LRA_ERR_INVALID_ARG : 0;
    return;
  }
  unsigned long long seq = A.seq ? *A.seq : 0ull;
  int status = LRA_OK, err = LRA_OK, total = 0, loops = 0, n32 = 0, n64 = 0;
  for (int s = 0; s < A.sweeps; ++s) {
    const bool cold0 = s == 0 && A.J0 == nullptr;
    StepResult r0 = run_step<Group, MIXED>(grp, A, S, 0, cold0, S.Js, seq, lead, n32, n64);
    if (A.work != nullptr && lead && tid == 0)
      *A.work += maxvol_step_flops(k, pcols(P), cold0, r0.nswaps, entry_flops(P));
    if (r0.status != LRA_OK && r0.status < 16) { err = r0.status; break; }
    if (r0.status > status) status = r0.status;
    __syncthreads();
    StepResult r1 = run_step<Group, MIXED>(grp, A, S, 1, false, S.Is, seq, lead, n32, n64);
    if (A.work != nullptr && lead && tid == 0) *A.work += maxvol_step_flops(k, P.m, false, r1.nswaps, entry_flops(P));
    if (r1.status != LRA_OK && r1.status < 16) { err = r1.status; break; }
    if (r1.status > status) status = r1.status;
    if (lead && tid == 0) { A.logvol[2 * s] = r0.logdet; A.logvol[2 * s + 1] = r1.logdet; }
    total += r0.nswaps + r1.nswaps;
    loops = s + 1;
    __syncthreads();
    if (s > 0 && r0.nswaps == 0 && r1.nswaps == 0) break;
  }
  if (A.seq) *A.seq = seq;                         // every thread keeps its own copy of the counter
  if (err != LRA_OK) {
    if (lead && tid == 0) {
      A.info[0] = 0; A.info[1] = total; A.info[2] = loops; A.info[3] = err;
      A.info[4] = n32; A.info[5] = n64; A.info[6] = k; A.info[7] = k;
    }
    return;
  }
  // outputs: C = W'[:, J] over this CTA's rows, R = W[I, :] over its columns
  // (a batch may keep only I, J and U: null C and R are not written)
  if (A.C != nullptr && A.R != nullptr) {
    const int64_t r0 = (int64_t)grp.rank() * A.chunk_m;
    const int rn = (int)max((int64_t)0, min((int64_t)A.chunk_m, P.m - r0));
    for (int it = tid; it < rn * k; it += nt) {
      int c = it / k, a = it - c * k;
      A.C[(r0 + c) * k + a] = c_entry(P, r0 + c, S.Js[a]);
    }
    const int64_t c0 = (int64_t)grp.rank() * A.chunk_n;
    const int cn = (int)max((int64_t)0, min((int64_t)A.chunk_n, P.n - c0));
    for (int it = tid; it < k * cn; it += nt) {
      int a = it / cn, c = it - a * cn;
      A.R[(int64_t)a * P.n + c0 + c] = r_entry(P, S.Is[a], c0 + c);
    }
  }
  if (lead) {
    for (int it = tid; it < k * k; it += nt) {
      int a = it / k, b = it - a * k;
      A.G[it] = wp_entry(P, S.Is[a], S.Js[b]);
    }
    for (int a = tid; a < k; a += nt) { A.I[a] = S.Is[a]; A.J[a] = S.Js[a]; }
    if (tid == 0) {
      A.info[0] = 0; A.info[1] = total; A.info[2] = loops; A.info[3] = status;
      A.info[4] = n32; A.info[5] = n64; A.info[6] = k; A.info[7] = k;
    }
  }
}


}  // namespace lra
