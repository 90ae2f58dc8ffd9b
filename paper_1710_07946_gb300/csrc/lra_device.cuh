// lra_device.cuh -- device-side building blocks of the C-A CUR library:
// input access (dense strips and kernel entry oracles), the fused multiplier
// column combinations, the (|c|, column, row) candidate order of the pivot
// searches, and the exchange between the CTAs that share one maxvol search.
//
// Floating point: the library is compiled with --fmad=false and every FP64
// operation that feeds a pivot decision is written as the explicit correctly
// rounded operation (fma(), +, -, *, /, sqrt) in a fixed order, so that a
// sequential FP64 evaluation of the same steps takes the same decisions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lra.h"

namespace lra {

constexpr int KMAX = 64;        // largest generator size k
constexpr int NT = 256;         // threads per CTA of the C-A kernels
constexpr int SLOT = 72;        // doubles per exchange slot: v, (i,j), flags, tag, col[KMAX]
constexpr double WAIT_NS = 2.0e9;   // bound on any device-side wait

// Flags carried through an exchange.
constexpr unsigned long long FLAG_NONFINITE = 1ull;

// ---------------------------------------------------------------------------
// Input view.  Dense W (FP64 or FP32, row-major) or a kernel on point sets,
// optionally post-multiplied by an implicit multiplier M (W' = W M).
// ---------------------------------------------------------------------------
struct DevProblem {
  int32_t src, dtype;
  int64_t m, n, ldw;
  const void* W;
  const double* X;
  const double* Y;
  double ell;
  // multiplier
  int32_t mkind, depth, nnz;
  int64_t s;                 // ARHT block size n / 2^d
  const int32_t* perm;       // ARHT permutation, or sparse rows (n*nnz)
  const int8_t* sign;        // ARHT diagonal, or sparse signs (n*nnz)
  double mscale;             // 2^{-d/2} or 1/sqrt(nnz), computed on the host
};

// w_ij of the original input (no multiplier).
__device__ __forceinline__ double w_entry(const DevProblem& P, int64_t i, int64_t j) {
  if (P.src == LRA_DENSE) {
    if (P.dtype == LRA_F32) return (double)__ldg(static_cast<const float*>(P.W) + i * P.ldw + j);
    return __ldg(static_cast<const double*>(P.W) + i * P.ldw + j);
  }
  const double* x = P.X + 3 * i;
  const double* y = P.Y + 3 * j;
  double dx = __ldg(x) - __ldg(y);
  double dy = __ldg(x + 1) - __ldg(y + 1);
  double dz = __ldg(x + 2) - __ldg(y + 2);
  double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
  if (P.src == LRA_KERNEL_LAPLACE) return 1.0 / sqrt(r2);
  return exp(-(r2 / (2.0 * P.ell * P.ell)));
}

// w'_ij = (W M)_ij.  ARHT: column j of M has 2^d entries, at rows a*s + t for
// perm[j] = b*s + t, of sign D_{a s + t} (-1)^{popcount(a & b)}; the terms are
// added in ascending a and the sum is scaled once.  Sparse: nnz signed terms in
// ascending stored order, scaled once.
__device__ __forceinline__ double wp_entry(const DevProblem& P, int64_t i, int64_t j) {
  if (P.mkind == LRA_MULT_NONE) return w_entry(P, i, j);
  double acc = 0.0;
  if (P.mkind == LRA_MULT_ARHT) {
    int64_t pj = __ldg(P.perm + j);
    int64_t b = pj / P.s, t = pj - b * P.s;
    int nt = 1 << P.depth;
    for (int a = 0; a < nt; ++a) {
      int64_t r = (int64_t)a * P.s + t;
      double v = w_entry(P, i, r) * (double)__ldg(P.sign + r);
      if (__popc((unsigned)(a & (int)b)) & 1) acc = acc - v; else acc = acc + v;
    }
  } else {
    const int32_t* rows = P.perm + j * P.nnz;
    const int8_t* sg = P.sign + j * P.nnz;
    for (int t = 0; t < P.nnz; ++t) {
      double v = w_entry(P, i, __ldg(rows + t));
      if (__ldg(sg + t) < 0) acc = acc - v; else acc = acc + v;
    }
  }
  return acc * P.mscale;
}

// ---------------------------------------------------------------------------
// Pivot candidates: larger |value| first, then lower column j, then lower row i.
// ---------------------------------------------------------------------------
struct Cand {
  double v;
  int32_t i, j;
};

__device__ __forceinline__ Cand cand_none() { return Cand{-1.0, 0x7fffffff, 0x7fffffff}; }

__device__ __forceinline__ bool cand_better(const Cand& a, const Cand& b) {
  return a.v > b.v || (a.v == b.v && (a.j < b.j || (a.j == b.j && a.i < b.i)));
}

__device__ __forceinline__ Cand cand_shfl_down(const Cand& c, int off) {
  Cand o;
  o.v = __shfl_down_sync(0xffffffffu, c.v, off);
  o.i = __shfl_down_sync(0xffffffffu, c.i, off);
  o.j = __shfl_down_sync(0xffffffffu, c.j, off);
  return o;
}

__device__ __forceinline__ Cand warp_best(Cand c) {
  for (int off = 16; off > 0; off >>= 1) {
    Cand o = cand_shfl_down(c, off);
    if (cand_better(o, c)) c = o;
  }
  return c;
}

// Best candidate of the CTA, returned to every thread.  red: >= 33 Cands of smem.
__device__ __forceinline__ Cand block_best(Cand c, Cand* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  c = warp_best(c);
  if (lane == 0) red[warp] = c;
  __syncthreads();
  if (warp == 0) {
    Cand d = (lane < (int)(blockDim.x >> 5)) ? red[lane] : cand_none();
    d = warp_best(d);
    if (lane == 0) red[32] = d;
  }
  __syncthreads();
  Cand r = red[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ unsigned long long block_or(unsigned long long f, unsigned long long* red) {
  for (int off = 16; off > 0; off >>= 1) f |= __shfl_down_sync(0xffffffffu, f, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = f;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long g = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) g |= red[w];
    red[32] = g;
  }
  __syncthreads();
  unsigned long long r = red[32];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Memory-model helpers (gpu scope) and a wall-clock bound for waits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// Exchange among the CTAs of one maxvol search.  Every CTA posts its best
// candidate and the current values of that candidate's column; every CTA then
// reads all posts and keeps the best one (the order above is total, so all CTAs
// agree) together with its column.  Results land in shared memory:
//   win  -- the winning candidate,  x[0..k) -- its column,  flags -- OR of flags.
// Returns false if a wait expired or another CTA aborted (status in *abort).
// ---------------------------------------------------------------------------

// A single CTA: nothing to exchange.
struct SoloGroup {
  __device__ __forceinline__ int rank() const { return 0; }
  __device__ __forceinline__ bool exchange(unsigned long long /*seq*/, const Cand& mine, const double* mycol,
                                           int mycol_stride, int k, unsigned long long myflags, Cand* win,
                                           double* x, unsigned long long* flags, int /*owner_chunk*/) const {
    if (threadIdx.x == 0) { *win = mine; *flags = myflags; }
    if (mycol != nullptr)
      for (int a = threadIdx.x; a < k; a += blockDim.x) x[a] = mycol[(int64_t)a * mycol_stride];
    __syncthreads();
    return true;
  }
};

// All CTAs of a cooperative grid, through double-buffered slots in global memory.
// A slot is (value, (i, j), flags, tag, column); its tag is written last with a
// release store and polled with acquire loads, so one round costs one post and
// one read of every slot (no atomics).  Round r uses buffer r & 1: a CTA can
// only post round r + 2 after every CTA posted round r + 1, i.e. after every CTA
// finished reading round r.
struct GridGroup {
  double* slots;             // [2][nblk][SLOT]
  unsigned int* abort;       // 0, or the status of the CTA that gave up
  int nblk;

  __device__ __forceinline__ int rank() const { return blockIdx.x; }

  __device__ bool exchange(unsigned long long seq, const Cand& mine, const double* mycol, int mycol_stride, int k,
                           unsigned long long myflags, Cand* win, double* x, unsigned long long* flags,
                           int owner_chunk) const {
    __shared__ Cand red[33];
    __shared__ unsigned long long redf[33];
    __shared__ int s_fail;
    const int tid = threadIdx.x;
    double* buf = slots + (size_t)(seq & 1ull) * nblk * SLOT;
    double* me = buf + (size_t)blockIdx.x * SLOT;
    if (mycol != nullptr)
      for (int a = tid; a < k; a += blockDim.x) me[4 + a] = mycol[(int64_t)a * mycol_stride];
    if (tid == 0) {
      me[0] = mine.v;
      reinterpret_cast<int2*>(me + 1)[0] = make_int2(mine.i, mine.j);
      reinterpret_cast<unsigned long long*>(me)[2] = myflags;
      s_fail = 0;
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release_u64(reinterpret_cast<unsigned long long*>(me) + 3, seq + 1ull);
    }
    // read every post
    Cand best = cand_none();
    unsigned long long f = 0;
    int fail = 0;
    for (int r = tid; r < nblk; r += blockDim.x) {
      const double* sl = buf + (size_t)r * SLOT;
      const unsigned long long* tag = reinterpret_cast<const unsigned long long*>(sl) + 3;
      unsigned long long t0 = 0;
      unsigned spins = 0;
      while (ld_acquire_u64(tag) != seq + 1ull) {
        if ((++spins & 255u) == 0u) {
          if (ld_relaxed_u32(abort) != 0u) { fail = 1; break; }
          unsigned long long now = globaltimer_ns();
          if (t0 == 0) t0 = now;
          else if ((double)(now - t0) > WAIT_NS) { fail = 2; break; }
        }
      }
      if (fail) break;
      Cand c;
      c.v = __ldcg(sl);
      int2 ij = __ldcg(reinterpret_cast<const int2*>(sl + 1));
      c.i = ij.x; c.j = ij.y;
      f |= __ldcg(reinterpret_cast<const unsigned long long*>(sl) + 2);
      if (cand_better(c, best)) best = c;
    }
    if (fail) {
      if (fail == 2) atomicCAS(abort, 0u, (unsigned)LRA_ERR_TIMEOUT);
      atomicOr(&s_fail, 1);
    }
    __syncthreads();
    if (s_fail) return false;
    best = block_best(best, red);
    f = block_or(f, redf);
    if (best.j != 0x7fffffff) {
      const double* ws = buf + (size_t)(best.j / owner_chunk) * SLOT;
      for (int a = tid; a < k; a += blockDim.x) x[a] = __ldcg(ws + 4 + a);
    }
    if (tid == 0) { *win = best; *flags = f; }
    __syncthreads();
    return true;
  }
};

}  // namespace lra
