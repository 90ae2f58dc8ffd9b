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
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "lra.h"

namespace lra {

constexpr int KMAX = 64;        // largest generator size k
constexpr int NT = 512;         // threads per CTA of the C-A kernels
constexpr int SLOT = 72;        // doubles per exchange slot: v, (i,j), flags, tag, col[KMAX]
constexpr double WAIT_NS = 2.0e9;   // bound on any device-side wait
constexpr int TERMS = 4;        // multiplier terms fetched together in a strip gather

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
  int32_t mside;             // 0: W' = W M (right, M n x n); 1: W' = M^T W (left, M m x m)
  int64_t s;                 // ARHT block size (n or m) / 2^d
  const int32_t* perm;       // ARHT permutation, or sparse rows (n*nnz)
  const int8_t* sign;        // ARHT diagonal, or sparse signs (n*nnz)
  const int32_t* bval;       // bidiagonal products: integer weights (n*nnz, nnz = min(2^q, n) slots)
  const double* fwt;         // ARFT real form: weights of the 2n columns (2n*nnz, nnz = 2^d slots)
  double mscale;             // 2^{-d/2} or 1/sqrt(nnz), computed on the host
  // FP32 copies for the mixed-precision steps
  const float* X32;          // kernel points rounded to FP32 (m x 3), or null
  const float* Y32;          // (n x 3), or null
  float mscale32;            // mscale rounded to FP32
  float mscale_err;          // bound on |mscale32 - exact scale|
};

// Columns of the pre-processed W': 2n for the real-form Fourier multiplier
// (W' = W [Re M, Im M]), n otherwise.
__host__ __device__ __forceinline__ int64_t pcols(const DevProblem& P) {
  return P.mkind == LRA_MULT_ARFT ? 2 * P.n : P.n;
}

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
  if (P.src == LRA_KERNEL_LAPLACE) {
    // FP32 entries: the FP64 squared distance rounded to FP32, then a correctly
    // rounded FP32 square root and reciprocal (the FP32 pipe instead of FP64)
    if (P.dtype == LRA_F32) return (double)__fdiv_rn(1.0f, __fsqrt_rn(__double2float_rn(r2)));
    // BF16 entries: the FP32 entry rounded to bfloat16, to nearest even
    if (P.dtype == LRA_BF16)
      return (double)__bfloat162float(__float2bfloat16_rn(__fdiv_rn(1.0f, __fsqrt_rn(__double2float_rn(r2)))));
    return 1.0 / sqrt(r2);
  }
  return exp(-(r2 / (2.0 * P.ell * P.ell)));
}

// w'_ij of the pre-processed input.  Right multiplier: W' = W M, w'_ij =
// sum over the nonzeros M_rj of M_rj w_ir (column j of M combines entries of
// row i).  Left multiplier: W' = M^T W, w'_ij = sum over the nonzeros M_ri of
// M_ri w_rj (column i of M combines entries of column j).  In both cases the
// terms of one column mc of M are taken in the same order.  ARHT: column mc of
// M has 2^d entries, at rows a*s + t for perm[mc] = b*s + t, of sign
// D_{a s + t} (-1)^{popcount(a & b)}; the terms are added in ascending a and
// the sum is scaled once.  Sparse: nnz signed terms in ascending stored order,
// scaled once.  The terms are fetched TERMS at a time before they are added
// (same order of additions), so their loads overlap.
// The multiplier's column combination, out of line: the C-A kernels inline
// wp_entry at every gather site, and only the no-multiplier case is hot there
// (the batched kernels never have one); keeping the combinations in one called
// function keeps them from crowding the registers of those sites.
static __device__ __noinline__ double wp_entry_mult(const DevProblem& P, int64_t i, int64_t j);

__device__ __forceinline__ double wp_entry(const DevProblem& P, int64_t i, int64_t j) {
  if (P.mkind == LRA_MULT_NONE) return w_entry(P, i, j);
  return wp_entry_mult(P, i, j);
}

static __device__ __noinline__ double wp_entry_mult(const DevProblem& P, int64_t i, int64_t j) {
  const bool left = P.mside != 0;
  const int64_t mc = left ? i : j;                  // the column of M that combines the terms
  auto term = [&](int64_t r) -> double { return left ? w_entry(P, r, j) : w_entry(P, i, r); };
  double acc = 0.0;
  if (P.mkind == LRA_MULT_ARFT) {
    // real-form Fourier column: 2^d real weights in ascending rows, each fma(weight, w, sum)
    const int32_t* rows = P.perm + mc * P.nnz;
    const double* ws = P.fwt + mc * P.nnz;
    for (int t0 = 0; t0 < P.nnz; t0 += TERMS) {
      double v[TERMS], c[TERMS];
#pragma unroll
      for (int e = 0; e < TERMS; ++e)
        if (t0 + e < P.nnz) { c[e] = __ldg(ws + t0 + e); v[e] = term(__ldg(rows + t0 + e)); }
#pragma unroll
      for (int e = 0; e < TERMS; ++e)
        if (t0 + e < P.nnz) acc = fma(c[e], v[e], acc);
    }
    return acc * P.mscale;
  }
  if (P.mkind == LRA_MULT_BIDIAG) {
    // product of bidiagonal factors: up to min(2^q, n) integer-weighted terms
    // in ascending rows (value 0 = unused slot), each fma(value, w, sum)
    const int32_t* rows = P.perm + mc * P.nnz;
    const int32_t* vs = P.bval + mc * P.nnz;
    for (int t0 = 0; t0 < P.nnz; t0 += TERMS) {
      double v[TERMS];
      int c[TERMS];
#pragma unroll
      for (int e = 0; e < TERMS; ++e) {
        c[e] = 0;
        if (t0 + e < P.nnz) {
          c[e] = __ldg(vs + t0 + e);
          if (c[e] != 0) v[e] = term(__ldg(rows + t0 + e));
        }
      }
#pragma unroll
      for (int e = 0; e < TERMS; ++e)
        if (c[e] != 0) acc = fma((double)c[e], v[e], acc);
    }
    return acc * P.mscale;
  }
  if (P.mkind == LRA_MULT_ARHT) {
    const int64_t pj = __ldg(P.perm + mc);
    const int64_t b = pj / P.s, t = pj - b * P.s;
    const int nt = 1 << P.depth;
    for (int a0 = 0; a0 < nt; a0 += TERMS) {
      double v[TERMS];
#pragma unroll
      for (int e = 0; e < TERMS; ++e) {
        const int a = a0 + e;
        if (a < nt) {
          const int64_t r = (int64_t)a * P.s + t;
          const double w = term(r);
          v[e] = (__ldg(P.sign + r) < 0) ? -w : w;       // == w * (double)sign, exactly
        }
      }
#pragma unroll
      for (int e = 0; e < TERMS; ++e) {
        const int a = a0 + e;
        if (a < nt) {
          if (__popc((unsigned)(a & (int)b)) & 1) acc = acc - v[e]; else acc = acc + v[e];
        }
      }
    }
  } else {
    const int32_t* rows = P.perm + mc * P.nnz;
    const int8_t* sg = P.sign + mc * P.nnz;
    for (int t0 = 0; t0 < P.nnz; t0 += TERMS) {
      double v[TERMS];
      bool neg[TERMS];
#pragma unroll
      for (int e = 0; e < TERMS; ++e) {
        if (t0 + e < P.nnz) {
          v[e] = term(__ldg(rows + t0 + e));
          neg[e] = __ldg(sg + t0 + e) < 0;
        }
      }
#pragma unroll
      for (int e = 0; e < TERMS; ++e) {
        if (t0 + e < P.nnz) { if (neg[e]) acc = acc - v[e]; else acc = acc + v[e]; }
      }
    }
  }
  return acc * P.mscale;
}

// Entries of the CUR factors of W from a generator (I, J) of the pre-processed
// W' (the back-transform of a pre-processed CUR): with a right multiplier
// C = W'[:, J] and R = W[I, :]; with a left one the roles swap, C = W[:, J] and
// R = W'[I, :].  The nucleus is pinv(W'[I, J]) in both cases.
__device__ __forceinline__ double c_entry(const DevProblem& P, int64_t i, int64_t j) {
  return P.mside ? w_entry(P, i, j) : wp_entry(P, i, j);
}
__device__ __forceinline__ double r_entry(const DevProblem& P, int64_t i, int64_t j) {
  return P.mside ? wp_entry(P, i, j) : w_entry(P, i, j);
}

// ---------------------------------------------------------------------------
// Pivot candidates.  The magnitude of an FP64 value is compared through its bit
// pattern: for |x| not NaN, |x| < |y| exactly when (bits(x) & ~sign) <
// (bits(y) & ~sign) as unsigned integers, so the pivot searches run on the
// integer pipe instead of the (slow, long-latency) FP64 pipe.  key = abs bits
// + 1, key 0 = no candidate; NaN never becomes a candidate, as in a search
// written with "fabs(x) > best".  Order: larger key first, then lower column j,
// then lower row i.  The reduction also ORs a flags word.
// ---------------------------------------------------------------------------
constexpr unsigned long long ABS_MASK = 0x7fffffffffffffffull;
constexpr unsigned long long INF_BITS = 0x7ff0000000000000ull;

__device__ __forceinline__ unsigned long long mag_key(double x) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(x) & ABS_MASK;
  return a > INF_BITS ? 0ull : a + 1ull;
}
__device__ __forceinline__ bool bits_finite(double x) {
  return ((unsigned long long)__double_as_longlong(x) & INF_BITS) != INF_BITS;
}

struct Cand {
  unsigned long long key;
  int32_t i, j;
};

__device__ __forceinline__ Cand cand_none() { return Cand{0ull, 0x7fffffff, 0x7fffffff}; }

__device__ __forceinline__ bool cand_better(const Cand& a, const Cand& b) {
  return a.key > b.key || (a.key == b.key && (a.j < b.j || (a.j == b.j && a.i < b.i)));
}

__device__ __forceinline__ void cand_consider(Cand& best, unsigned long long key, int32_t i, int32_t j) {
  const Cand c{key, i, j};
  if (key != 0ull && cand_better(c, best)) best = c;
}

// cand_consider for a thread that visits its entries in ascending (j, i) order:
// an equal key never replaces the earlier entry, which is the lower (j, i), so a
// single 64-bit compare gives cand_consider's result.
__device__ __forceinline__ void cand_take(Cand& best, unsigned long long key, int32_t i, int32_t j) {
  if (key > best.key) best = Cand{key, i, j};
}

// cand_take with a 32-bit pre-test: an entry whose |v| has a smaller high word
// than the best's |v| cannot beat it, and most entries are rejected there.  bhi:
// the high word of the best's |v| bits (0 while there is none).  NaN passes the
// pre-test and is then refused (key 0), as by cand_take.
__device__ __forceinline__ void cand_take_val(Cand& best, unsigned& bhi, double v, int32_t i, int32_t j) {
  const unsigned h = (unsigned)__double2hiint(v) & 0x7fffffffu;
  if (h >= bhi) {
    const unsigned long long key = mag_key(v);
    if (key > best.key) { best = Cand{key, i, j}; bhi = h; }
  }
}

// cand_take_val restricted to keys above `floor`: start with bhi = the high word
// of the floor's |v| bits, and entries at or below the floor are never taken.
__device__ __forceinline__ void cand_take_above(Cand& best, unsigned& bhi, double v, int32_t i, int32_t j,
                                                unsigned long long floor) {
  const unsigned h = (unsigned)__double2hiint(v) & 0x7fffffffu;
  if (h >= bhi) {
    const unsigned long long key = mag_key(v);
    if (key > floor && key > best.key) { best = Cand{key, i, j}; bhi = h; }
  }
}

// Best candidate of the CTA (and the OR of the flags), returned to every thread.
struct CandRed {
  Cand c[33];
  unsigned long long f[33];
};

__device__ __forceinline__ Cand block_best(Cand c, unsigned long long& flags, CandRed* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    Cand o;
    o.key = __shfl_down_sync(0xffffffffu, c.key, off);
    o.i = __shfl_down_sync(0xffffffffu, c.i, off);
    o.j = __shfl_down_sync(0xffffffffu, c.j, off);
    flags |= __shfl_down_sync(0xffffffffu, flags, off);
    if (cand_better(o, c)) c = o;
  }
  if (lane == 0) { red->c[warp] = c; red->f[warp] = flags; }
  __syncthreads();
  if (warp == 0) {
    const bool act = lane < (int)(blockDim.x >> 5);
    Cand d = act ? red->c[lane] : cand_none();
    unsigned long long g = act ? red->f[lane] : 0ull;
    for (int off = 16; off > 0; off >>= 1) {
      Cand o;
      o.key = __shfl_down_sync(0xffffffffu, d.key, off);
      o.i = __shfl_down_sync(0xffffffffu, d.i, off);
      o.j = __shfl_down_sync(0xffffffffu, d.j, off);
      g |= __shfl_down_sync(0xffffffffu, g, off);
      if (cand_better(o, d)) d = o;
    }
    if (lane == 0) { red->c[32] = d; red->f[32] = g; }
  }
  __syncthreads();
  const Cand r = red->c[32];
  flags = red->f[32];
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
// Exchange among the CTAs of one maxvol search.  Every CTA reduces its threads'
// candidates, posts its best candidate together with the current values of that
// candidate's column, reads all posts and keeps the best one (the order above is
// total, so all CTAs agree) with its column.  Results land in shared memory:
//   win  -- the winning candidate,  x[0..k) -- its column,  flags -- OR of flags.
// Two CTA barriers per exchange: warp results -> warp 0 does the rest (one when
// the caller lets warp 0 finish its step first: exchange<false>).
// Returns false (in every thread) if a wait expired or another CTA aborted.
// ---------------------------------------------------------------------------
__device__ __forceinline__ Cand warp_best(Cand c) {
  for (int off = 16; off > 0; off >>= 1) {
    Cand o;
    o.key = __shfl_xor_sync(0xffffffffu, c.key, off);
    o.i = __shfl_xor_sync(0xffffffffu, c.i, off);
    o.j = __shfl_xor_sync(0xffffffffu, c.j, off);
    if (cand_better(o, c)) c = o;
  }
  return c;       // every lane holds the warp's best
}

struct ExchangeOut {
  Cand* win;
  double* x;
  unsigned long long* flags;
  int* fail;
  CandRed* red;
};

// warp_best for candidates of one CTA's columns (q0 <= j < q0 + 2^26, 0 <= i <
// 64): the key's high word, then its low word, then the position (j - q0) * 64
// + i -- the order of cand_better -- each reduced by one warp instruction.
__device__ __forceinline__ Cand warp_best_local(Cand c, int64_t q0) {
  const unsigned hi = (unsigned)(c.key >> 32), lo = (unsigned)c.key;
  const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
  const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
  const unsigned pos = (c.key != 0ull && hi == mhi && lo == mlo) ? (unsigned)((c.j - q0) * 64 + c.i) : 0xffffffffu;
  const unsigned mpos = __reduce_min_sync(0xffffffffu, pos);
  if (mpos == 0xffffffffu) return cand_none();
  return Cand{((unsigned long long)mhi << 32) | mlo, (int32_t)(mpos & 63u), (int32_t)(q0 + (mpos >> 6))};
}

// First half, common to all groups: the CTA's best candidate (its columns start
// at q0), in warp 0.
__device__ __forceinline__ Cand cta_best_in_warp0(Cand mine, CandRed* red, int64_t q0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  mine = warp_best_local(mine, q0);
  if (lane == 0) red->c[warp] = mine;
  __syncthreads();
  Cand d = cand_none();
  if (warp == 0) {
    if (lane < (int)(blockDim.x >> 5)) d = red->c[lane];
    d = warp_best_local(d, q0);
  }
  return d;       // meaningful in warp 0 only
}

// A single CTA: nothing to exchange.
//
// exchange<false> skips the closing CTA barrier: the results are then visible to
// warp 0 only (after a warp barrier), which can finish the step's serial work on
// them before the caller's own CTA barrier; after that barrier failed() tells
// every thread whether the exchange gave up.
struct SoloGroup {
  __device__ __forceinline__ int rank() const { return 0; }
  template <bool kBar = true>
  __device__ __forceinline__ bool exchange(unsigned long long /*seq*/, Cand mine, unsigned long long myflags,
                                           const double* M, int ldm, int64_t q0, int k, int /*owner_chunk*/,
                                           const ExchangeOut& o) const {
    const Cand d = cta_best_in_warp0(mine, o.red, q0);
    if (threadIdx.x < 32) {
      if (threadIdx.x == 0) { *o.win = d; *o.flags = myflags; }
      if (d.key != 0ull)
        for (int a = threadIdx.x; a < k; a += 32) o.x[a] = M[(int64_t)a * ldm + (d.j - q0)];
    }
    if (kBar) __syncthreads();
    else __syncwarp();
    return true;
  }
  __device__ __forceinline__ bool failed(const ExchangeOut&) const { return false; }
};

// All CTAs of a cooperative grid, through double-buffered slots in global memory.
// A slot is (key, (i, j), flags, tag, column); one thread writes it and then the
// tag with a release store, readers poll tags with acquire loads: one round is
// one post and one read of every slot (no atomics).  Round r uses buffer r & 1:
// a CTA can only post round r + 2 after every CTA posted round r + 1, i.e. after
// every CTA finished reading round r.
struct GridGroup {
  double* slots;             // [2][nblk][SLOT]
  unsigned int* abort;       // 0, or the status of the CTA that gave up
  int nblk;
  int first = 0;             // the group is CTAs first .. first + nblk - 1 of the grid

  __device__ __forceinline__ int rank() const { return (int)blockIdx.x - first; }

  __device__ __forceinline__ bool failed(const ExchangeOut& o) const { return *o.fail != 0; }

  template <bool kBar = true>
  __device__ bool exchange(unsigned long long seq, Cand mine, unsigned long long myflags, const double* M, int ldm,
                           int64_t q0, int k, int owner_chunk, const ExchangeOut& o) const {
    const Cand d = cta_best_in_warp0(mine, o.red, q0);
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
      double* buf = slots + (size_t)(seq & 1ull) * nblk * SLOT;
      {
        // post: the warp writes the column (a lane per entry), then lane 0 the
        // candidate and, after a fence and the warp barrier, the tag (release)
        double* me = buf + (size_t)rank() * SLOT;
        unsigned long long* mu = reinterpret_cast<unsigned long long*>(me);
        if (d.key != 0ull)
          for (int a = lane; a < k; a += 32) me[4 + a] = M[(int64_t)a * ldm + (d.j - q0)];
        if (lane == 0) {
          mu[0] = d.key;
          reinterpret_cast<int2*>(me + 1)[0] = make_int2(d.i, d.j);
          mu[2] = myflags;
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release_u64(mu + 3, seq + 1ull);       // orders the slot before the tag
      }
      Cand best = cand_none();
      unsigned long long f = 0;
      int fail = 0;
      // wait for all of this lane's slots (r = lane, lane + 32, ...) at once: their
      // tags are polled together, so one round trip serves them all
      constexpr int PER_LANE = 8;                   // slots per lane: nblk <= 256
      unsigned ready = 0u, need = 0u;
      for (int q = 0; q < PER_LANE; ++q)
        if (lane + 32 * q < nblk) need |= 1u << q;
      {
        unsigned long long t0 = 0;
        unsigned spins = 0;
        while (ready != need) {
#pragma unroll
          for (int q = 0; q < PER_LANE; ++q) {
            const int r = lane + 32 * q;
            if (((need & ~ready) >> q) & 1u) {
              const unsigned long long* sl = reinterpret_cast<const unsigned long long*>(buf + (size_t)r * SLOT);
              if (ld_acquire_u64(sl + 3) == seq + 1ull) ready |= 1u << q;
            }
          }
          if (ready != need && (++spins & 63u) == 0u) {
            if (ld_relaxed_u32(abort) != 0u) { fail = 1; break; }
            const unsigned long long now = globaltimer_ns();
            if (t0 == 0) t0 = now;
            else if ((double)(now - t0) > WAIT_NS) { fail = 2; break; }
          }
        }
      }
      if (!fail) {
#pragma unroll
        for (int q = 0; q < PER_LANE; ++q) {
          const int r = lane + 32 * q;
          if (r >= nblk) continue;
          const unsigned long long* sl = reinterpret_cast<const unsigned long long*>(buf + (size_t)r * SLOT);
          Cand c;
          c.key = __ldcg(sl);
          const int2 ij = __ldcg(reinterpret_cast<const int2*>(sl + 1));
          c.i = ij.x; c.j = ij.y;
          f |= __ldcg(sl + 2);
          if (cand_better(c, best)) best = c;
        }
      }
      if (fail == 2) atomicCAS(abort, 0u, (unsigned)LRA_ERR_TIMEOUT);
      fail = __any_sync(0xffffffffu, fail != 0);
      best = warp_best(best);
      for (int off = 16; off > 0; off >>= 1) f |= __shfl_xor_sync(0xffffffffu, f, off);
      if (!fail && best.key != 0ull) {
        const double* ws = buf + (size_t)(best.j / owner_chunk) * SLOT;
        for (int a = lane; a < k; a += 32) o.x[a] = __ldcg(ws + 4 + a);
      }
      if (lane == 0) { *o.win = best; *o.flags = f; *o.fail = fail; }
    }
    if (!kBar) {
      __syncwarp();
      return true;
    }
    __syncthreads();
    return *o.fail == 0;
  }
};

}  // namespace lra
