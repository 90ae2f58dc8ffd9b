// lra_apply.cu -- products with a CUR triple and the sampled a-posteriori
// residual, FP64.
//
// cur_apply:  Y = C (U (R X))   (paper: FMM / HSS stage (iii), multiplication
//   with the low-rank generators).  Stage 1 splits the n-long contraction R X
//   over CTAs (partial k x nrhs sums in the workspace), stage 2 adds the
//   partials in CTA order and applies U, stage 3 forms Y row by row.  All three
//   stages stream their operands once: the product is HBM-bound (about
//   k nrhs / (k + nrhs) flops per byte).
// residual_sample:  E[Q,S] = W[Q,S] - (C U)[Q,:] R[:,S] and its statistics
//   (paper: Section "Superfast a posteriori error estimation for LRA of a matrix
//   filled with i.i.d. values of a single variable").
#include <algorithm>
#include <type_traits>

#include <cuda_bf16.h>

#include "lra_internal.h"
#include "lra_profile.h"

namespace lra {

constexpr int APPLY_ROWS_PER_CTA = 512;

// ---------------------------------------------------------------------------
// Stored factors in FP32 or BF16 (lra_cur_apply with dtype LRA_F32 / LRA_BF16).
// The factors are streamed from HBM once at 4 or 2 bytes an entry; every
// product is taken in FP32 and accumulated in FP32 over short runs (a tile of
// LP_TJ columns of R, one row of C), the runs in FP64.  The FP64 vector operand
// (X, then T2 = U T1) is split into an FP32 head and an FP32 tail and both go
// through the same stored entries: one refinement step, after which the error
// is the factors' storage rounding plus the FP32 accumulation.
// ---------------------------------------------------------------------------
constexpr int LP_TJ = 512;                 // columns of R per tile (16 per lane)
constexpr int LP_MAX_NRHS = 64;
constexpr int LP_THREADS = 256;

__device__ __forceinline__ float lp_load(const float* p) { return __ldg(p); }
__device__ __forceinline__ float lp_load(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }

// Four consecutive entries (16-byte aligned for FP32, 8-byte for BF16) as floats.
__device__ __forceinline__ void lp_load4(const float* p, float v[4]) {
  const float4 q = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void lp_load4(const __nv_bfloat16* p, float v[4]) {
  const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
  const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&q.x);
  const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&q.y);
  const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
  v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
}

// Stage 2 on one CTA: T1 = sum_b partial[b] (a warp per entry of T1: lane l
// adds the partials b = l, l + 32, ... in order, then a fixed butterfly -- the
// same order for a given number of partials), then T2 = U T1 (a thread per entry,
// an ascending fma chain).  Called by every thread of the CTA.
__device__ inline void fold_and_apply_u(const double* __restrict__ partial, int nb, const double* __restrict__ U,
                                        int k, int nrhs, double* __restrict__ T1, double* __restrict__ T2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int it = warp; it < k * nrhs; it += nw) {
    double s = 0.0;
#pragma unroll 8
    for (int b = lane; b < nb; b += 32) s = s + __ldcg(partial + (size_t)b * k * nrhs + it);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) T1[it] = s;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < k * nrhs; it += blockDim.x) {
    const int a = it / nrhs, c = it - a * nrhs;
    double s = 0.0;
#pragma unroll 8
    for (int b = 0; b < k; ++b) s = fma(__ldg(U + a * k + b), __ldcg(T1 + b * nrhs + c), s);
    T2[it] = s;
  }
}

// Stage 1: partial[cta][a][c] = sum over this CTA's tiles of R[a][j] X[j][c]
// (persistent CTAs over the tiles of LP_TJ columns).  Per tile and group of up
// to 16 right-hand sides: X's entries in shared memory (FP32 head and tail for
// FP32 / BF16 storage, column c of the group contiguous in j); warp w takes rows
// a = w, w + 8, ..., two at a time, lane l the 16 entries j0 + 128 g + 4 l + e
// (g, e < 4) of each (vector loads, each covering 128 consecutive entries of
// the row across the warp); a lane's 16 products and the warp's butterfly in
// the product precision, added to the row's FP64 sum.  vec: R's rows allow the vector loads.
// Dynamic shared memory: lp_rx_smem(k, nrhs, element size of the tile).
__host__ __device__ inline size_t lp_rx_smem(int k, int nrhs, size_t esz) {
  const int cg = nrhs < 16 ? nrhs : 16;
  return esz * (esz == 8 ? 1 : 2) * (size_t)LP_TJ * cg + sizeof(double) * (size_t)k * nrhs;
}

__device__ __forceinline__ double lp_load(const double* p) { return __ldg(p); }
__device__ __forceinline__ void lp_load4(const double* p, double v[4]) {
  const double2 q0 = __ldg(reinterpret_cast<const double2*>(p));
  const double2 q1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
  v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

template <class T>
__global__ void __launch_bounds__(LP_THREADS) apply_rx_lp_kernel(const T* __restrict__ R, const double* __restrict__ X,
                                                                  int64_t n, int k, int nrhs, int vec,
                                                                  double* __restrict__ partial, const double* U,
                                                                  double* __restrict__ T1, double* __restrict__ T2,
                                                                  unsigned int* done) {
  constexpr bool kF64 = std::is_same<T, double>::value;
  constexpr int RQ = 2;                    // rows of a warp whose loads are in flight together
  using A = typename std::conditional<kF64, double, float>::type;
  extern __shared__ __align__(16) unsigned char lp_smem[];
  const int cg = nrhs < 16 ? nrhs : 16;
  A* xh = reinterpret_cast<A*>(lp_smem);                                  // [cg][LP_TJ]
  A* xl = kF64 ? xh : xh + (size_t)cg * LP_TJ;                            // [cg][LP_TJ] (FP32 tail)
  double* acc = reinterpret_cast<double*>(xl + (kF64 ? (size_t)cg * LP_TJ : (size_t)cg * LP_TJ));   // [k][nrhs]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int it = threadIdx.x; it < k * nrhs; it += blockDim.x) acc[it] = 0.0;
  const int64_t ntiles = (n + LP_TJ - 1) / LP_TJ;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t j0 = tile * LP_TJ;
    const int tj = (int)min((int64_t)LP_TJ, n - j0);
    for (int c0 = 0; c0 < nrhs; c0 += 16) {
      const int cn = min(16, nrhs - c0);
      __syncthreads();
      for (int it = threadIdx.x; it < LP_TJ * cn; it += blockDim.x) {
        const int j = it / cn, c = it - j * cn;
        const double v = (j < tj) ? X[(j0 + j) * nrhs + c0 + c] : 0.0;
        if (kF64) {
          xh[c * LP_TJ + j] = (A)v;
        } else {
          const float h = __double2float_rn(v);
          xh[c * LP_TJ + j] = h;
          xl[c * LP_TJ + j] = __double2float_rn(v - (double)h);
        }
      }
      __syncthreads();
      for (int ap = warp; RQ * ap < k; ap += nw) {
        // lane l: entries 4 l + 128 g + e (g < 4, e < 4): each group's loads cover
        // 128 consecutive entries of the row, and the float4 reads of X's tile are
        // conflict-free
        A r[RQ][16];
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
          const int a = RQ * ap + q;
          const T* row = R + (int64_t)min(a, k - 1) * n + j0;
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const int jj = 128 * g + 4 * lane;
            if (a < k && vec && jj + 3 < tj) lp_load4(row + jj, &r[q][4 * g]);
            else
#pragma unroll
              for (int e = 0; e < 4; ++e) r[q][4 * g + e] = (a < k && jj + e < tj) ? (A)lp_load(row + jj + e) : (A)0;
          }
        }
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
          const int a = RQ * ap + q;
          if (a >= k) break;
          for (int c = 0; c < cn; ++c) {
            A sh = 0, sl = 0;
#pragma unroll
            for (int g = 0; g < 4; ++g) {
              const A* xr = xh + c * LP_TJ + 128 * g + 4 * lane;
              const A* xt = xl + c * LP_TJ + 128 * g + 4 * lane;
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                sh = fma(r[q][4 * g + e], xr[e], sh);
                if (!kF64) sl = fma(r[q][4 * g + e], xt[e], sl);
              }
            }
            for (int off = 16; off > 0; off >>= 1) {
              sh += __shfl_xor_sync(0xffffffffu, sh, off);
              if (!kF64) sl += __shfl_xor_sync(0xffffffffu, sl, off);
            }
            if (lane == 0) acc[a * nrhs + c0 + c] += kF64 ? (double)sh : (double)sh + (double)sl;
          }
        }
      }
    }
  }
  __syncthreads();
  for (int it = threadIdx.x; it < k * nrhs; it += blockDim.x) partial[(size_t)blockIdx.x * k * nrhs + it] = acc[it];
  // stage 2 in the last CTA to finish (its partials and everyone's are visible
  // after the fences); *done must be 0 at launch and is left at 0
  __threadfence();
  __shared__ unsigned int s_last;
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(done, 1u) == gridDim.x - 1) ? 1u : 0u;
  __syncthreads();
  if (s_last) {
    __threadfence();
    fold_and_apply_u(partial, gridDim.x, U, k, nrhs, T1, T2);
    if (threadIdx.x == 0) *done = 0u;
  }
}

// Stage 3: Y[i][c] = sum_a C[i][a] T2[a][c], a thread per row: the row's k
// stored entries in registers, T2 as FP32 head / tail in shared memory, each
// output an FP32 sum over k products of the head plus one of the tail.
template <class T, int KC>
__global__ void __launch_bounds__(LP_THREADS) apply_c_lp_kernel(const T* __restrict__ C, const double* __restrict__ T2,
                                                                 int64_t m, int k, int nrhs, double* __restrict__ Y) {
  __shared__ float th[KMAX * LP_MAX_NRHS], tl[KMAX * LP_MAX_NRHS];
  for (int it = threadIdx.x; it < k * nrhs; it += blockDim.x) {
    const double v = T2[it];
    const float h = __double2float_rn(v);
    th[it] = h;
    tl[it] = __double2float_rn(v - (double)h);
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    float cv[KC];
    const T* row = C + i * k;
#pragma unroll
    for (int a = 0; a < KC; ++a) cv[a] = (a < k) ? lp_load(row + a) : 0.f;
    for (int c = 0; c < nrhs; ++c) {
      float sh = 0.f, sl = 0.f;
#pragma unroll
      for (int a = 0; a < KC; ++a)
        if (a < k) { sh = fmaf(cv[a], th[a * nrhs + c], sh); sl = fmaf(cv[a], tl[a * nrhs + c], sl); }
      Y[i * nrhs + c] = (double)sh + (double)sl;
    }
  }
}

// Stage 1: partial[b][a][c] = sum over this CTA's rows j of R[a][j] X[j][c].
__global__ void __launch_bounds__(NT) apply_rx_kernel(const double* __restrict__ R, const double* __restrict__ X,
                                                      int64_t n, int k, int nrhs, double* __restrict__ partial) {
  const int64_t j0 = (int64_t)blockIdx.x * APPLY_ROWS_PER_CTA;
  const int64_t j1 = min(n, j0 + APPLY_ROWS_PER_CTA);
  for (int it = threadIdx.x; it < k * nrhs; it += blockDim.x) {
    const int a = it / nrhs, c = it - a * nrhs;
    double s = 0.0;
    for (int64_t j = j0; j < j1; ++j) s = fma(__ldg(R + (int64_t)a * n + j), __ldg(X + j * nrhs + c), s);
    partial[((size_t)blockIdx.x * k + a) * nrhs + c] = s;
  }
}

// Stage 2 as a kernel of its own (the untiled FP64 path).
__global__ void __launch_bounds__(NT) apply_u_kernel(const double* __restrict__ partial, int nb, const double* U,
                                                     int k, int nrhs, double* __restrict__ T1,
                                                     double* __restrict__ T2) {
  fold_and_apply_u(partial, nb, U, k, nrhs, T1, T2);
}

// Stage 3: Y[i][c] = sum_a C[i][a] T2[a][c].
__global__ void __launch_bounds__(NT) apply_c_kernel(const double* __restrict__ C, const double* __restrict__ T2,
                                                     int64_t m, int k, int nrhs, double* __restrict__ Y) {
  const int64_t total = m * nrhs;
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < total; it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = it / nrhs;
    const int c = (int)(it - i * nrhs);
    double s = 0.0;
    for (int a = 0; a < k; ++a) s = fma(__ldg(C + i * k + a), __ldg(T2 + a * nrhs + c), s);
    Y[it] = s;
  }
}

// Stage 3, vector form (k a multiple of the entries in 16 bytes, 16-byte
// aligned rows, nrhs <= LP_MAX_NRHS): a row of C is read by L lanes, one
// 16-byte vector each (a warp reads 32 / L consecutive rows, contiguous in
// memory); each lane multiplies its VEC entries by T2, the L lanes' partial sums
// meet in a fixed butterfly.  FP64 storage: FP64 products and sums.  FP32 /
// BF16 storage: FP32 products and sums of T2's FP32 head and tail (the
// refinement step), added in FP64.
template <class T> struct Vec16;
template <> struct Vec16<double> {
  static constexpr int N = 2;
  __device__ static void load(const double* p, double v[2]) {
    const double2 q = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = q.x; v[1] = q.y;
  }
};
template <> struct Vec16<float> {
  static constexpr int N = 4;
  __device__ static void load(const float* p, float v[4]) { lp_load4(p, v); }
};
template <> struct Vec16<__nv_bfloat16> {
  static constexpr int N = 8;
  __device__ static void load(const __nv_bfloat16* p, float v[8]) {
    const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
    const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[e]));
      v[2 * e] = f.x; v[2 * e + 1] = f.y;
    }
  }
};

template <class T>
__global__ void __launch_bounds__(LP_THREADS) apply_c_vec_kernel(const T* __restrict__ C, const double* __restrict__ T2,
                                                                  int64_t m, int k, int nrhs, int L,
                                                                  double* __restrict__ Y) {
  constexpr int VEC = Vec16<T>::N;
  constexpr bool kF64 = std::is_same<T, double>::value;
  __shared__ __align__(16) unsigned char tbuf[sizeof(double) * KMAX * LP_MAX_NRHS];
  double* t64 = reinterpret_cast<double*>(tbuf);             // FP64 storage: T2
  float* th = reinterpret_cast<float*>(tbuf);                // otherwise: T2's head
  float* tl = th + (size_t)k * nrhs;                         //            and tail
  for (int it = threadIdx.x; it < k * nrhs; it += blockDim.x) {
    const double v = T2[it];
    if (kF64) t64[it] = v;
    else {
      const float h = __double2float_rn(v);
      th[it] = h;
      tl[it] = __double2float_rn(v - (double)h);
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, sub = lane % L, rpw = 32 / L;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int a0 = sub * VEC;
  // UNR row groups of rpw rows each: their loads are in flight together, and
  // their UNR * rpw results are gathered into lanes 0 .. UNR * rpw - 1 (row
  // u * rpw + r from lane r * L of group u), so that the FP64 combination of
  // head and tail and the store of Y take one warp instruction for all of them
  constexpr int UNR = 4;
  const int gu = lane / rpw, gr = lane % rpw;            // the gathered row of this lane
  for (int64_t g0 = gw * UNR; g0 * rpw < m; g0 += warps * UNR) {
    typename std::conditional<kF64, double, float>::type vv[UNR][VEC];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const int64_t i = (g0 + u) * rpw + lane / L;
      if (i < m && a0 < k) Vec16<T>::load(C + i * k + a0, vv[u]);
      else
#pragma unroll
        for (int e = 0; e < VEC; ++e) vv[u][e] = 0;
    }
    const int64_t iout = g0 * rpw + lane;                // rows g0*rpw .. +UNR*rpw-1, one per gathering lane
    for (int c = 0; c < nrhs; ++c) {
      if (kF64) {
        double got = 0.0;
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          double sacc = 0.0;
#pragma unroll
          for (int e = 0; e < VEC; ++e) sacc = fma((double)vv[u][e], t64[min(a0 + e, k - 1) * nrhs + c], sacc);
          for (int off = L >> 1; off > 0; off >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, off);
          const double v = __shfl_sync(0xffffffffu, sacc, gr * L);
          if (gu == u) got = v;
        }
        if (lane < UNR * rpw && iout < m) Y[iout * nrhs + c] = got;
      } else {
        float gh = 0.f, gl = 0.f;
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          float sh = 0.f, sl = 0.f;
#pragma unroll
          for (int e = 0; e < VEC; ++e) {
            const int ae = min(a0 + e, k - 1);                 // lanes past the row's end hold zeros
            sh = fmaf((float)vv[u][e], th[ae * nrhs + c], sh);
            sl = fmaf((float)vv[u][e], tl[ae * nrhs + c], sl);
          }
          for (int off = L >> 1; off > 0; off >>= 1) {
            sh += __shfl_xor_sync(0xffffffffu, sh, off);
            sl += __shfl_xor_sync(0xffffffffu, sl, off);
          }
          const float vh = __shfl_sync(0xffffffffu, sh, gr * L), vl = __shfl_sync(0xffffffffu, sl, gr * L);
          if (gu == u) { gh = vh; gl = vl; }
        }
        if (lane < UNR * rpw && iout < m) Y[iout * nrhs + c] = (double)gh + (double)gl;
      }
    }
  }
}

// Lanes per row of the vector form of stage 3 (a power of two >= k / VEC), or
// 0 when the rows do not allow it.
template <class T>
static int vec_lanes(const T* C, int k, int nrhs) {
  constexpr int VEC = Vec16<T>::N;
  if (nrhs > LP_MAX_NRHS || k % VEC != 0 || (reinterpret_cast<uintptr_t>(C) & 15u) != 0) return 0;
  int L = 4;                               // at least 4 lanes a row: a warp's 4 groups gather into <= 32 lanes
  while (L * VEC < k) L *= 2;
  return L <= 32 ? L : 0;
}

// Residual: rows of C U at the sampled rows, then E and its statistics.
// A sample index outside 0 <= Q[a] < m, 0 <= S[c] < n is never dereferenced:
// the kernels set *bad instead, and the statistics come out NaN.
__global__ void __launch_bounds__(NT) resid_cu_kernel(const double* __restrict__ C, const double* __restrict__ U,
                                                      const int32_t* __restrict__ Q, int q, int k, int64_t m,
                                                      double* __restrict__ CU, int* bad) {
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < (int64_t)q * k;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(it / k), b = (int)(it - (int64_t)a * k);
    const int64_t row = Q[a];
    if (row < 0 || row >= m) {
      atomicOr(bad, 1);
      CU[it] = __longlong_as_double(0x7ff8000000000000ll);
      continue;
    }
    double t = 0.0;
    for (int d = 0; d < k; ++d) t = fma(C[row * k + d], U[d * k + b], t);
    CU[it] = t;
  }
}

__global__ void __launch_bounds__(NT) resid_e_kernel(DevProblem P, const double* __restrict__ CU,
                                                     const double* __restrict__ R, const int32_t* __restrict__ Q,
                                                     const int32_t* __restrict__ S, int q, int s, int k,
                                                     double* __restrict__ E, double* __restrict__ W2, int* bad) {
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < (int64_t)q * s;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(it / s), c = (int)(it - (int64_t)a * s);
    const int64_t col = S[c], row = Q[a];
    if (row < 0 || row >= P.m || col < 0 || col >= P.n) {
      atomicOr(bad, 1);
      E[it] = __longlong_as_double(0x7ff8000000000000ll);
      W2[it] = 0.0;
      continue;
    }
    double t = 0.0;
    for (int b = 0; b < k; ++b) t = fma(CU[(int64_t)a * k + b], R[(int64_t)b * P.n + col], t);
    const double w = w_entry(P, row, col);
    E[it] = w - t;
    W2[it] = w * w;
  }
}

// Fixed-order block sum of per-thread values (deterministic for a fixed blockDim).
__device__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += red[w];
    red[32] = r;
  }
  __syncthreads();
  r = red[32];
  __syncthreads();
  return r;
}

__device__ double block_max(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
    red[32] = r;
  }
  __syncthreads();
  double r = red[32];
  __syncthreads();
  return r;
}

// Sample statistics over K = q s errors in three grid passes: per-CTA partial
// sums (sum e, sum |e|, max |e|, sum e^2, sum w^2), then each CTA folds the
// partial sums into the mean and adds its share of sum (e - mean)^2, then one
// CTA folds the partials in CTA order into the five statistics.
constexpr int RESID_MAX_PARTS = 1024;

__global__ void __launch_bounds__(NT) resid_part_kernel(const double* __restrict__ E, const double* __restrict__ W2,
                                                        int64_t K, double* __restrict__ part) {
  __shared__ double red[33];
  double s = 0.0, sa = 0.0, mx = 0.0, se2 = 0.0, sw2 = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < K; t += (int64_t)gridDim.x * blockDim.x) {
    const double e = E[t];
    s += e;
    sa += fabs(e);
    mx = fmax(mx, fabs(e));
    se2 = fma(e, e, se2);
    sw2 += W2[t];
  }
  s = block_sum(s, red);
  sa = block_sum(sa, red);
  mx = block_max(mx, red);
  se2 = block_sum(se2, red);
  sw2 = block_sum(sw2, red);
  if (threadIdx.x == 0) {
    double* o = part + 6 * (size_t)blockIdx.x;
    o[0] = s; o[1] = sa; o[2] = mx; o[3] = se2; o[4] = sw2;
  }
}

__global__ void __launch_bounds__(NT) resid_var_kernel(const double* __restrict__ E, int64_t K,
                                                       double* __restrict__ part) {
  __shared__ double red[33];
  __shared__ double s_mean;
  const int nparts = gridDim.x;
  if (threadIdx.x < 32) {          // every CTA folds the partial sums in the same order
    double s = 0.0;
    for (int b = threadIdx.x; b < nparts; b += 32) s += part[6 * (size_t)b];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) s_mean = s / (double)K;
  }
  __syncthreads();
  const double mean = s_mean;
  double v = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < K; t += (int64_t)gridDim.x * blockDim.x) {
    const double d = E[t] - mean;
    v = fma(d, d, v);
  }
  v = block_sum(v, red);
  if (threadIdx.x == 0) part[6 * (size_t)blockIdx.x + 5] = v;
}

__global__ void resid_final_kernel(const double* __restrict__ part, int nparts, int64_t K, const int* bad,
                                   double* __restrict__ stats) {
  // one warp: lane l folds the partials l, l + 32, ..., then a butterfly
  const int lane = threadIdx.x;
  double s = 0.0, sa = 0.0, mx = 0.0, se2 = 0.0, sw2 = 0.0, v = 0.0;
  for (int b = lane; b < nparts; b += 32) {
    const double* o = part + 6 * (size_t)b;
    s += o[0]; sa += o[1]; mx = fmax(mx, o[2]); se2 += o[3]; sw2 += o[4]; v += o[5];
  }
  for (int off = 16; off > 0; off >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, off);
    sa += __shfl_xor_sync(0xffffffffu, sa, off);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    se2 += __shfl_xor_sync(0xffffffffu, se2, off);
    sw2 += __shfl_xor_sync(0xffffffffu, sw2, off);
    v += __shfl_xor_sync(0xffffffffu, v, off);
  }
  if (lane == 0) {
    stats[0] = s / (double)K;
    stats[1] = v / (double)K;
    stats[2] = sa / (double)K;
    stats[3] = mx;
    stats[4] = sw2 > 0.0 ? sqrt(se2) / sqrt(sw2) : 0.0;
    if (*bad)
      for (int e = 0; e < 5; ++e) stats[e] = __longlong_as_double(0x7ff8000000000000ll);
  }
}

}  // namespace lra

using namespace lra;

namespace lra {
static size_t apply_ws_bytes(int64_t n, int32_t k, int32_t nrhs) {
  const int64_t nb = (n + APPLY_ROWS_PER_CTA - 1) / APPLY_ROWS_PER_CTA;
  return align_up(sizeof(double) * (size_t)nb * k * nrhs, 256) + 2 * align_up(sizeof(double) * (size_t)k * nrhs, 256) +
         256;   // the tiled stage 1's completion counter
}

// The low-precision path's persistent grid of stage 1 has a fixed number of
// CTAs (LP_PARTS, at most), whose FP64 partial sums the FP64 stage 2 folds.
constexpr int LP_PARTS = 2048;
static size_t apply_lp_ws_bytes(int32_t k, int32_t nrhs) {
  return align_up(sizeof(double) * (size_t)LP_PARTS * k * nrhs, 256) + 2 * align_up(sizeof(double) * (size_t)k * nrhs, 256) +
         256;   // the tiled stage 1's completion counter
}

template <class T>
static void launch_lp(const T* C, const double* U, const T* R, int64_t m, int64_t n, int k, const double* X, int nrhs,
                      double* Y, int parts, int grid3, double* partial, double* T1, double* T2, unsigned int* done,
                      cudaStream_t stream) {
  const size_t esz = sizeof(T);
  const int vec = ((n * esz) % 16 == 0 && (reinterpret_cast<uintptr_t>(R) & 15u) == 0) ? 1 : 0;
  {
    const size_t smem = lp_rx_smem(k, nrhs, std::is_same<T, double>::value ? 8 : 4);
    cudaFuncSetAttribute(apply_rx_lp_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    LaunchScope ls(stream, "apply_rx_lp_kernel");
    apply_rx_lp_kernel<T><<<parts, LP_THREADS, smem, stream>>>(R, X, n, k, nrhs, vec, partial, U, T1, T2, done);
  }
  const int L = vec_lanes(C, k, nrhs);
  if (L > 0) {
    const int64_t rows_per_cta = (int64_t)(LP_THREADS / 32) * (32 / L) * 4;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((m + rows_per_cta - 1) / rows_per_cta,
                                                                 (int64_t)grid3));
    LaunchScope ls(stream, "apply_c_lp_kernel");
    apply_c_vec_kernel<T><<<grid, LP_THREADS, 0, stream>>>(C, T2, m, k, nrhs, L, Y);
    return;
  }
  LaunchScope ls(stream, "apply_c_lp_kernel");
  if (k <= 16) apply_c_lp_kernel<T, 16><<<grid3, LP_THREADS, 0, stream>>>(C, T2, m, k, nrhs, Y);
  else if (k <= 32) apply_c_lp_kernel<T, 32><<<grid3, LP_THREADS, 0, stream>>>(C, T2, m, k, nrhs, Y);
  else apply_c_lp_kernel<T, 64><<<grid3, LP_THREADS, 0, stream>>>(C, T2, m, k, nrhs, Y);
}

static lra_status apply_lp(const void* C, const double* U, const void* R, int64_t m, int64_t n, int32_t k,
                           const double* X, int32_t nrhs, double* Y, int32_t dtype, void* workspace,
                           size_t workspace_bytes, cudaStream_t stream) {
  if (nrhs > LP_MAX_NRHS) return LRA_ERR_INVALID_ARG;
  const size_t need = apply_lp_ws_bytes(k, nrhs);
  if (workspace == nullptr || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return LRA_ERR_WORKSPACE;
  DeviceInfo dev;
  lra_status st = current_device_info(&dev);
  if (st != LRA_OK) return st;
  const int64_t ntiles = (n + LP_TJ - 1) / LP_TJ;
  int occ = 1;
  if (dtype == LRA_F32)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, apply_rx_lp_kernel<float>, LP_THREADS, lp_rx_smem(k, nrhs, 4));
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, apply_rx_lp_kernel<__nv_bfloat16>, LP_THREADS,
                                                  lp_rx_smem(k, nrhs, 4));
  // at most two CTAs an SM: fewer partials for the last CTA to fold
  const int parts = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, std::min(LP_PARTS, dev.sms * std::min(std::max(occ, 1), 2))));
  const int grid3 = (int)std::max<int64_t>(1, std::min<int64_t>((m + LP_THREADS - 1) / LP_THREADS, (int64_t)dev.sms * 7));
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  double* partial = reinterpret_cast<double*>(ws);
  double* T1 = reinterpret_cast<double*>(ws + align_up(sizeof(double) * (size_t)LP_PARTS * k * nrhs, 256));
  double* T2 = T1 + align_up(sizeof(double) * (size_t)k * nrhs, 256) / sizeof(double);
  unsigned int* done = reinterpret_cast<unsigned int*>(T2 + align_up(sizeof(double) * (size_t)k * nrhs, 256) / 8);
  LRA_CUDA_TRY(cudaMemsetAsync(done, 0, sizeof(unsigned int), stream));
  if (dtype == LRA_F32)
    launch_lp(static_cast<const float*>(C), U, static_cast<const float*>(R), m, n, k, X, nrhs, Y, parts, grid3,
              partial, T1, T2, done, stream);
  else
    launch_lp(static_cast<const __nv_bfloat16*>(C), U, static_cast<const __nv_bfloat16*>(R), m, n, k, X, nrhs, Y,
              parts, grid3, partial, T1, T2, done, stream);
  return cuda_status(cudaGetLastError());
}
}  // namespace lra

extern "C" {

lra_status lra_cur_apply_workspace_size(int64_t n, int32_t k, int32_t nrhs, size_t* bytes) {
  if (bytes == nullptr || n < 1 || k < 1 || k > KMAX || nrhs < 1 || nrhs > 1024) return LRA_ERR_INVALID_ARG;
  *bytes = std::max(apply_ws_bytes(n, k, nrhs), apply_lp_ws_bytes(k, nrhs));
  return LRA_OK;
}

lra_status lra_cur_apply(const void* C, const double* U, const void* R, int64_t m, int64_t n, int32_t k,
                         const double* X, int32_t nrhs, double* Y, int32_t dtype, void* workspace,
                         size_t workspace_bytes, lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (!C || !U || !R || !X || !Y || m < 1 || n < 1 || k < 1 || k > KMAX || nrhs < 1 || nrhs > 1024)
    return LRA_ERR_INVALID_ARG;
  if (dtype != LRA_F64 && dtype != LRA_F32 && dtype != LRA_BF16) return LRA_ERR_INVALID_ARG;
  if (dtype != LRA_F64) return apply_lp(C, U, R, m, n, k, X, nrhs, Y, dtype, workspace, workspace_bytes, stream);
  const size_t need = apply_ws_bytes(n, k, nrhs);
  if (workspace == nullptr || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return LRA_ERR_WORKSPACE;
  const int nb = (int)((n + APPLY_ROWS_PER_CTA - 1) / APPLY_ROWS_PER_CTA);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  double* partial = reinterpret_cast<double*>(ws);
  double* T1 = reinterpret_cast<double*>(ws + align_up(sizeof(double) * (size_t)nb * k * nrhs, 256));
  double* T2 = T1 + align_up(sizeof(double) * (size_t)k * nrhs, 256) / sizeof(double);
  const double* R64 = static_cast<const double*>(R);
  const double* C64 = static_cast<const double*>(C);
  DeviceInfo dev;
  lra_status st = current_device_info(&dev);
  if (st != LRA_OK) return st;
  if (nrhs <= LP_MAX_NRHS) {
    // the tiled stage 1 (coalesced rows of R, persistent CTAs), FP64 products
    const int64_t ntiles = (n + LP_TJ - 1) / LP_TJ;
    const int vec = ((n * 8) % 16 == 0 && (reinterpret_cast<uintptr_t>(R64) & 15u) == 0) ? 1 : 0;
    const size_t smem = lp_rx_smem(k, nrhs, 8);
    LRA_CUDA_TRY(cudaFuncSetAttribute(apply_rx_lp_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    int occ = 1;
    LRA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, apply_rx_lp_kernel<double>, LP_THREADS, smem));
    const int parts = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, std::min<int64_t>(nb, dev.sms * std::min(std::max(occ, 1), 2))));
    unsigned int* done = reinterpret_cast<unsigned int*>(T2 + align_up(sizeof(double) * (size_t)k * nrhs, 256) / 8);
    LRA_CUDA_TRY(cudaMemsetAsync(done, 0, sizeof(unsigned int), stream));
    {
      LaunchScope ls(stream, "apply_rx_kernel");
      apply_rx_lp_kernel<double><<<parts, LP_THREADS, smem, stream>>>(R64, X, n, k, nrhs, vec, partial, U, T1, T2,
                                                                       done);
    }
  } else {
    { LaunchScope ls(stream, "apply_rx_kernel"); apply_rx_kernel<<<nb, NT, 0, stream>>>(R64, X, n, k, nrhs, partial); }
    { LaunchScope ls(stream, "apply_u_kernel"); apply_u_kernel<<<1, NT, 0, stream>>>(partial, nb, U, k, nrhs, T1, T2); }
  }
  const int L = vec_lanes(C64, k, nrhs);
  if (L > 0) {
    const int64_t rows_per_cta = (int64_t)(LP_THREADS / 32) * (32 / L) * 4;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((m + rows_per_cta - 1) / rows_per_cta,
                                                                 (int64_t)dev.sms * 7));
    LaunchScope ls(stream, "apply_c_kernel");
    apply_c_vec_kernel<double><<<grid, LP_THREADS, 0, stream>>>(C64, T2, m, k, nrhs, L, Y);
    return cuda_status(cudaGetLastError());
  }
  const int64_t tot = m * nrhs;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((tot + NT - 1) / NT, (int64_t)dev.sms * 8));
  { LaunchScope ls(stream, "apply_c_kernel"); apply_c_kernel<<<grid, NT, 0, stream>>>(C64, T2, m, k, nrhs, Y); }
  return cuda_status(cudaGetLastError());
}

lra_status lra_residual_sample_workspace_size(int32_t k, int32_t q, int32_t s, size_t* bytes) {
  if (bytes == nullptr || k < 1 || k > KMAX || q < 1 || s < 1) return LRA_ERR_INVALID_ARG;
  *bytes = align_up(sizeof(double) * (size_t)q * k, 256) + 2 * align_up(sizeof(double) * (size_t)q * s, 256) +
           align_up(sizeof(double) * 6 * RESID_MAX_PARTS, 256) + 256;
  return LRA_OK;
}

lra_status lra_residual_sample(const lra_problem* prob, const double* C, const double* U, const double* R,
                               int32_t k, const int32_t* Q, int32_t q, const int32_t* S, int32_t s, double* stats,
                               double* E, void* workspace, size_t workspace_bytes, lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  DevProblem P;
  lra_status st = make_dev_problem(prob, nullptr, &P);
  if (st != LRA_OK) return st;
  if (!C || !U || !R || !Q || !S || !stats || k < 1 || k > KMAX || k > std::min(P.m, P.n) || q < 1 || s < 1)
    return LRA_ERR_INVALID_ARG;
  size_t need = 0;
  lra_residual_sample_workspace_size(k, q, s, &need);
  if (workspace == nullptr || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return LRA_ERR_WORKSPACE;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  double* CU = reinterpret_cast<double*>(ws);
  double* Ews = reinterpret_cast<double*>(ws + align_up(sizeof(double) * (size_t)q * k, 256));
  double* W2 = Ews + align_up(sizeof(double) * (size_t)q * s, 256) / sizeof(double);
  double* part = W2 + align_up(sizeof(double) * (size_t)q * s, 256) / sizeof(double);
  int* bad = reinterpret_cast<int*>(part + align_up(sizeof(double) * 6 * RESID_MAX_PARTS, 256) / sizeof(double));
  double* Eout = E ? E : Ews;
  DeviceInfo dev;
  if ((st = current_device_info(&dev)) != LRA_OK) return st;
  LRA_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), stream));
  const int g1 = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)q * k + NT - 1) / NT, dev.sms * 4));
  { LaunchScope ls(stream, "resid_cu_kernel"); resid_cu_kernel<<<g1, NT, 0, stream>>>(C, U, Q, q, k, P.m, CU, bad); }
  const int g2 = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)q * s + NT - 1) / NT, dev.sms * 8));
  { LaunchScope ls(stream, "resid_e_kernel"); resid_e_kernel<<<g2, NT, 0, stream>>>(P, CU, R, Q, S, q, s, k, Eout, W2, bad); }
  const int64_t K = (int64_t)q * s;
  const int g3 = (int)std::max<int64_t>(1, std::min<int64_t>((K + 4 * NT - 1) / (4 * NT),
                                                             std::min<int64_t>(RESID_MAX_PARTS, dev.sms * 4)));
  { LaunchScope ls(stream, "resid_part_kernel"); resid_part_kernel<<<g3, NT, 0, stream>>>(Eout, W2, K, part); }
  { LaunchScope ls(stream, "resid_var_kernel"); resid_var_kernel<<<g3, NT, 0, stream>>>(Eout, K, part); }
  { LaunchScope ls(stream, "resid_final_kernel"); resid_final_kernel<<<1, 32, 0, stream>>>(part, g3, K, bad, stats); }
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
