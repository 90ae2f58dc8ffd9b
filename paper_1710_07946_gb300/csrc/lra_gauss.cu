// lra_gauss.cu -- differentiable CUR apply y = C U R x on Gaussian-kernel
// blocks at fixed pivots (the FMM stage (iii) product of the generators, made
// differentiable in x, in the sampled kernel entries and in the length scale).
//
// Per block: K(x, y) = exp(-|x - y|^2 / (2 l^2)), C = K(X, Y_J) (m x k),
// R = K(X_I, Y) (k x n), G = K(X_I, Y_J), U = G^{-1}.  The entries of C and R are
// evaluated on the fly in FP32 (never stored); G and U are FP64 (Gauss-Jordan
// with partial pivoting); t1 = R x is accumulated in FP32, t2 = U t1 in FP64,
// y = C t2 in FP32.  The backward recomputes the entries and fuses
//   s1 = C^T dy, dC = dy t2^T, s2 = U^T s1, dx = R^T s2, dR = s2 x^T,
//   dG = -s2 t2^T (U = G^{-1}), dl = sum over C, R, G of dK * K |x - y|^2 / l^3.
// One CTA per block; the tiles of C and R live in shared memory only.
#include <algorithm>
#include <cstring>

#include "lra_internal.h"
#include "lra_profile.h"

namespace lra {

constexpr int GT = 512;          // threads per CTA
constexpr int TILE = 64;         // rows (of C) or columns (of R) per tile

struct GaussArgs {
  const double* X;
  const double* Y;
  const int32_t* I;
  const int32_t* J;
  int32_t nb, m, n, k, nrhs;
  double ell;
  const float* x;
  const float* dy;
  float* y;
  float* dx;
  double* ctx;                   // per block: U (k*k), t1 (k*nrhs), t2 (k*nrhs)
  double* dell;                  // per block
  float* dC;
  float* dR;
  float* dG;
};

// Points are staged in shared memory as FP32 (hi, lo) pairs, x = hi + lo: the
// difference (ph - qh) + (pl - ql) is then as accurate as the rounded FP64
// difference, and the entry costs FP32 work only.
struct P32 {
  float h[3], l[3];
};
__device__ __forceinline__ P32 split_point(const double* p) {
  P32 r;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    r.h[c] = __double2float_rn(p[c]);
    r.l[c] = __double2float_rn(p[c] - (double)r.h[c]);
  }
  return r;
}
__device__ __forceinline__ float gk32s(const P32& p, const P32& q, float inv2l2, float* d2) {
  const float dx = (p.h[0] - q.h[0]) + (p.l[0] - q.l[0]);
  const float dy = (p.h[1] - q.h[1]) + (p.l[1] - q.l[1]);
  const float dz = (p.h[2] - q.h[2]) + (p.l[2] - q.l[2]);
  const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  *d2 = r2;
  return expf(-r2 * inv2l2);
}

__device__ __forceinline__ double gk64(const double* p, const double* q, double ell, double* d2) {
  const double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
  const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
  *d2 = r2;
  return exp(-(r2 / (2.0 * ell * ell)));
}

__device__ double block_sum_d(double v, double* red) {
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
}

// Row stride (floats) of the right-hand-side tiles and of t2, s2: nrhs + 4 when
// nrhs is a multiple of 4 (rows 16-byte aligned for float4 loads; the pad puts
// consecutive rows 4 banks apart, so the 8 rows of one 128-bit load phase fall in
// distinct banks), else nrhs | 1 (odd: consecutive rows in distinct banks).
__host__ __device__ inline int gauss_ldr(int nrhs) { return (nrhs & 3) == 0 ? nrhs + 4 : (nrhs | 1); }

// Four outputs at once (the register-tiled form of the scalar loops, same
// arithmetic): s[q] = fmaf(P[r * pr], Q[r * ldq + q], s[q]) for r = 0..nr-1 in
// ascending order, q < 4; Q 16-byte aligned with ldq a multiple of 4.  Each
// s[q] is the one ascending fmaf chain the scalar loop forms for its output.
__device__ __forceinline__ void chain4(const float* P, int pr, int nr, const float* Q, int ldq, float s[4]) {
  for (int r = 0; r < nr; ++r) {
    const float p = P[r * pr];
    const float4 q = *reinterpret_cast<const float4*>(Q + (size_t)r * ldq);
    s[0] = fmaf(p, q.x, s[0]);
    s[1] = fmaf(p, q.y, s[1]);
    s[2] = fmaf(p, q.z, s[2]);
    s[3] = fmaf(p, q.w, s[3]);
  }
}

// Two dot products over c < nrhs (a multiple of 4) sharing the row A:
// s0 = sum A[c] B0[c], s1 = sum A[c] B1[c], each one ascending fmaf chain (the
// scalar loop's order), the rows read as float4.
__device__ __forceinline__ void dot2(const float* A, const float* B0, const float* B1, int nrhs, float& s0,
                                     float& s1) {
  for (int c = 0; c < nrhs; c += 4) {
    const float4 a = *reinterpret_cast<const float4*>(A + c);
    const float4 b0 = *reinterpret_cast<const float4*>(B0 + c);
    const float4 b1 = *reinterpret_cast<const float4*>(B1 + c);
    s0 = fmaf(a.x, b0.x, s0); s0 = fmaf(a.y, b0.y, s0); s0 = fmaf(a.z, b0.z, s0); s0 = fmaf(a.w, b0.w, s0);
    s1 = fmaf(a.x, b1.x, s1); s1 = fmaf(a.y, b1.y, s1); s1 = fmaf(a.z, b1.z, s1); s1 = fmaf(a.w, b1.w, s1);
  }
}

// U = G^{-1} (k x k, FP64) by Gauss-Jordan with partial pivoting on [G | I] in
// shared memory A (k x 2k).  Returns 0 when a pivot is exactly zero.
__device__ int gauss_jordan(double* A, int k, double* f, int* ctl) {
  const int w2 = 2 * k, tid = threadIdx.x, nt = blockDim.x;
  for (int t = 0; t < k; ++t) {
    if (tid < 32) {
      int best = -1;
      double bv = -1.0;
      for (int p = t + tid; p < k; p += 32) {
        const double v = fabs(A[p * w2 + t]);
        if (v > bv) { bv = v; best = p; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, off);
        const int ob = __shfl_down_sync(0xffffffffu, best, off);
        if (ov > bv || (ov == bv && ob >= 0 && (best < 0 || ob < best))) { bv = ov; best = ob; }
      }
      if (tid == 0) { ctl[0] = best; ctl[1] = (bv > 0.0); }
    }
    __syncthreads();
    if (!ctl[1]) return 0;
    const int r = ctl[0];
    if (r != t)
      for (int j = tid; j < w2; j += nt) {
        const double tmp = A[t * w2 + j]; A[t * w2 + j] = A[r * w2 + j]; A[r * w2 + j] = tmp;
      }
    __syncthreads();
    const double rp = 1.0 / A[t * w2 + t];
    for (int p = tid; p < k; p += nt) f[p] = A[p * w2 + t];
    __syncthreads();
    for (int j = tid; j < w2; j += nt) A[t * w2 + j] = A[t * w2 + j] * rp;
    __syncthreads();
    for (int it = tid; it < k * w2; it += nt) {
      const int p = it / w2, j = it - p * w2;
      if (p != t) A[it] = fma(-f[p], A[t * w2 + j], A[it]);
    }
    __syncthreads();
  }
  return 1;
}

// Every CTA thread checks its share of the block's pivots: true when all
// 0 <= I[a] < m and 0 <= J[a] < n (a block with a bad pivot reads no point).
__device__ __forceinline__ bool pivots_in_range(const int32_t* I, const int32_t* J, int k, int m, int n) {
  int bad = 0;
  for (int a = threadIdx.x; a < k; a += blockDim.x) bad |= (I[a] < 0) | (I[a] >= m) | (J[a] < 0) | (J[a] >= n);
  return !__syncthreads_or(bad);
}

__global__ void __launch_bounds__(GT, 2) gauss_fwd_kernel(GaussArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = g.k, nrhs = g.nrhs, m = g.m, n = g.n, tid = threadIdx.x, nt = blockDim.x;
  const int ldr = gauss_ldr(nrhs);
  const bool v4 = (nrhs & 3) == 0;                               // register-tiled loops
  const int nq = nrhs >> 2;
  const float inv2l2 = (float)(1.0 / (2.0 * g.ell * g.ell));
  double* A = reinterpret_cast<double*>(smem);                  // k x 2k
  double* f = A + (size_t)k * 2 * k;                            // KMAX
  double* t1d = f + KMAX;                                       // k x nrhs
  P32* pk = reinterpret_cast<P32*>(t1d + (size_t)k * nrhs);      // k pivot points (I, then J)
  P32* pt = pk + KMAX;                                          // TILE tile points
  float* tile = reinterpret_cast<float*>(pt + TILE);            // TILE x (k|1) entries
  float* xt = tile + (size_t)TILE * (k | 1);                    // TILE x ldr
  float* t2f = xt + (size_t)TILE * ldr;                         // k x ldr
  const int ldk = k | 1;
  __shared__ int ctl[4];
  for (int b = blockIdx.x; b < g.nb; b += gridDim.x) {
    const double* X = g.X + (size_t)b * m * 3;
    const double* Y = g.Y + (size_t)b * n * 3;
    const int32_t* I = g.I + (size_t)b * k;
    const int32_t* J = g.J + (size_t)b * k;
    double* ctx = g.ctx + (size_t)b * ((size_t)k * k + 2 * (size_t)k * nrhs);
    double* U = ctx;
    double* t1 = U + (size_t)k * k;
    double* t2 = t1 + (size_t)k * nrhs;
    if (!pivots_in_range(I, J, k, m, n)) {      // failed block: NaN context and outputs
      const double qn = __longlong_as_double(0x7ff8000000000000ll);
      for (size_t it = tid; it < (size_t)k * k + 2 * (size_t)k * nrhs; it += nt) ctx[it] = qn;
      for (size_t it = tid; it < (size_t)m * nrhs; it += nt) g.y[(size_t)b * m * nrhs + it] = __int_as_float(0x7fc00000);
      __syncthreads();
      continue;
    }
    // G and U = G^{-1}
    for (int it = tid; it < k * k; it += nt) {
      const int a = it / k, c = it - a * k;
      double d2;
      A[a * 2 * k + c] = gk64(X + 3 * (size_t)I[a], Y + 3 * (size_t)J[c], g.ell, &d2);
      A[a * 2 * k + k + c] = (a == c) ? 1.0 : 0.0;
    }
    for (int a = tid; a < k; a += nt) pk[a] = split_point(X + 3 * (size_t)I[a]);
    __syncthreads();
    const int ok = gauss_jordan(A, k, f, ctl);
    for (int it = tid; it < k * k; it += nt) {
      const int a = it / k, c = it - a * k;
      U[it] = ok ? A[a * 2 * k + k + c] : __longlong_as_double(0x7ff8000000000000ll);
    }
    // t1 = R x, R entries on the fly
    for (int it = tid; it < k * nrhs; it += nt) t1d[it] = 0.0;
    __syncthreads();
    for (int j0 = 0; j0 < n; j0 += TILE) {
      const int tj = min(TILE, n - j0);
      for (int j = tid; j < tj; j += nt) pt[j] = split_point(Y + 3 * (size_t)(j0 + j));
      for (int it = tid; it < tj * nrhs; it += nt) {
        const int j = it / nrhs, c = it - j * nrhs;
        xt[j * ldr + c] = g.x[((size_t)b * n + j0) * nrhs + it];
      }
      __syncthreads();
      for (int it = tid; it < k * tj; it += nt) {
        const int a = it / tj, j = it - a * tj;
        float d2;
        tile[j * ldk + a] = gk32s(pk[a], pt[j], inv2l2, &d2);
      }
      __syncthreads();
      if (v4) {
        for (int o = tid; o < k * nq; o += nt) {
          const int a = o / nq, c = (o - a * nq) << 2;
          float s4[4] = {0.f, 0.f, 0.f, 0.f};
          chain4(tile + a, ldk, tj, xt + c, ldr, s4);
          for (int q = 0; q < 4; ++q) t1d[a * nrhs + c + q] += (double)s4[q];
        }
      } else {
        for (int o = tid; o < k * nrhs; o += nt) {
          const int a = o / nrhs, c = o - a * nrhs;
          float s = 0.f;
          for (int j = 0; j < tj; ++j) s = fmaf(tile[j * ldk + a], xt[j * ldr + c], s);
          t1d[o] += (double)s;
        }
      }
      __syncthreads();
    }
    // t2 = U t1 (FP64); the J points replace the I points
    for (int o = tid; o < k * nrhs; o += nt) {
      const int a = o / nrhs, c = o - a * nrhs;
      double s = 0.0;
      for (int q = 0; q < k; ++q) s = fma(U[a * k + q], t1d[q * nrhs + c], s);
      t2[o] = s;
      t1[o] = t1d[o];
      t2f[a * ldr + c] = (float)s;
    }
    __syncthreads();
    for (int a = tid; a < k; a += nt) pk[a] = split_point(Y + 3 * (size_t)J[a]);
    // y = C t2, C entries on the fly
    for (int i0 = 0; i0 < m; i0 += TILE) {
      const int ti = min(TILE, m - i0);
      for (int i = tid; i < ti; i += nt) pt[i] = split_point(X + 3 * (size_t)(i0 + i));
      __syncthreads();
      for (int it = tid; it < ti * k; it += nt) {
        const int i = it / k, a = it - i * k;
        float d2;
        tile[i * ldk + a] = gk32s(pt[i], pk[a], inv2l2, &d2);
      }
      __syncthreads();
      if (v4) {
        for (int o = tid; o < ti * nq; o += nt) {
          const int i = o / nq, c = (o - i * nq) << 2;
          float s4[4] = {0.f, 0.f, 0.f, 0.f};
          chain4(tile + i * ldk, 1, k, t2f + c, ldr, s4);
          float* yo = g.y + ((size_t)b * m + i0 + i) * nrhs + c;
          for (int q = 0; q < 4; ++q) yo[q] = s4[q];
        }
      } else {
        for (int o = tid; o < ti * nrhs; o += nt) {
          const int i = o / nrhs, c = o - i * nrhs;
          float s = 0.f;
          for (int a = 0; a < k; ++a) s = fmaf(tile[i * ldk + a], t2f[a * ldr + c], s);
          g.y[((size_t)b * m + i0) * nrhs + o] = s;
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(GT, 2) gauss_bwd_kernel(GaussArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = g.k, nrhs = g.nrhs, m = g.m, n = g.n, tid = threadIdx.x, nt = blockDim.x;
  const int ldr = gauss_ldr(nrhs), ldk = k | 1;
  const bool v4 = (nrhs & 3) == 0;                               // register-tiled loops
  const int nq = nrhs >> 2;
  const float inv2l2 = (float)(1.0 / (2.0 * g.ell * g.ell));
  const float il3 = (float)(1.0 / (g.ell * g.ell * g.ell));
  double* s1 = reinterpret_cast<double*>(smem);                 // k x nrhs
  double* s2d = s1 + (size_t)k * nrhs;                           // k x nrhs
  P32* pk = reinterpret_cast<P32*>(s2d + (size_t)k * nrhs);      // k pivot points
  P32* pt = pk + KMAX;                                          // TILE tile points
  float* t2f = reinterpret_cast<float*>(pt + TILE);             // k x ldr
  float* s2f = t2f + (size_t)k * ldr;                            // k x ldr
  float* tile = s2f + (size_t)k * ldr;                           // TILE x ldk entries
  float* dtile = tile + (size_t)TILE * ldk;                      // TILE x ldk dK/dl
  float* vt = dtile + (size_t)TILE * ldk;                        // TILE x ldr (dy or x tile)
  __shared__ double red[33];
  for (int b = blockIdx.x; b < g.nb; b += gridDim.x) {
    const double* X = g.X + (size_t)b * m * 3;
    const double* Y = g.Y + (size_t)b * n * 3;
    const int32_t* I = g.I + (size_t)b * k;
    const int32_t* J = g.J + (size_t)b * k;
    const double* ctx = g.ctx + (size_t)b * ((size_t)k * k + 2 * (size_t)k * nrhs);
    const double* U = ctx;
    const double* t2 = ctx + (size_t)k * k + (size_t)k * nrhs;
    if (!pivots_in_range(I, J, k, m, n)) {      // failed block: NaN gradients
      const float qf = __int_as_float(0x7fc00000);
      for (size_t it = tid; it < (size_t)n * nrhs; it += nt) g.dx[(size_t)b * n * nrhs + it] = qf;
      if (g.dC) for (size_t it = tid; it < (size_t)m * k; it += nt) g.dC[(size_t)b * m * k + it] = qf;
      if (g.dR) for (size_t it = tid; it < (size_t)k * n; it += nt) g.dR[(size_t)b * k * n + it] = qf;
      if (g.dG) for (size_t it = tid; it < (size_t)k * k; it += nt) g.dG[(size_t)b * k * k + it] = qf;
      if (tid == 0) g.dell[b] = __longlong_as_double(0x7ff8000000000000ll);
      __syncthreads();
      continue;
    }
    double dl = 0.0;
    for (int it = tid; it < k * nrhs; it += nt) {
      const int a = it / nrhs, c = it - a * nrhs;
      s1[it] = 0.0;
      t2f[a * ldr + c] = (float)t2[it];
    }
    for (int a = tid; a < k; a += nt) pk[a] = split_point(Y + 3 * (size_t)J[a]);
    __syncthreads();
    // pass over C: s1 = C^T dy, dC = dy t2^T, dl_C
    for (int i0 = 0; i0 < m; i0 += TILE) {
      const int ti = min(TILE, m - i0);
      for (int i = tid; i < ti; i += nt) pt[i] = split_point(X + 3 * (size_t)(i0 + i));
      for (int it = tid; it < ti * nrhs; it += nt) {
        const int i = it / nrhs, c = it - i * nrhs;
        vt[i * ldr + c] = g.dy[((size_t)b * m + i0) * nrhs + it];
      }
      __syncthreads();
      for (int it = tid; it < ti * k; it += nt) {
        const int i = it / k, a = it - i * k;
        float d2;
        const float kv = gk32s(pt[i], pk[a], inv2l2, &d2);
        tile[i * ldk + a] = kv;
        dtile[i * ldk + a] = kv * d2 * il3;
      }
      __syncthreads();
      float dls = 0.f;
      if (v4) {
        for (int o = tid; o < k * nq; o += nt) {
          const int a = o / nq, c = (o - a * nq) << 2;
          float s4[4] = {0.f, 0.f, 0.f, 0.f};
          chain4(tile + a, ldk, ti, vt + c, ldr, s4);
          for (int q = 0; q < 4; ++q) s1[a * nrhs + c + q] += (double)s4[q];
        }
        // two rows i per thread, lanes over a (rows of t2f in distinct banks)
        const int nip = (ti + 1) >> 1;
        for (int it = tid; it < nip * k; it += nt) {
          const int ip = it / k, a = it - ip * k, i = 2 * ip;
          const int i1 = min(i + 1, ti - 1);
          float s0 = 0.f, s1v = 0.f;
          dot2(t2f + a * ldr, vt + i * ldr, vt + i1 * ldr, nrhs, s0, s1v);
          if (g.dC) g.dC[((size_t)b * m + i0 + i) * k + a] = s0;
          dls = fmaf(s0, dtile[i * ldk + a], dls);
          if (i + 1 < ti) {
            if (g.dC) g.dC[((size_t)b * m + i0 + i + 1) * k + a] = s1v;
            dls = fmaf(s1v, dtile[(i + 1) * ldk + a], dls);
          }
        }
      } else {
        for (int o = tid; o < k * nrhs; o += nt) {
          const int a = o / nrhs, c = o - a * nrhs;
          float s = 0.f;
          for (int i = 0; i < ti; ++i) s = fmaf(tile[i * ldk + a], vt[i * ldr + c], s);
          s1[o] += (double)s;
        }
        for (int it = tid; it < ti * k; it += nt) {
          const int i = it / k, a = it - i * k;
          float s = 0.f;
          for (int c = 0; c < nrhs; ++c) s = fmaf(vt[i * ldr + c], t2f[a * ldr + c], s);
          if (g.dC) g.dC[((size_t)b * m + i0 + i) * k + a] = s;
          dls = fmaf(s, dtile[i * ldk + a], dls);
        }
      }
      dl += (double)dls;
      __syncthreads();
    }
    // s2 = U^T s1
    for (int o = tid; o < k * nrhs; o += nt) {
      const int a = o / nrhs, c = o - a * nrhs;
      double s = 0.0;
      for (int q = 0; q < k; ++q) s = fma(U[q * k + a], s1[q * nrhs + c], s);
      s2d[o] = s;
      s2f[a * ldr + c] = (float)s;
    }
    __syncthreads();
    for (int a = tid; a < k; a += nt) pk[a] = split_point(X + 3 * (size_t)I[a]);
    // pass over R: dx = R^T s2, dR = s2 x^T, dl_R
    for (int j0 = 0; j0 < n; j0 += TILE) {
      const int tj = min(TILE, n - j0);
      for (int j = tid; j < tj; j += nt) pt[j] = split_point(Y + 3 * (size_t)(j0 + j));
      for (int it = tid; it < tj * nrhs; it += nt) {
        const int j = it / nrhs, c = it - j * nrhs;
        vt[j * ldr + c] = g.x[((size_t)b * n + j0) * nrhs + it];
      }
      __syncthreads();
      for (int it = tid; it < k * tj; it += nt) {
        const int a = it / tj, j = it - a * tj;
        float d2;
        const float kv = gk32s(pk[a], pt[j], inv2l2, &d2);
        tile[j * ldk + a] = kv;
        dtile[j * ldk + a] = kv * d2 * il3;
      }
      __syncthreads();
      float dls = 0.f;
      if (v4) {
        for (int o = tid; o < tj * nq; o += nt) {
          const int j = o / nq, c = (o - j * nq) << 2;
          float s4[4] = {0.f, 0.f, 0.f, 0.f};
          chain4(tile + j * ldk, 1, k, s2f + c, ldr, s4);
          float* dxo = g.dx + ((size_t)b * n + j0 + j) * nrhs + c;
          for (int q = 0; q < 4; ++q) dxo[q] = s4[q];
        }
        // two rows a per thread, lanes over j (rows of vt in distinct banks; dR stores coalesced)
        const int nap = (k + 1) >> 1;
        for (int it = tid; it < nap * tj; it += nt) {
          const int ap = it / tj, j = it - ap * tj, a = 2 * ap;
          const int a1 = min(a + 1, k - 1);
          float s0 = 0.f, s1v = 0.f;
          dot2(vt + j * ldr, s2f + a * ldr, s2f + a1 * ldr, nrhs, s0, s1v);
          if (g.dR) g.dR[((size_t)b * k + a) * n + j0 + j] = s0;
          dls = fmaf(s0, dtile[j * ldk + a], dls);
          if (a + 1 < k) {
            if (g.dR) g.dR[((size_t)b * k + a + 1) * n + j0 + j] = s1v;
            dls = fmaf(s1v, dtile[j * ldk + a + 1], dls);
          }
        }
      } else {
        for (int o = tid; o < tj * nrhs; o += nt) {
          const int j = o / nrhs, c = o - j * nrhs;
          float s = 0.f;
          for (int a = 0; a < k; ++a) s = fmaf(tile[j * ldk + a], s2f[a * ldr + c], s);
          g.dx[((size_t)b * n + j0) * nrhs + o] = s;
        }
        for (int it = tid; it < k * tj; it += nt) {
          const int j = it / k, a = it - j * k;
          float s = 0.f;
          for (int c = 0; c < nrhs; ++c) s = fmaf(s2f[a * ldr + c], vt[j * ldr + c], s);
          if (g.dR) g.dR[((size_t)b * k + a) * n + j0 + j] = s;
          dls = fmaf(s, dtile[j * ldk + a], dls);
        }
      }
      dl += (double)dls;
      __syncthreads();
    }
    // dG = -s2 t2^T and dl_G
    for (int it = tid; it < k * k; it += nt) {
      const int a = it / k, c = it - a * k;
      double s = 0.0;
      for (int q = 0; q < nrhs; ++q) s = fma(-s2d[a * nrhs + q], t2[c * nrhs + q], s);
      double d2;
      const double gv = gk64(X + 3 * (size_t)I[a], Y + 3 * (size_t)J[c], g.ell, &d2);
      if (g.dG) g.dG[(size_t)b * k * k + it] = (float)s;
      dl = fma(s, gv * d2 / (g.ell * g.ell * g.ell), dl);
    }
    dl = block_sum_d(dl, red);
    if (tid == 0) g.dell[b] = dl;
    __syncthreads();
  }
}

static lra_status gauss_check(const lra_gauss_blocks* gb, int32_t nrhs) {
  if (gb == nullptr || gb->X == nullptr || gb->Y == nullptr || gb->I == nullptr || gb->J == nullptr) return LRA_ERR_INVALID_ARG;
  if (gb->nb < 1 || gb->m < 1 || gb->n < 1 || gb->k < 1 || gb->k > KMAX || gb->k > gb->m || gb->k > gb->n)
    return LRA_ERR_INVALID_ARG;
  if (nrhs < 1 || nrhs > 256 || !(gb->length_scale > 0.0)) return LRA_ERR_INVALID_ARG;
  return LRA_OK;
}

static size_t fwd_smem(int k, int nrhs) {
  return sizeof(double) * ((size_t)k * 2 * k + KMAX + (size_t)k * nrhs) + sizeof(P32) * (KMAX + TILE) +
         sizeof(float) * ((size_t)TILE * (k | 1) + (size_t)TILE * gauss_ldr(nrhs) + (size_t)k * gauss_ldr(nrhs));
}
static size_t bwd_smem(int k, int nrhs) {
  return sizeof(double) * 2 * (size_t)k * nrhs + sizeof(P32) * (KMAX + TILE) +
         sizeof(float) * (2 * (size_t)k * gauss_ldr(nrhs) + 2 * (size_t)TILE * (k | 1) + (size_t)TILE * gauss_ldr(nrhs));
}

}  // namespace lra

using namespace lra;

extern "C" {

lra_status lra_gauss_cur_forward(const lra_gauss_blocks* gb, const float* x, int32_t nrhs, float* y, double* ctx,
                                 lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  lra_status st = gauss_check(gb, nrhs);
  if (st != LRA_OK) return st;
  if (!x || !y || !ctx) return LRA_ERR_INVALID_ARG;
  GaussArgs a;
  std::memset(&a, 0, sizeof(a));
  a.X = gb->X; a.Y = gb->Y; a.I = gb->I; a.J = gb->J;
  a.nb = gb->nb; a.m = gb->m; a.n = gb->n; a.k = gb->k; a.nrhs = nrhs; a.ell = gb->length_scale;
  a.x = x; a.y = y; a.ctx = ctx;
  const size_t smem = fwd_smem(gb->k, nrhs);
  DeviceInfo dev;
  if ((st = current_device_info(&dev)) != LRA_OK) return st;
  if (smem > dev.smem_optin - 1024) return LRA_ERR_INVALID_ARG;
  LRA_CUDA_TRY(cudaFuncSetAttribute(gauss_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  {
    LaunchScope ls(stream, "gauss_fwd_kernel");
    gauss_fwd_kernel<<<std::min(gb->nb, dev.sms * 4), GT, smem, stream>>>(a);
  }
  return cuda_status(cudaGetLastError());
}

lra_status lra_gauss_cur_backward(const lra_gauss_blocks* gb, const float* x, const float* dy, int32_t nrhs,
                                  const double* ctx, float* dx, double* dell, float* dC, float* dR, float* dG,
                                  lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  lra_status st = gauss_check(gb, nrhs);
  if (st != LRA_OK) return st;
  if (!x || !dy || !ctx || !dx || !dell) return LRA_ERR_INVALID_ARG;
  GaussArgs a;
  std::memset(&a, 0, sizeof(a));
  a.X = gb->X; a.Y = gb->Y; a.I = gb->I; a.J = gb->J;
  a.nb = gb->nb; a.m = gb->m; a.n = gb->n; a.k = gb->k; a.nrhs = nrhs; a.ell = gb->length_scale;
  a.x = x; a.dy = dy; a.ctx = const_cast<double*>(ctx); a.dx = dx; a.dell = dell; a.dC = dC; a.dR = dR; a.dG = dG;
  const size_t smem = bwd_smem(gb->k, nrhs);
  DeviceInfo dev;
  if ((st = current_device_info(&dev)) != LRA_OK) return st;
  if (smem > dev.smem_optin - 1024) return LRA_ERR_INVALID_ARG;
  LRA_CUDA_TRY(cudaFuncSetAttribute(gauss_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  {
    LaunchScope ls(stream, "gauss_bwd_kernel");
    gauss_bwd_kernel<<<std::min(gb->nb, dev.sms * 4), GT, smem, stream>>>(a);
  }
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
