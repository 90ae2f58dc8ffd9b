// lra_nucleus.cuh -- the canonical nucleus U = pinv(G_r) of a k x k generator G
// on one CTA, in FP64 (paper: Algorithm algcnnncl, with the rank-revealing
// factorisation that Remark reubsc allows in place of the SVD).
//
//   1. Householder QR with column pivoting, G P = Q R: at step t the column with
//      the largest squared norm over rows t.. (recomputed each step) moves to
//      position t, the lowest index winning ties.  Every inner product of the
//      QR (the norms, each reflector's ||x||^2 and v^T y) is one ascending fma
//      chain owned by one thread.
//   2. r = number of leading |R_tt| > tol |R_00|.
//   3. U = P Z S^{-T} Q_r^T, where T = [R11 R12] (r x k) and T^T = Z S is its QR
//      (a complete orthogonal decomposition); for r = k this is P R^{-1} Q^T.
// Every reflector is the textbook H = I - tau v v^T with v_0 = 1 and
// beta = -sign(alpha) ||x||; every other inner product is an ascending fma
// chain owned by one thread, so the result does not depend on the thread count.
#pragma once

#include "lra_device.cuh"

namespace lra {

// Shared memory needed by nucleus_cta for generator size k.
// Columns are stored with an odd stride ld = k | 1 so that threads owning
// different columns hit different shared-memory banks.
__host__ __device__ inline int nucleus_ld(int k) { return k | 1; }
__host__ __device__ inline size_t nucleus_smem_bytes(int k) {
  return sizeof(double) * (3 * (size_t)k * nucleus_ld(k) + 4 * (size_t)KMAX) + sizeof(int32_t) * 2 * KMAX + 64;
}

// Householder reflector of the column x[0..len) (unit stride, shared memory),
// computed by thread 0, scaled by all threads.  Returns tau to every thread.
__device__ inline double house_cta(double* x, int len, double* bcast) {
  if (threadIdx.x == 0) {
    double alpha = x[0], xn2 = 0.0, tau = 0.0, scal = 0.0, beta = alpha;
    for (int i = 1; i < len; ++i) xn2 = fma(x[i], x[i], xn2);
    if (xn2 != 0.0) {
      double nrm = sqrt(fma(alpha, alpha, xn2));
      beta = (alpha >= 0.0) ? -nrm : nrm;
      tau = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
    }
    bcast[0] = tau; bcast[1] = scal; bcast[2] = beta;
  }
  __syncthreads();
  const double tau = bcast[0], scal = bcast[1];
  if (tau != 0.0) {
    for (int i = 1 + threadIdx.x; i < len; i += blockDim.x) x[i] = x[i] * scal;
  }
  __syncthreads();
  if (threadIdx.x == 0 && tau != 0.0) x[0] = bcast[2];
  __syncthreads();
  return tau;
}

// y <- (I - tau v v^T) y for one column, by the calling thread alone.
__device__ __forceinline__ void apply_house_seq(const double* v, double tau, double* y, int len) {
  if (tau == 0.0) return;
  double w = y[0];
  for (int i = 1; i < len; ++i) w = fma(v[i], y[i], w);
  const double c = tau * w;
  y[0] = y[0] - c;
  for (int i = 1; i < len; ++i) y[i] = fma(-c, v[i], y[i]);
}

// Columns j = j0 .. j0 + ncol - 1 (stride ld) <- (I - tau v v^T) applied to
// rows 0..len-1: one thread per column, v^T y = y[0] + v[1] y[1] + ... as one
// ascending fma chain (apply_house_seq).
__device__ inline void apply_house_cols(const double* v, double tau, double* A, int ld, int j0, int ncol, int len) {
  for (int g = threadIdx.x; g < ncol; g += blockDim.x) apply_house_seq(v, tau, A + (size_t)(j0 + g) * ld, len);
}

// Squared norms over rows t..k-1 of columns j0 .. j0 + ncol - 1 into nrm[j]:
// one thread per column, one ascending fma chain.
__device__ inline void col_norms(const double* A, int ld, int t, int k, int j0, int ncol, double* nrm) {
  for (int g = threadIdx.x; g < ncol; g += blockDim.x) {
    const double* col = A + (size_t)(j0 + g) * ld;
    double s = 0.0;
    for (int i = t; i < k; ++i) s = fma(col[i], col[i], s);
    nrm[j0 + g] = s;
  }
}

// U (k x k, row-major, global or shared) <- pinv of the rank-r QRP truncation of
// G (k x k row-major, global).  smem: nucleus_smem_bytes(k).  Returns r.
static __device__ __noinline__ int nucleus_cta(const double* G, int k, double tol, double* U, unsigned char* smem) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ld = nucleus_ld(k);
  double* A = reinterpret_cast<double*>(smem);          // column-major k x k, stride ld
  double* Q = A + (size_t)k * ld;                       // Q^T, column-major
  double* T = Q + (size_t)k * ld;                       // T^T (k x r), column-major
  double* taus = T + (size_t)k * ld;
  double* tz = taus + KMAX;
  double* nrm = tz + KMAX;
  double* bc = nrm + KMAX;
  int32_t* perm = reinterpret_cast<int32_t*>(bc + KMAX);
  int32_t* ctl = perm + KMAX;

  for (int it = tid; it < k * k; it += nt) {
    int i = it / k, j = it - i * k;
    A[j * ld + i] = G[it];
  }
  for (int j = tid; j < k; j += nt) perm[j] = j;
  __syncthreads();
  for (int t = 0; t < k; ++t) {
    col_norms(A, ld, t, k, t, k - t, nrm);
    __syncthreads();
    if (tid < 32) {
      // largest squared norm, lowest column on ties (integer keys, one warp)
      Cand c = cand_none();
      for (int j = t + tid; j < k; j += 32) cand_consider(c, mag_key(nrm[j]), 0, j);
      for (int off = 16; off > 0; off >>= 1) {
        Cand o;
        o.key = __shfl_down_sync(0xffffffffu, c.key, off);
        o.i = __shfl_down_sync(0xffffffffu, c.i, off);
        o.j = __shfl_down_sync(0xffffffffu, c.j, off);
        if (cand_better(o, c)) c = o;
      }
      if (tid == 0) {
        const int pj = (c.key == 0ull) ? t : c.j;
        ctl[0] = pj;
        if (pj != t) { int tp = perm[t]; perm[t] = perm[pj]; perm[pj] = tp; }
      }
    }
    __syncthreads();
    const int pj = ctl[0];
    if (pj != t)
      for (int i = tid; i < k; i += nt) {
        double tmp = A[t * ld + i]; A[t * ld + i] = A[pj * ld + i]; A[pj * ld + i] = tmp;
      }
    __syncthreads();
    const double tau = house_cta(&A[t * ld + t], k - t, bc);
    if (tid == 0) taus[t] = tau;
    apply_house_cols(&A[t * ld + t], tau, &A[t], ld, t + 1, k - t - 1, k - t);
    __syncthreads();
  }
  if (tid == 0) {
    int r = 0;
    const double r00 = fabs(A[0]);
    if (r00 > 0.0) while (r < k && fabs(A[r * ld + r]) > tol * r00) ++r;
    ctl[1] = r;
  }
  __syncthreads();
  const int r = ctl[1];
  for (int it = tid; it < k * k; it += nt) U[it] = 0.0;
  if (r == 0) { __syncthreads(); return 0; }

  // Q^T = H_{k-1} ... H_0 I, one column per thread
  for (int j = tid; j < k; j += nt) {
    for (int i = 0; i < k; ++i) Q[j * ld + i] = (i == j) ? 1.0 : 0.0;
    for (int t = 0; t < k; ++t) apply_house_seq(&A[t * ld + t], taus[t], &Q[j * ld + t], k - t);
  }
  if (r < k) {
    for (int it = tid; it < k * r; it += nt) {
      int c = it / k, i = it - c * k;
      T[c * ld + i] = (i >= c) ? A[i * ld + c] : 0.0;
    }
    __syncthreads();
    for (int c = 0; c < r; ++c) {
      const double tau = house_cta(&T[c * ld + c], k - c, bc);
      if (tid == 0) tz[c] = tau;
      for (int j = c + 1 + tid; j < r; j += nt) apply_house_seq(&T[c * ld + c], tau, &T[j * ld + c], k - c);
      __syncthreads();
    }
  }
  __syncthreads();
  // X = Z S^{-T} Q_r^T (or R^{-1} Q^T), one column per thread, in place in Q
  for (int col = tid; col < k; col += nt) {
    double* v = &Q[col * ld];
    if (r == k) {
      for (int i = k - 1; i >= 0; --i) {
        double s = v[i];
        for (int p = i + 1; p < k; ++p) s = fma(-A[p * ld + i], v[p], s);
        v[i] = s / A[i * ld + i];
      }
    } else {
      for (int i = 0; i < r; ++i) {
        double s = v[i];
        for (int p = 0; p < i; ++p) s = fma(-T[i * ld + p], v[p], s);
        v[i] = s / T[i * ld + i];
      }
      for (int i = r; i < k; ++i) v[i] = 0.0;
      for (int c = r - 1; c >= 0; --c) apply_house_seq(&T[c * ld + c], tz[c], &v[c], k - c);
    }
  }
  __syncthreads();
  for (int it = tid; it < k * k; it += nt) {
    int i = it / k, col = it - i * k;
    U[(size_t)perm[i] * k + col] = Q[col * ld + i];
  }
  __syncthreads();
  return r;
}

// Shared memory of nucleus_rect_cta for a k x l generator.
__host__ __device__ inline size_t nucleus_rect_smem_bytes(int k, int l) {
  const size_t ldk = (size_t)(k | 1), ldl = (size_t)(l | 1);
  return sizeof(double) * ((size_t)l * ldk + (size_t)k * ldk + 2 * (size_t)k * ldl + 2 * (size_t)KMAX + 4) +
         sizeof(int32_t) * ((size_t)l + 4) + 64;
}

// U (l x k, row-major) <- pinv of the rank-r QRP truncation of the k x l
// generator G (row-major, global, k <= l <= 2 KMAX): QRP over the l columns
// (k steps), r = #{|R_tt| > tol |R_00|}, then T^T = (rows 0..r-1 of R)^T = Z S
// and U = P Z S^{-T} Q_r^T, each inner product an ascending fma chain owned by
// one thread (the arithmetic of the FP64 reference's rectangular nucleus).
// smem: nucleus_rect_smem_bytes(k, l).  Returns r.
__device__ inline int nucleus_rect_cta(const double* G, int k, int l, double tol, double* U, unsigned char* smem) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ldk = k | 1, ldl = l | 1;
  double* A = reinterpret_cast<double*>(smem);          // column-major k x l, stride ldk
  double* Q = A + (size_t)l * ldk;                      // Q^T, column-major k x k
  double* T = Q + (size_t)k * ldk;                      // T^T (l x r), column-major, stride ldl
  double* X = T + (size_t)k * ldl;                      // l x k, column-major, stride ldl
  double* taus = X + (size_t)k * ldl;
  double* tz = taus + KMAX;
  double* bc = tz + KMAX;
  int32_t* perm = reinterpret_cast<int32_t*>(bc + 4);
  int32_t* ctl = perm + l;

  for (int it = tid; it < k * l; it += nt) {
    const int i = it / l, j = it - i * l;
    A[j * ldk + i] = G[it];
  }
  for (int j = tid; j < l; j += nt) perm[j] = j;
  __syncthreads();
  for (int t = 0; t < k; ++t) {
    // largest squared column norm over rows t.., lowest column on ties (one thread
    // per column accumulates, one warp compares integer keys)
    double* nrm = X;                                    // l scratch doubles (X is unused yet)
    col_norms(A, ldk, t, k, t, l - t, nrm);
    __syncthreads();
    if (tid < 32) {
      Cand c = cand_none();
      for (int j = t + tid; j < l; j += 32) cand_consider(c, mag_key(nrm[j]), 0, j);
      for (int off = 16; off > 0; off >>= 1) {
        Cand o;
        o.key = __shfl_down_sync(0xffffffffu, c.key, off);
        o.i = __shfl_down_sync(0xffffffffu, c.i, off);
        o.j = __shfl_down_sync(0xffffffffu, c.j, off);
        if (cand_better(o, c)) c = o;
      }
      if (tid == 0) {
        const int pj = (c.key == 0ull) ? t : c.j;
        ctl[0] = pj;
        if (pj != t) { int tp = perm[t]; perm[t] = perm[pj]; perm[pj] = tp; }
      }
    }
    __syncthreads();
    const int pj = ctl[0];
    if (pj != t)
      for (int i = tid; i < k; i += nt) {
        double tmp = A[t * ldk + i]; A[t * ldk + i] = A[pj * ldk + i]; A[pj * ldk + i] = tmp;
      }
    __syncthreads();
    const double tau = house_cta(&A[t * ldk + t], k - t, bc);
    if (tid == 0) taus[t] = tau;
    apply_house_cols(&A[t * ldk + t], tau, &A[t], ldk, t + 1, l - t - 1, k - t);
    __syncthreads();
  }
  if (tid == 0) {
    int r = 0;
    const double r00 = fabs(A[0]);
    if (r00 > 0.0) while (r < k && fabs(A[r * ldk + r]) > tol * r00) ++r;
    ctl[1] = r;
  }
  __syncthreads();
  const int r = ctl[1];
  for (int it = tid; it < l * k; it += nt) U[it] = 0.0;
  if (r == 0) { __syncthreads(); return 0; }
  // Q^T = H_{k-1} ... H_0 I, one column per thread
  for (int j = tid; j < k; j += nt) {
    for (int i = 0; i < k; ++i) Q[j * ldk + i] = (i == j) ? 1.0 : 0.0;
    for (int t = 0; t < k; ++t) apply_house_seq(&A[t * ldk + t], taus[t], &Q[j * ldk + t], k - t);
  }
  // T^T and its QR
  for (int it = tid; it < l * r; it += nt) {
    const int c = it / l, i = it - c * l;
    T[c * ldl + i] = (i >= c) ? A[i * ldk + c] : 0.0;
  }
  __syncthreads();
  for (int c = 0; c < r; ++c) {
    const double tz_c = house_cta(&T[c * ldl + c], l - c, bc);
    if (tid == 0) tz[c] = tz_c;
    for (int j = c + 1 + tid; j < r; j += nt) apply_house_seq(&T[c * ldl + c], tz_c, &T[j * ldl + c], l - c);
    __syncthreads();
  }
  // X = Z S^{-T} Q_r^T, one column per thread
  for (int col = tid; col < k; col += nt) {
    double* v = &X[col * ldl];
    for (int i = 0; i < l; ++i) v[i] = 0.0;
    for (int i = 0; i < r; ++i) {
      double s = Q[col * ldk + i];
      for (int p = 0; p < i; ++p) s = fma(-T[i * ldl + p], v[p], s);
      v[i] = s / T[i * ldl + i];
    }
    for (int c = r - 1; c >= 0; --c) apply_house_seq(&T[c * ldl + c], tz[c], &v[c], l - c);
  }
  __syncthreads();
  for (int it = tid; it < l * k; it += nt) {
    const int i = it / k, col = it - i * k;
    U[(size_t)perm[i] * k + col] = X[col * ldl + i];
  }
  __syncthreads();
  return r;
}

}  // namespace lra
