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
  return sizeof(double) * (3 * (size_t)k * nucleus_ld(k) + 9 * (size_t)KMAX) + sizeof(int32_t) * 2 * KMAX + 64;
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

// Reflector scalars from alpha = x[0] and xn2 = x[1]^2 + ... (one ascending
// fma chain, computed by the caller): beta = -sign(alpha) sqrt(alpha^2 + xn2),
// tau = (beta - alpha) / beta, scal = 1 / (alpha - beta); tau = scal = 0 and
// beta = alpha when xn2 = 0.  Called by a whole warp (the same operands in every
// lane): lanes 0 and 1 take the two divisions in one instruction stream, so the
// step costs one division's latency.  Lane 0 stores tau, scal, beta in bc.
__device__ __forceinline__ void house_scalars_warp(double alpha, double xn2, double* bc) {
  const int lane = threadIdx.x & 31;
  double tau = 0.0, scal = 0.0, beta = alpha;
  if (xn2 != 0.0) {
    const double nrm = sqrt(fma(alpha, alpha, xn2));
    beta = (alpha >= 0.0) ? -nrm : nrm;
    const double num = (lane == 0) ? beta - alpha : 1.0;
    const double den = (lane == 0) ? beta : alpha - beta;
    const double q = num / den;
    tau = __shfl_sync(0xffffffffu, q, 0);
    scal = __shfl_sync(0xffffffffu, q, 1);
  }
  if (lane == 0) { bc[0] = tau; bc[1] = scal; bc[2] = beta; }
}

// The same scalars from one thread: tau, scal, beta into out[0..2] (the two
// divisions are independent, so their latencies overlap).
__device__ __forceinline__ void house_scalars(double alpha, double xn2, double* out) {
  double tau = 0.0, scal = 0.0, beta = alpha;
  if (xn2 != 0.0) {
    const double nrm = sqrt(fma(alpha, alpha, xn2));
    beta = (alpha >= 0.0) ? -nrm : nrm;
    tau = (beta - alpha) / beta;
    scal = 1.0 / (alpha - beta);
  }
  out[0] = tau; out[1] = scal; out[2] = beta;
}

// U (k x k, row-major, global or shared) <- pinv of the rank-r QRP truncation of
// G (k x k row-major, global).  smem: nucleus_smem_bytes(k).  Returns r.  When
// r >= rank_only_from only r is computed and U is left as it is (a staged run
// that will go on to a larger size needs the rank alone).
//
// Every arithmetic operation, and the order of every inner product, is the one
// the header comment states; what is parallel is only which thread runs which
// chain when.  A warp's FP64 instruction costs its SM sub-partition the same
// time whatever the number of active lanes, and one chain step costs that time,
// so the work is laid out by sub-partition: the pivot-search norms run on warps
// 0-1 while warps 2-3 run the norms the reflector needs (rows t+1..) and the
// reflector scalars each candidate would get (a square root and two divisions,
// about 1800 cycles of latency, that no longer follow the pivot search), the
// reflector products with the columns of Q^T run on warps 2-3 while warps 0-1
// run those with A's columns (Q^T is built during the QR, reflector by
// reflector, in the same order as after it), and the rank-1 updates y -= c v
// are spread over every thread.  CTAs of 64 threads run the second group's
// chains after the first's.
static __device__ __noinline__ int nucleus_cta(const double* G, int k, double tol, double* U, unsigned char* smem,
                                               int rank_only_from = KMAX + 1) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ld = nucleus_ld(k);
  const int bbase = nt >= 128 ? 64 : 0;                // first thread of the second group
  double* A = reinterpret_cast<double*>(smem);          // column-major k x k, stride ld
  double* Q = A + (size_t)k * ld;                       // Q^T, column-major
  double* T = Q + (size_t)k * ld;                       // T^T (k x r), column-major
  double* taus = T + (size_t)k * ld;
  double* tz = taus + KMAX;
  double* nrm = tz + KMAX;
  double* cw = nrm + KMAX;                              // 2 KMAX: tau (v^T y) per column of A, then of Q^T
  double* bc = cw + 2 * KMAX;
  double* hs = bc + KMAX;                               // 3 KMAX: tau, scal, beta per column
  int32_t* perm = reinterpret_cast<int32_t*>(hs + 3 * KMAX);
  int32_t* ctl = perm + KMAX;

  for (int it = tid; it < k * k; it += nt) {
    const int i = it / k, j = it - i * k;
    A[j * ld + i] = G[it];
    Q[j * ld + i] = (i == j) ? 1.0 : 0.0;
  }
  for (int j = tid; j < k; j += nt) perm[j] = j;
  __syncthreads();
  for (int t = 0; t < k; ++t) {
    const int nc = k - t;
    // squared norms of columns t.. over rows t.. (pivot search) and over rows
    // t+1.. (the reflector's ||x||^2 once the column is the pivot)
    if (tid < nc) {
      const double* col = A + (size_t)(t + tid) * ld;
      double s = 0.0;
      for (int i = t; i < k; ++i) s = fma(col[i], col[i], s);
      nrm[t + tid] = s;
    }
    {
      // and, from it, the reflector scalars every column would get as the
      // pivot (its sqrt and two divisions then stay off the pivot's path)
      const int g = tid - bbase;
      if (g >= 0 && g < nc) {
        const double* col = A + (size_t)(t + g) * ld;
        double s = 0.0;
        for (int i = t + 1; i < k; ++i) s = fma(col[i], col[i], s);
        house_scalars(col[t], s, hs + 3 * (t + g));
      }
    }
    __syncthreads();
    if (tid < 32) {
      // largest squared norm, lowest column on ties (integer keys, one warp)
      Cand c = cand_none();
      for (int j = t + tid; j < k; j += 32) cand_consider(c, mag_key(nrm[j]), 0, j);
      c = warp_best_local(c, 0);                     // every lane holds the winner
      const int pj = (c.key == 0ull) ? t : c.j;
      if (tid == 0) {
        ctl[0] = pj;
        taus[t] = hs[3 * pj];
        if (pj != t) { const int tp = perm[t]; perm[t] = perm[pj]; perm[pj] = tp; }
      }
    }
    __syncthreads();
    const int pj = ctl[0];
    const double tau = hs[3 * pj], scal = hs[3 * pj + 1], beta = hs[3 * pj + 2];
    // interchange columns t and pj; column t becomes beta e_t + v (v scaled)
    for (int i = tid; i < k; i += nt) {
      const double at = A[t * ld + i], ap = A[pj * ld + i];
      double nv = ap;
      if (tau != 0.0) {
        if (i > t) nv = ap * scal;
        else if (i == t) nv = beta;
      }
      A[t * ld + i] = nv;
      if (pj != t) A[pj * ld + i] = at;
    }
    __syncthreads();
    if (tau == 0.0) continue;                           // H_t = I: nothing to apply (uniform)
    const double* v = A + (size_t)t * ld;               // v[t] = 1 implicit, v[t+1..]
    // w = y[t] + v[t+1] y[t+1] + ... (ascending chain), c = tau w: columns t+1..
    // of A on the first group, the columns of Q^T on the second
    if (t + 1 + tid < k) {
      const double* y = A + (size_t)(t + 1 + tid) * ld;
      double w = y[t];
      for (int i = t + 1; i < k; ++i) w = fma(v[i], y[i], w);
      cw[t + 1 + tid] = tau * w;
    }
    {
      const int g = tid - bbase;
      if (g >= 0 && g < k) {
        const double* y = Q + (size_t)g * ld;
        double w = y[t];
        for (int i = t + 1; i < k; ++i) w = fma(v[i], y[i], w);
        cw[KMAX + g] = tau * w;
      }
    }
    __syncthreads();
    // y[t] -= c, y[i] = fma(-c, v[i], y[i]): every thread, one entry at a time
    {
      const int na = k - t - 1, ncol = na + k;
      for (int e = tid; e < ncol * nc; e += nt) {
        const int cix = e / nc, i = t + (e - cix * nc);
        double* y;
        double c;
        if (cix < na) { y = A + (size_t)(t + 1 + cix) * ld; c = cw[t + 1 + cix]; }
        else { y = Q + (size_t)(cix - na) * ld; c = cw[KMAX + cix - na]; }
        y[i] = fma(-c, (i == t) ? 1.0 : v[i], y[i]);     // i = t: y[t] - c, rounded once
      }
    }
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
  if (r >= rank_only_from) return r;                    // uniform; nothing below is needed
  for (int it = tid; it < k * k; it += nt) U[it] = 0.0;
  if (r == 0) { __syncthreads(); return 0; }

  if (r < k) {
    for (int it = tid; it < k * r; it += nt) {
      const int c = it / k, i = it - c * k;
      T[c * ld + i] = (i >= c) ? A[i * ld + c] : 0.0;
    }
    __syncthreads();
    // QR of T^T: reflector c from column c, applied to columns c+1..r-1
    for (int c = 0; c < r; ++c) {
      const int len = k - c;
      double* x = T + (size_t)c * ld;
      if (tid < 32) {
        double xn2 = 0.0;
        if (tid == 0)
          for (int i = c + 1; i < k; ++i) xn2 = fma(x[i], x[i], xn2);
        xn2 = __shfl_sync(0xffffffffu, xn2, 0);
        house_scalars_warp(x[c], xn2, bc);
        if (tid == 0) tz[c] = bc[0];
      }
      __syncthreads();
      const double tau = bc[0], scal = bc[1], beta = bc[2];
      if (tau == 0.0) { __syncthreads(); continue; }    // uniform; bc is rewritten next step
      for (int i = c + 1 + tid; i < k; i += nt) x[i] = x[i] * scal;
      if (tid == 0) x[c] = beta;
      __syncthreads();
      if (c + 1 + tid < r) {
        const double* y = T + (size_t)(c + 1 + tid) * ld;
        double w = y[c];
        for (int i = c + 1; i < k; ++i) w = fma(x[i], y[i], w);
        cw[c + 1 + tid] = tau * w;
      }
      __syncthreads();
      const int na = r - c - 1;
      for (int e = tid; e < na * len; e += nt) {
        const int cix = e / len, i = c + (e - cix * len);
        double* y = T + (size_t)(c + 1 + cix) * ld;
        const double cc = cw[c + 1 + cix];
        y[i] = fma(-cc, (i == c) ? 1.0 : x[i], y[i]);
      }
      __syncthreads();
    }
  }
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
    }
  }
  __syncthreads();
  if (r < k) {
    // v <- H'_0 ... H'_{r-1} v on every column: chains per column, updates by all threads
    for (int c = r - 1; c >= 0; --c) {
      const double tau = tz[c];
      if (tau == 0.0) continue;                         // uniform
      const double* x = T + (size_t)c * ld;
      const int len = k - c;
      if (tid < k) {
        const double* y = Q + (size_t)tid * ld;
        double w = y[c];
        for (int i = c + 1; i < k; ++i) w = fma(x[i], y[i], w);
        cw[tid] = tau * w;
      }
      __syncthreads();
      for (int e = tid; e < k * len; e += nt) {
        const int col = e / len, i = c + (e - col * len);
        double* y = Q + (size_t)col * ld;
        const double cc = cw[col];
        y[i] = fma(-cc, (i == c) ? 1.0 : x[i], y[i]);
      }
      __syncthreads();
    }
  }
  for (int it = tid; it < k * k; it += nt) {
    const int i = it / k, col = it - i * k;
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
