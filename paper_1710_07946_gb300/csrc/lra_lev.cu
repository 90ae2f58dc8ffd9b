// lra_lev.cu -- C-A iterations whose steps select by DMM08 Algorithm 1 on the
// sketches (the paper's tests of C-A incorporating [DMM08, Algorithm 1]), for a
// batch of blocks, one CTA per block from a work queue.
//
// Per block, iters times: the horizontal sketch W[I, :] (kI x n), its SVD-based
// leverage scores (eq. eqlevsc, beta = 1: the Gram matrix A A^T diagonalised by
// round-robin Jacobi sweeps, the top-r eigenpairs above 1e-12 of the largest,
// v_j = sum (u_t . a_j)^2 / sigma_t^2), l = k columns sampled by Exactly(l)
// (Algorithm algsmplex: inverse CDF of the caller's uniform draws) or
// Expected(l) (Algorithm algsmplexp); then the same on the vertical sketch
// W[:, J] for the rows.  Finally U = pinv of the rank-r QRP truncation of
// W[I, J], C = W[:, J], R = W[I, :].  Every floating-point step is the oracle's
// operation for operation (sequential sums where the oracle sums sequentially),
// so the sampled indices match bit for bit.  With uniform scores (kind 2, 3) the
// SVD stage is skipped and every score is 1: for perturbed factor-Gaussian
// inputs with r << n the leverage scores are nearly equal, which is how the
// paper makes that stage superfast.
#include <algorithm>
#include <cstring>

#include "lra_device.cuh"
#include "lra_internal.h"
#include "lra_nucleus.cuh"
#include "lra_profile.h"

namespace lra {

constexpr int LEV_JAC_SWEEPS = 10;
constexpr double LEV_EIG_TOL = 1e-12;

struct LevArgs {
  DevProblem base;
  const int64_t* blocks;   // nb x 4
  const int64_t* offs;     // nb x 2: offsets of C_b (nrows x k) and R_b (k x ncols)
  const int32_t* order;
  int32_t nb, k, r, iters, kind;
  double rank_tol;
  const int32_t* I0;       // nb x k
  const double* draws;     // nb x (2 iters) x max_len uniforms in [0, 1)
  int32_t* I;              // nb x k
  int32_t* J;              // nb x k
  double* C;
  double* R;
  double* U;               // nb x k x k (kJ x kI used)
  int32_t* info;           // nb x LRA_INFO_LEN
  unsigned int* counter;
  double* scratch;         // per CTA: sketch (k x max_len), v, cum (max_len each), G (k x k), flags (max_len ints)
  size_t scratch_stride;
  int64_t max_len;
};

__device__ __forceinline__ void lev_pair(int kp, int t, int i, int& p, int& q) {
  const int a = (i == 0) ? 0 : 1 + (t + i) % (kp - 1);
  const int b = 1 + (t + kp - 1 - i) % (kp - 1);
  p = a < b ? a : b;
  q = a < b ? b : a;
}

// Round-robin Jacobi on the symmetric k x k G (shared, row-major, ld k): every
// rotation of a round from G at the round's start, then all row pairs, then all
// column pairs and the columns of Q; after each sweep, stop when the largest
// off-diagonal |G| is at most 2^-48 times the largest diagonal |G| (maxima of
// absolute values: the same decision in any evaluation order).
__device__ void lev_jacobi(double* G, double* Q, double* cs, double* red, int k) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int kp = k + (k & 1), half = kp / 2;
  for (int e = tid; e < k * k; e += nt) Q[e] = (e / k == e % k) ? 1.0 : 0.0;
  __syncthreads();
  for (int sw = 0; sw < LEV_JAC_SWEEPS; ++sw) {
    for (int t = 0; t < kp - 1; ++t) {
      for (int i = tid; i < half; i += nt) {
        int p, q;
        lev_pair(kp, t, i, p, q);
        double c = 1.0, sn = 0.0;
        if (q < k && G[p * k + q] != 0.0) {
          const double tau = (G[q * k + q] - G[p * k + p]) / (2.0 * G[p * k + q]);
          const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + tt * tt);
          sn = tt * c;
        }
        cs[2 * i] = c;
        cs[2 * i + 1] = sn;
      }
      __syncthreads();
      for (int e = tid; e < half * k; e += nt) {
        const int i = e / k, j = e - i * k;
        int p, q;
        lev_pair(kp, t, i, p, q);
        if (q >= k) continue;
        const double c = cs[2 * i], sn = cs[2 * i + 1];
        const double x = G[p * k + j], y = G[q * k + j];
        G[p * k + j] = c * x - sn * y;
        G[q * k + j] = sn * x + c * y;
      }
      __syncthreads();
      for (int e = tid; e < half * k; e += nt) {
        const int i = e / k, j = e - i * k;
        int p, q;
        lev_pair(kp, t, i, p, q);
        if (q >= k) continue;
        const double c = cs[2 * i], sn = cs[2 * i + 1];
        const double x = G[j * k + p], y = G[j * k + q];
        G[j * k + p] = c * x - sn * y;
        G[j * k + q] = sn * x + c * y;
        const double xq = Q[j * k + p], yq = Q[j * k + q];
        Q[j * k + p] = c * xq - sn * yq;
        Q[j * k + q] = sn * xq + c * yq;
      }
      __syncthreads();
    }
    double off = 0.0, dmax = 0.0;
    for (int e = tid; e < k * k; e += nt) {
      const int p = e / k, q = e - p * k;
      if (p == q) dmax = fmax(dmax, fabs(G[e]));
      else if (p < q) off = fmax(off, fabs(G[e]));
    }
    for (int o = 16; o > 0; o >>= 1) {
      off = fmax(off, __shfl_xor_sync(0xffffffffu, off, o));
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    }
    if ((tid & 31) == 0) { red[2 * (tid >> 5)] = off; red[2 * (tid >> 5) + 1] = dmax; }
    __syncthreads();
    off = 0.0;
    dmax = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) { off = fmax(off, red[2 * w]); dmax = fmax(dmax, red[2 * w + 1]); }
    __syncthreads();
    if (off <= ldexp(1.0, -48) * dmax) break;
  }
}

// Scores v_j of the n columns of the kS x n sketch S (global, row-major) for
// rank r: Gram matrix, Jacobi, top eigenpairs, squared projections.  Returns
// the number of eigenpairs used (in every thread).
__device__ int lev_scores(const double* S, int kS, int64_t n, int r, double* G, double* Q, double* tile, double* cs,
                          int* sel, int* s_re, double* v) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int npair = kS * (kS + 1) / 2;
  // Gram matrix over 32-column tiles of S staged in shared memory (tile: kS x
  // 33 doubles): every entry is still one ascending chain over the columns
  for (int e = tid; e < npair; e += nt) {
    int a = 0, rem = e;
    while (rem >= kS - a) { rem -= kS - a; ++a; }
    G[a * kS + a + rem] = 0.0;
  }
  for (int64_t j0 = 0; j0 < n; j0 += 32) {
    const int w = (int)min((int64_t)32, n - j0);
    __syncthreads();
    for (int e = tid; e < kS * 32; e += nt) {
      const int a = e >> 5, jj = e & 31;
      tile[a * 33 + jj] = jj < w ? S[(int64_t)a * n + j0 + jj] : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < npair; e += nt) {
      int a = 0, rem = e;
      while (rem >= kS - a) { rem -= kS - a; ++a; }
      const int b = a + rem;
      double acc = G[a * kS + b];
      for (int jj = 0; jj < w; ++jj) acc = fma(tile[a * 33 + jj], tile[b * 33 + jj], acc);
      G[a * kS + b] = acc;
    }
  }
  __syncthreads();
  for (int e = tid; e < npair; e += nt) {
    int a = 0, rem = e;
    while (rem >= kS - a) { rem -= kS - a; ++a; }
    G[(a + rem) * kS + a] = G[a * kS + a + rem];
  }
  __syncthreads();
  lev_jacobi(G, Q, cs, tile, kS);
  if (tid == 0) {
    int re = 0;
    double dmax = 0.0;
    for (int t = 0; t < r && t < kS; ++t) {
      int best = -1;
      for (int a = 0; a < kS; ++a) {
        bool used = false;
        for (int u = 0; u < re; ++u) used = used || sel[u] == a;
        if (!used && (best < 0 || G[a * kS + a] > G[best * kS + best])) best = a;
      }
      if (best < 0 || !(G[best * kS + best] > 0.0)) break;
      if (t == 0) dmax = G[best * kS + best];
      else if (G[best * kS + best] < LEV_EIG_TOL * dmax) break;
      sel[re++] = best;
    }
    *s_re = re;
  }
  __syncthreads();
  const int re = *s_re;
  for (int64_t j = tid; j < n; j += nt) {
    double acc = 0.0;
    for (int t = 0; t < re; ++t) {
      const int c = sel[t];
      double e = 0.0;
      for (int a = 0; a < kS; ++a) e = fma(Q[a * kS + c], S[(int64_t)a * n + j], e);
      const double w = e * e;
      acc = acc + w / G[c * kS + c];
    }
    v[j] = acc;
  }
  __syncthreads();
  return re;
}

// Exactly(l) (kind 0) or Expected(l) (kind 1) sampling of out[] from the scores
// v (n), with the uniforms u.  Returns the count (in every thread).
__device__ int lev_sample(const double* v, int64_t n, int l, int kind, const double* u, double* cum, int* flags,
                          int32_t* out, int* s_cnt, double* s_tot, long long* s_last) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    double c = 0.0;
    long long last = -1;
    for (int64_t j = 0; j < n; ++j) {
      c = c + v[j];
      cum[j] = c;
      if (v[j] > 0.0) last = j;
    }
    *s_tot = c;
    *s_last = last;
  }
  __syncthreads();
  const double total = *s_tot;
  const long long last = *s_last;
  if (!(total > 0.0) || last < 0) {
    const int cnt = (int)min((int64_t)l, n);
    for (int t = tid; t < cnt; t += nt) out[t] = t;
    __syncthreads();
    return cnt;
  }
  if (kind == 0) {
    for (int t = tid; t < l; t += nt) {
      const double target = u[t] * total;
      int64_t lo = 0, hi = n;
      while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (cum[mid] > target) hi = mid;
        else lo = mid + 1;
      }
      out[t] = (int32_t)(lo < n ? lo : last);
    }
    __syncthreads();
    return l;
  }
  for (int64_t j = tid; j < n; j += nt) {
    double pr = ((double)l * v[j]) / total;
    if (pr > 1.0) pr = 1.0;
    flags[j] = (u[j] < pr) ? 1 : 0;
  }
  __syncthreads();
  if (tid == 0) {
    int cnt = 0;
    for (int64_t j = 0; j < n && cnt < l; ++j)
      if (flags[j]) out[cnt++] = (int32_t)j;
    if (cnt == 0) {
      int64_t best = 0;
      for (int64_t j = 1; j < n; ++j)
        if (v[j] > v[best]) best = j;
      out[cnt++] = (int32_t)best;
    }
    *s_cnt = cnt;
  }
  __syncthreads();
  return *s_cnt;
}

__global__ void __launch_bounds__(NT, 1) lev_batched_kernel(LevArgs B) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_b, s_re, s_cnt, s_bad;
  __shared__ double s_tot;
  __shared__ long long s_last;
  __shared__ double s_cs[KMAX + 2];
  __shared__ int s_sel[KMAX];
  __shared__ int32_t s_I[KMAX], s_J[KMAX];
  const int tid = threadIdx.x, nt = blockDim.x, k = B.k;
  double* Gs = reinterpret_cast<double*>(smem);               // k x k
  double* Qs = Gs + (size_t)k * k;                             // k x k
  double* Ts = Qs + (size_t)k * k;                             // k x 33: Gram tiles
  double* S = B.scratch + (size_t)blockIdx.x * B.scratch_stride;
  double* v = S + (size_t)k * B.max_len;
  double* cum = v + B.max_len;
  double* Gn = cum + B.max_len;                                // k x k (the core for the nucleus)
  int* flags = reinterpret_cast<int*>(Gn + (size_t)k * k);
  for (;;) {
    if (tid == 0) {
      const unsigned int qh = atomicAdd(B.counter, 1u);
      s_b = (qh < (unsigned)B.nb) ? (B.order ? B.order[qh] : (int)qh) : -1;
    }
    __syncthreads();
    const int b = s_b;
    __syncthreads();
    if (b < 0) break;
    int32_t* info = B.info + LRA_INFO_LEN * (size_t)b;
    const int64_t r0 = B.blocks[4 * (size_t)b], nr = B.blocks[4 * (size_t)b + 1];
    const int64_t c0 = B.blocks[4 * (size_t)b + 2], nc = B.blocks[4 * (size_t)b + 3];
    const int32_t* I0b = B.I0 + (size_t)b * k;
    bool bad = r0 < 0 || c0 < 0 || nr < k || nc < k || r0 + nr > B.base.m || c0 + nc > B.base.n ||
               nr > B.max_len || nc > B.max_len;
    if (tid == 0) {
      int v0 = 0;
      for (int a = 0; a < k && !bad; ++a) v0 |= (I0b[a] < 0 || I0b[a] >= nr);
      s_bad = v0;
    }
    __syncthreads();
    bad = bad || s_bad != 0;
    __syncthreads();
    if (bad) {
      for (int e = tid; e < LRA_INFO_LEN; e += nt) info[e] = (e == 3) ? LRA_ERR_INVALID_ARG : 0;
      continue;
    }
    DevProblem P = B.base;
    P.m = nr;
    P.n = nc;
    if (P.src == LRA_DENSE) {
      const size_t esz = (P.dtype == LRA_F32) ? 4 : 8;
      P.W = static_cast<const unsigned char*>(B.base.W) + (size_t)(r0 * B.base.ldw + c0) * esz;
    } else {
      P.X = B.base.X + 3 * r0;
      P.Y = B.base.Y + 3 * c0;
    }
    const double* ub = B.draws + (size_t)b * 2 * B.iters * B.max_len;
    for (int a = tid; a < k; a += nt) s_I[a] = I0b[a];
    int kI = k, kJ = 0, st = LRA_OK;
    __syncthreads();
    for (int it = 0; it < B.iters && st != LRA_ERR_NONFINITE; ++it) {
      for (int dir = 0; dir < 2; ++dir) {
        const int kS = dir == 0 ? kI : kJ;
        const int64_t len = dir == 0 ? nc : nr;
        if (tid == 0) s_bad = 0;
        __syncthreads();
        for (int64_t e = tid; e < (int64_t)kS * len; e += nt) {
          const int a = (int)(e / len);
          const int64_t c = e - (int64_t)a * len;
          const double x = dir == 0 ? wp_entry(P, s_I[a], c) : wp_entry(P, c, s_J[a]);
          if (!bits_finite(x)) s_bad = 1;
          S[e] = x;
        }
        __syncthreads();
        if (s_bad) { st = LRA_ERR_NONFINITE; break; }
        if (B.kind & 2) {
          // uniform scores (the SVD stage bypassed): v_j = 1
          for (int64_t j = tid; j < len; j += nt) v[j] = 1.0;
          __syncthreads();
        } else {
          const int re = lev_scores(S, kS, len, min(B.r, kS), Gs, Qs, Ts, s_cs, s_sel, &s_re, v);
          if (re == 0) st = max(st, (int)LRA_WARN_RANK_DEFICIENT);
        }
        const double* u = ub + (size_t)(2 * it + dir) * B.max_len;
        const int cnt = lev_sample(v, len, k, B.kind & 1, u, cum, flags, dir == 0 ? s_J : s_I, &s_cnt, &s_tot,
                                   &s_last);
        if (dir == 0) kJ = cnt;
        else kI = cnt;
      }
    }
    if (st == LRA_ERR_NONFINITE) {
      if (tid == 0) {
        info[0] = 0; info[1] = 0; info[2] = 0; info[3] = st; info[4] = 0; info[5] = 0; info[6] = kI; info[7] = kJ;
      }
      __syncthreads();
      continue;
    }
    // outputs: C = W[:, J] (nr x kJ), R = W[I, :] (kI x nc), the core G = W[I, J]
    double* Cb = B.C + B.offs[2 * (size_t)b];
    double* Rb = B.R + B.offs[2 * (size_t)b + 1];
    for (int64_t e = tid; e < nr * kJ; e += nt) {
      const int64_t i = e / kJ;
      const int a = (int)(e - i * kJ);
      Cb[e] = c_entry(P, i, s_J[a]);
    }
    for (int64_t e = tid; e < (int64_t)kI * nc; e += nt) {
      const int a = (int)(e / nc);
      const int64_t c = e - (int64_t)a * nc;
      Rb[e] = r_entry(P, s_I[a], c);
    }
    const bool tr = kI > kJ;
    for (int e = tid; e < kI * kJ; e += nt) {
      const int a = e / kJ, c = e - a * kJ;
      const double g = wp_entry(P, s_I[a], s_J[c]);
      if (tr) Gn[c * kI + a] = g;
      else Gn[e] = g;
    }
    for (int a = tid; a < k; a += nt) {
      B.I[(size_t)b * k + a] = a < kI ? s_I[a] : 0;
      B.J[(size_t)b * k + a] = a < kJ ? s_J[a] : 0;
    }
    __syncthreads();
    double* Ub = B.U + (size_t)b * k * k;
    int rank;
    if (!tr) {
      rank = nucleus_rect_cta(Gn, kI, kJ, B.rank_tol, Ub, smem);         // kJ x kI
    } else {
      // pinv(G) = pinv(G^T)^T: the kI x kJ result goes to the scratch, then transposed into U
      rank = nucleus_rect_cta(Gn, kJ, kI, B.rank_tol, S, smem);
      __syncthreads();
      for (int e = tid; e < kI * kJ; e += nt) {
        const int bcol = e / kI, a = e - bcol * kI;
        Ub[e] = S[(size_t)a * kJ + bcol];
      }
    }
    __syncthreads();
    if (tid == 0) {
      if (rank < min(kI, kJ) && st == LRA_OK) st = LRA_WARN_RANK_DEFICIENT;
      info[0] = rank; info[1] = 0; info[2] = B.iters; info[3] = st; info[4] = 0; info[5] = 0; info[6] = kI;
      info[7] = kJ;
    }
    __syncthreads();
  }
}

struct LevPlan {
  int grid;
  size_t smem, stride, bytes;
};

static lra_status lev_plan(int k, int64_t max_len, LevPlan* pl) {
  DeviceInfo dev;
  lra_status st = current_device_info(&dev);
  if (st != LRA_OK) return st;
  const size_t need = std::max(sizeof(double) * (2 * (size_t)k * k + 33 * (size_t)k), nucleus_rect_smem_bytes(k, k));
  if (need > dev.smem_optin - 8192) return LRA_ERR_INVALID_ARG;
  LRA_CUDA_TRY(cudaFuncSetAttribute(lev_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
  int occ = 0;
  LRA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lev_batched_kernel, NT, need));
  if (occ < 1) return LRA_ERR_INVALID_ARG;
  pl->grid = occ * dev.sms;
  pl->smem = need;
  // sketch k x max_len, v and cum (max_len each), core k x k, flags (max_len ints)
  pl->stride = align_up((size_t)(k + 2) * max_len + (size_t)k * k + (size_t)(max_len + 1) / 2 + 1, 32);
  pl->bytes = align_up(256 + sizeof(double) * pl->stride * pl->grid, 256);
  return LRA_OK;
}

static lra_status lev_check(const lra_problem* base, const lra_batch* batch, int32_t k, int32_t r, int32_t iters,
                            int32_t kind, DevProblem* P) {
  lra_status st = make_dev_problem(base, nullptr, P);
  if (st != LRA_OK) return st;
  if (batch == nullptr || batch->blocks == nullptr || batch->offsets == nullptr || batch->nb < 1 ||
      batch->max_len < 1)
    return LRA_ERR_INVALID_ARG;
  if (k < 1 || k > KMAX || r < 1 || r > k || iters < 1 || kind < 0 || kind > 3) return LRA_ERR_INVALID_ARG;
  return LRA_OK;
}

}  // namespace lra

using namespace lra;

extern "C" {

lra_status lra_ca_lev_batched_workspace_size(const lra_problem* base, const lra_batch* batch, int32_t k, int32_t r,
                                             int32_t iters, int32_t kind, size_t* bytes) {
  if (bytes == nullptr) return LRA_ERR_INVALID_ARG;
  DevProblem P;
  lra_status st = lev_check(base, batch, k, r, iters, kind, &P);
  if (st != LRA_OK) return st;
  LevPlan pl;
  if ((st = lev_plan(k, batch->max_len, &pl)) != LRA_OK) return st;
  *bytes = pl.bytes;
  return LRA_OK;
}

lra_status lra_ca_lev_batched(const lra_problem* base, const lra_batch* batch, int32_t k, int32_t r, int32_t iters,
                              int32_t kind, double rank_tol, const int32_t* I0, const double* draws,
                              const lra_cur_batch* out, void* workspace, size_t workspace_bytes,
                              lra_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  DevProblem P;
  lra_status st = lev_check(base, batch, k, r, iters, kind, &P);
  if (st != LRA_OK) return st;
  if (!(rank_tol >= 0.0) || !(rank_tol < 1.0) || I0 == nullptr || draws == nullptr || out == nullptr || !out->I ||
      !out->J || !out->C || !out->U || !out->R || !out->info)
    return LRA_ERR_INVALID_ARG;
  LevPlan pl;
  if ((st = lev_plan(k, batch->max_len, &pl)) != LRA_OK) return st;
  if (workspace == nullptr || workspace_bytes < pl.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return LRA_ERR_WORKSPACE;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  LevArgs A;
  std::memset(&A, 0, sizeof(A));
  A.base = P;
  A.blocks = batch->blocks;
  A.offs = batch->offsets;
  A.order = batch->order;
  A.nb = batch->nb;
  A.k = k;
  A.r = r;
  A.iters = iters;
  A.kind = kind;
  A.rank_tol = rank_tol;
  A.I0 = I0;
  A.draws = draws;
  A.I = out->I;
  A.J = out->J;
  A.C = out->C;
  A.R = out->R;
  A.U = out->U;
  A.info = out->info;
  A.counter = reinterpret_cast<unsigned int*>(ws);
  A.scratch = reinterpret_cast<double*>(ws + 256);
  A.scratch_stride = pl.stride;
  A.max_len = batch->max_len;
  LRA_CUDA_TRY(cudaMemsetAsync(ws, 0, 256, stream));
  {
    LaunchScope ls(stream, "lev_batched_kernel");
    lev_batched_kernel<<<pl.grid, NT, pl.smem, stream>>>(A);
  }
  return cuda_status(cudaGetLastError());
}

}  // extern "C"
