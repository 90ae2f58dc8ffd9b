// lra_ca_core.cuh -- one maxvol step of cross-approximation and the whole C-A
// loop, written once over a "group" of CTAs that share the search (a single CTA,
// or every CTA of a cooperative grid).
//
// Paper: Algorithm algdomin (dominant submatrix by swaps), Algorithm alggos (its
// LUP initialisation), the C-A loop of Section "CUR LRA; primitive, cynical, and
// cross-approximation algorithms" in the Tests 2 schedule (random initial rows,
// horizontal step then vertical step, warm start of every later step).
//
// Data layout.  A maxvol step works on a k x len strip: the row strip W'[I,:]
// (len = n, strip row a = row I[a] of W') or the transposed column strip
// W'[:,J]^T (len = m, strip row a = column J[a] of W').  The strip's columns are
// split into contiguous chunks, one per CTA of the group; a CTA holds its chunk
// k x qn, row-major with leading dimension ldm, in shared memory (or in its part
// of a global scratch area when the chunk is too large).  The chunk is gathered
// straight from W (dense, with the multiplier's column combinations fused, or
// from the kernel entry oracle): no strip is materialised elsewhere.
//
// A warm start needs B = strip[:, Jw] only; every CTA gathers those k columns
// itself and replays the same pivoted LU of B, so a warm step exchanges nothing
// until its first swap test.  A cold step exchanges once per elimination step
// (global pivot search), and the swap loop once per swap.
#pragma once

#include "lra_device.cuh"

namespace lra {

struct CaArgs {
  DevProblem P;
  int32_t k, sweeps, max_swaps;
  double h;
  const int32_t* I0;
  int32_t* I;
  int32_t* J;
  double* C;           // m x k
  double* R;           // k x n
  double* logvol;      // 2*sweeps
  int32_t* info;       // rank, swaps, loops, status
  double* G;           // k x k core W'[I,J] for the nucleus (workspace)
  double* gstrip;      // global chunks when not in shared memory (nblk * k * ldm)
  int32_t chunk_n, chunk_m, ldm;
  int32_t strip_in_smem;
};

// Shared-memory layout of the C-A kernels (all offsets in bytes, 16-aligned).
struct CaSmem {
  double* LU;        // k*k : U0 (cold) or the pivoted LU of B (warm)
  double* x;         // KMAX : the exchanged column
  double* lmul;      // KMAX : multipliers of the current elimination step
  double* tq;        // ldm  : per-column scratch (swap ratios)
  int32_t* Is;       // KMAX : current rows I
  int32_t* Js;       // KMAX : current columns J
  int32_t* piv;      // KMAX : row interchanges of the warm LU
  int32_t* pos;      // ldm  : 0 = unchosen, else 1 + position in the selected set
  Cand* win;         // the winner of the last exchange
  unsigned long long* flags;
  int32_t* ctl;      // small control words
  double* M;         // the chunk (k x ldm), shared or global
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

__host__ __device__ inline size_t ca_smem_fixed(int k, int ldm) {
  size_t b = 0;
  b += align16(sizeof(double) * (size_t)k * k);
  b += align16(sizeof(double) * KMAX) * 2;
  b += align16(sizeof(double) * (size_t)ldm);
  b += align16(sizeof(int32_t) * KMAX) * 3;
  b += align16(sizeof(int32_t) * (size_t)ldm);
  b += align16(sizeof(Cand));
  b += align16(sizeof(unsigned long long));
  b += align16(sizeof(int32_t) * 8);
  return b;
}

__device__ inline CaSmem ca_smem_carve(unsigned char* base, int k, int ldm, double* gchunk) {
  CaSmem S;
  size_t o = 0;
  S.LU = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * (size_t)k * k);
  S.x = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * KMAX);
  S.lmul = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * KMAX);
  S.tq = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * (size_t)ldm);
  S.Is = reinterpret_cast<int32_t*>(base + o); o += align16(sizeof(int32_t) * KMAX);
  S.Js = reinterpret_cast<int32_t*>(base + o); o += align16(sizeof(int32_t) * KMAX);
  S.piv = reinterpret_cast<int32_t*>(base + o); o += align16(sizeof(int32_t) * KMAX);
  S.pos = reinterpret_cast<int32_t*>(base + o); o += align16(sizeof(int32_t) * (size_t)ldm);
  S.win = reinterpret_cast<Cand*>(base + o); o += align16(sizeof(Cand));
  S.flags = reinterpret_cast<unsigned long long*>(base + o); o += align16(sizeof(unsigned long long));
  S.ctl = reinterpret_cast<int32_t*>(base + o); o += align16(sizeof(int32_t) * 8);
  S.M = gchunk ? gchunk : reinterpret_cast<double*>(base + o);
  return S;
}

// Strip entry (a, q): phase 0 = row strip W'[I[a], q]; phase 1 = W'[q, J[a]].
__device__ __forceinline__ double strip_entry(const DevProblem& P, int phase, const int32_t* Is, const int32_t* Js,
                                              int a, int64_t q) {
  return phase == 0 ? wp_entry(P, Is[a], q) : wp_entry(P, q, Js[a]);
}

// Result of one maxvol step.
struct StepResult {
  int status;       // LRA_OK, LRA_WARN_*, or an error
  int nswaps;
  double logdet;
};

// One maxvol step over the k x len strip of `phase`.  Jsel: in = warm set (ignored
// when cold), out = selected k strip columns in generator order.  seq: exchange
// round counter, advanced identically in every CTA of the group.
template <class Group>
__device__ StepResult maxvol_step(const Group& grp, const CaArgs& A, const CaSmem& S, int phase, bool cold,
                                  int32_t* Jsel, unsigned long long& seq) {
  const DevProblem& P = A.P;
  const int k = A.k, ldm = A.ldm, tid = threadIdx.x, nt = blockDim.x;
  const int64_t len = phase == 0 ? P.n : P.m;
  const int chunk = phase == 0 ? A.chunk_n : A.chunk_m;
  const int64_t q0 = (int64_t)grp.rank() * chunk;
  const int qn = (int)max((int64_t)0, min((int64_t)chunk, len - q0));
  double* M = S.M;
  StepResult res{LRA_OK, 0, 0.0};

  // gather the chunk; flag non-finite entries
  int nonfinite = 0;
  for (int it = tid; it < k * qn; it += nt) {
    int a = it / qn, c = it - a * qn;
    double v = strip_entry(P, phase, S.Is, S.Js, a, q0 + c);
    M[(int64_t)a * ldm + c] = v;
    if (!isfinite(v)) nonfinite = 1;
  }
  for (int c = tid; c < qn; c += nt) S.pos[c] = 0;
  if (tid == 0) { S.ctl[0] = 0; S.ctl[1] = 0; }
  __syncthreads();
  if (nonfinite) atomicOr(&S.ctl[0], 1);
  __syncthreads();
  unsigned long long myflags = S.ctl[0] ? FLAG_NONFINITE : 0ull;
  double logdet = 0.0;
  bool deficient = false;

  if (!cold) {
    // ---- warm start: B = strip[:, Jsel]; pivoted LU of B replayed by every CTA
    for (int it = tid; it < k * k; it += nt) {
      int a = it / k, t = it - a * k;
      S.LU[a * k + t] = strip_entry(P, phase, S.Is, S.Js, a, Jsel[t]);
    }
    __syncthreads();
    int fallback = 0;
    for (int t = 0; t < k; ++t) {
      if (tid == 0) {
        int r = t;
        double bv = fabs(S.LU[t * k + t]);
        for (int p = t + 1; p < k; ++p) {
          double v = fabs(S.LU[p * k + t]);
          if (v > bv) { bv = v; r = p; }
        }
        S.piv[t] = r;
      }
      __syncthreads();
      // interchange rows t and r in columns t.. only: column t' < t keeps the
      // multipliers of step t' in the row positions of that step, which is the
      // order in which they are replayed on the CTA's own columns below
      const int r = S.piv[t];
      if (r != t)
        for (int j = t + tid; j < k; j += nt) {
          double tmp = S.LU[t * k + j]; S.LU[t * k + j] = S.LU[r * k + j]; S.LU[r * k + j] = tmp;
        }
      __syncthreads();
      const double pv = S.LU[t * k + t];
      if (pv == 0.0) { fallback = 1; break; }     // same decision in every CTA
      for (int p = t + 1 + tid; p < k; p += nt) S.LU[p * k + t] = S.LU[p * k + t] / pv;
      __syncthreads();
      const int w = k - t - 1;
      for (int it = tid; it < w * w; it += nt) {
        int p = t + 1 + it / w, j = t + 1 + it % w;
        S.LU[p * k + j] = fma(-S.LU[p * k + t], S.LU[t * k + j], S.LU[p * k + j]);
      }
      __syncthreads();
    }
    if (fallback) {
      cold = true;
      __syncthreads();
    } else {
      for (int t = 0; t < k; ++t) {
        int64_t jt = Jsel[t];
        if (jt >= q0 && jt < q0 + qn && tid == 0) S.pos[jt - q0] = t + 1;
      }
      __syncthreads();
      for (int t = 0; t < k; ++t) {
        const int r = S.piv[t];
        if (r != t)
          for (int c = tid; c < qn; c += nt) {
            double tmp = M[(int64_t)t * ldm + c];
            M[(int64_t)t * ldm + c] = M[(int64_t)r * ldm + c];
            M[(int64_t)r * ldm + c] = tmp;
          }
        __syncthreads();
        const int w = k - t - 1;
        for (int it = tid; it < w * qn; it += nt) {
          int p = t + 1 + it / qn, c = it - (p - t - 1) * qn;
          if (S.pos[c] == 0)
            M[(int64_t)p * ldm + c] = fma(-S.LU[p * k + t], M[(int64_t)t * ldm + c], M[(int64_t)p * ldm + c]);
        }
        __syncthreads();
      }
      for (int t = 0; t < k; ++t) logdet += log(fabs(S.LU[t * k + t]));
    }
  }

  if (cold) {
    // ---- cold start: LU with column pivoting over the whole strip
    for (int t = 0; t < k; ++t) {
      Cand mine = cand_none();
      for (int c = tid; c < qn; c += nt) {
        if (S.pos[c]) continue;
        double v = fabs(M[(int64_t)t * ldm + c]);
        if (v > mine.v) { mine.v = v; mine.i = 0; mine.j = (int32_t)(q0 + c); }
      }
      __shared__ Cand red[33];
      mine = block_best(mine, red);
      const double* mycol = (mine.j != 0x7fffffff) ? M + (mine.j - q0) : nullptr;
      if (!grp.exchange(seq, mine, mycol, ldm, k, myflags, S.win, S.x, S.flags, chunk)) {
        res.status = LRA_ERR_TIMEOUT;
        return res;
      }
      ++seq;
      if (*S.flags & FLAG_NONFINITE) { res.status = LRA_ERR_NONFINITE; return res; }
      const Cand w = *S.win;
      if (tid == 0) {
        Jsel[t] = w.j;
        if (w.j >= q0 && w.j < q0 + qn) S.pos[w.j - q0] = t + 1;
      }
      const double pv = S.x[t];
      if (pv == 0.0) { deficient = true; __syncthreads(); continue; }
      for (int p = tid; p <= t; p += nt) S.LU[p * k + t] = S.x[p];
      for (int p = t + 1 + tid; p < k; p += nt) S.lmul[p] = S.x[p] / pv;
      __syncthreads();
      const int wrows = k - t - 1;
      for (int it = tid; it < wrows * qn; it += nt) {
        int p = t + 1 + it / qn, c = it - (p - t - 1) * qn;
        if (S.pos[c] == 0)
          M[(int64_t)p * ldm + c] = fma(-S.lmul[p], M[(int64_t)t * ldm + c], M[(int64_t)p * ldm + c]);
      }
      logdet += log(fabs(pv));
      __syncthreads();
    }
    if (deficient) {
      res.status = LRA_WARN_RANK_DEFICIENT;
      res.logdet = -INFINITY;
      return res;
    }
  }

  // ---- C = (I | U0^{-1} U1): column-sweep back substitution on unchosen columns
  for (int i = k - 1; i >= 0; --i) {
    const double d = S.LU[i * k + i];
    for (int c = tid; c < qn; c += nt)
      if (S.pos[c] == 0) M[(int64_t)i * ldm + c] = M[(int64_t)i * ldm + c] / d;
    __syncthreads();
    for (int it = tid; it < i * qn; it += nt) {
      int p = it / qn, c = it - p * qn;
      if (S.pos[c] == 0)
        M[(int64_t)p * ldm + c] = fma(-S.LU[p * k + i], M[(int64_t)i * ldm + c], M[(int64_t)p * ldm + c]);
    }
    __syncthreads();
  }
  for (int it = tid; it < k * qn; it += nt) {
    int a = it / qn, c = it - a * qn;
    if (S.pos[c]) M[(int64_t)a * ldm + c] = (S.pos[c] - 1 == a) ? 1.0 : 0.0;
  }
  __syncthreads();

  // ---- dominance swaps (Algorithm algdomin)
  int nsw = 0;
  for (;;) {
    Cand mine = cand_none();
    for (int c = tid; c < qn; c += nt) {
      if (S.pos[c]) continue;
      for (int a = 0; a < k; ++a) {
        double v = fabs(M[(int64_t)a * ldm + c]);
        if (v > mine.v) { mine.v = v; mine.i = a; mine.j = (int32_t)(q0 + c); }
      }
    }
    __shared__ Cand red2[33];
    mine = block_best(mine, red2);
    const double* mycol = (mine.j != 0x7fffffff) ? M + (mine.j - q0) : nullptr;
    if (!grp.exchange(seq, mine, mycol, ldm, k, myflags, S.win, S.x, S.flags, chunk)) {
      res.status = LRA_ERR_TIMEOUT;
      return res;
    }
    ++seq;
    if (*S.flags & FLAG_NONFINITE) { res.status = LRA_ERR_NONFINITE; return res; }
    const Cand w = *S.win;
    if (w.j == 0x7fffffff || !(w.v > A.h)) break;
    if (nsw >= A.max_swaps) { res.status = LRA_WARN_NOT_CONVERGED; break; }
    const double cs = S.x[w.i];
    for (int c = tid; c < qn; c += nt) S.tq[c] = M[(int64_t)w.i * ldm + c] / cs;
    __syncthreads();
    for (int it = tid; it < k * qn; it += nt) {
      int p = it / qn, c = it - p * qn;
      if (p == w.i) M[(int64_t)p * ldm + c] = S.tq[c];
      else M[(int64_t)p * ldm + c] = fma(-S.x[p], S.tq[c], M[(int64_t)p * ldm + c]);
    }
    __syncthreads();
    if (tid == 0) {
      int64_t old = Jsel[w.i];
      if (old >= q0 && old < q0 + qn) S.pos[old - q0] = 0;
      if (w.j >= q0 && w.j < q0 + qn) S.pos[w.j - q0] = w.i + 1;
      Jsel[w.i] = w.j;
    }
    logdet += log(fabs(cs));
    ++nsw;
    __syncthreads();
  }
  res.nswaps = nsw;
  res.logdet = logdet;
  return res;
}

// The whole C-A loop for one problem, then the outputs C, R, I, J, G, logvol.
template <class Group>
__device__ void ca_loop(const Group& grp, const CaArgs& A, const CaSmem& S) {
  const DevProblem& P = A.P;
  const int k = A.k, tid = threadIdx.x, nt = blockDim.x;
  const bool lead = grp.rank() == 0;
  // initial rows; every CTA validates them identically
  if (tid == 0) {
    int bad = 0;
    for (int a = 0; a < k; ++a) {
      int32_t v = A.I0[a];
      S.Is[a] = v;
      if (v < 0 || v >= P.m) bad = 1;
      for (int b = 0; b < a; ++b) if (S.Is[b] == v) bad = 1;
    }
    S.ctl[4] = bad;
  }
  if (lead) for (int s = tid; s < 2 * A.sweeps; s += nt) A.logvol[s] = __longlong_as_double(0x7ff8000000000000ll);
  __syncthreads();
  if (S.ctl[4]) {
    if (lead && tid == 0) { A.info[0] = 0; A.info[1] = 0; A.info[2] = 0; A.info[3] = LRA_ERR_INVALID_ARG; }
    return;
  }
  unsigned long long seq = 0;
  int status = LRA_OK, err = LRA_OK, total = 0, loops = 0;
  for (int s = 0; s < A.sweeps; ++s) {
    StepResult r0 = maxvol_step(grp, A, S, 0, s == 0, S.Js, seq);
    if (r0.status != LRA_OK && r0.status < 16) { err = r0.status; break; }
    if (r0.status > status) status = r0.status;
    __syncthreads();
    StepResult r1 = maxvol_step(grp, A, S, 1, false, S.Is, seq);
    if (r1.status != LRA_OK && r1.status < 16) { err = r1.status; break; }
    if (r1.status > status) status = r1.status;
    if (lead && tid == 0) { A.logvol[2 * s] = r0.logdet; A.logvol[2 * s + 1] = r1.logdet; }
    total += r0.nswaps + r1.nswaps;
    loops = s + 1;
    __syncthreads();
    if (s > 0 && r0.nswaps == 0 && r1.nswaps == 0) break;
  }
  if (err != LRA_OK) {
    if (lead && tid == 0) { A.info[0] = 0; A.info[1] = total; A.info[2] = loops; A.info[3] = err; }
    return;
  }
  // outputs: C = W'[:, J] over this CTA's rows, R = W[I, :] over its columns
  {
    const int64_t r0 = (int64_t)grp.rank() * A.chunk_m;
    const int rn = (int)max((int64_t)0, min((int64_t)A.chunk_m, P.m - r0));
    for (int it = tid; it < rn * k; it += nt) {
      int c = it / k, a = it - c * k;
      A.C[(r0 + c) * k + a] = wp_entry(P, r0 + c, S.Js[a]);
    }
    const int64_t c0 = (int64_t)grp.rank() * A.chunk_n;
    const int cn = (int)max((int64_t)0, min((int64_t)A.chunk_n, P.n - c0));
    for (int it = tid; it < k * cn; it += nt) {
      int a = it / cn, c = it - a * cn;
      A.R[(int64_t)a * P.n + c0 + c] = w_entry(P, S.Is[a], c0 + c);
    }
  }
  if (lead) {
    for (int it = tid; it < k * k; it += nt) {
      int a = it / k, b = it - a * k;
      A.G[it] = wp_entry(P, S.Is[a], S.Js[b]);
    }
    for (int a = tid; a < k; a += nt) { A.I[a] = S.Is[a]; A.J[a] = S.Js[a]; }
    if (tid == 0) { A.info[0] = 0; A.info[1] = total; A.info[2] = loops; A.info[3] = status; }
  }
}

}  // namespace lra
