// lra_ca_core.cuh -- one maxvol step of cross-approximation and the whole C-A
// loop, written once over a "group" of CTAs that share the search (a single CTA,
// every CTA of a cooperative grid, or a pair of CTAs of a batched launch).
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
  const int32_t* J0 = nullptr;   // columns warm-starting the first column step, or null (cold start)
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
  int32_t mixed;       // try the FP32 certified step first (single-CTA groups)
  double* work = nullptr;   // if set (lead CTA, thread 0): += the algorithmic flops of each maxvol step
  double* Cstrip = nullptr; // if set (no multiplier): every row step stores the strip it gathers, W'[:, J] = C
                            // (m x k row-major), so the last one leaves the run's C there
  unsigned long long* seq = nullptr;   // the group's exchange round counter when it outlives one run (a CTA
                                       // pair that runs several problems); null: the run counts from 0
};

// Nominal FP64 flops of one kernel entry of the problem (dense: none).
__host__ __device__ inline double entry_flops(const DevProblem& P) {
  return P.src == LRA_DENSE ? 0.0 : (P.src == LRA_KERNEL_LAPLACE ? 8.0 : 10.0);
}

// Algorithmic flops of one maxvol step on a k x len strip (fma = 2, reciprocal
// or division = 1) with nsw swaps: the LU (cold: with column pivoting over the
// strip; warm: of B, then replayed on the other columns -- the same count
// (len - k) k (k - 1) / 2 + (k - 1) k (2k - 1) / 6 fmas), the back substitution
// (len - k) k (k - 1) / 2 fmas and (len - k) k + 2k reciprocals and products,
// each swap 2 (k - 1) len + len, and the strip's entries (plus B's when warm).
__host__ __device__ inline double maxvol_step_flops(int k, int64_t len, bool cold, int nsw, double ent) {
  const double K = k, L = (double)len;
  const double lu = (L - K) * K * (K - 1) / 2 + (K - 1) * K * (2 * K - 1) / 6;
  const double bs = (L - K) * K * (K - 1) / 2;
  const double div = (L - K) * K + 2 * K;
  return 2 * (lu + bs) + div + nsw * (2 * (K - 1) * L + L) + ent * (K * L + (cold ? 0.0 : K * K));
}

struct Cert;           // lra_mixed.cuh

// Shared-memory layout of the C-A kernels (all offsets in bytes, 16-aligned).
struct CaSmem {
  double* LU;        // k*ldl : U0 (cold) or the pivoted LU of B (warm), its multipliers below the diagonal
  double* Lm;        // k*ldl : the FP32 certified steps' multipliers and bounds (null when not carved)
  double* x;         // KMAX : the exchanged column
  double* lmul;      // KMAX : multipliers of the current elimination step
  double* rdiag;     // KMAX : reciprocals of the U0 diagonal
  double* logt;      // LOGBUF : |pivots| whose logs are still to be added
  double* tq;        // ldm  : per-column scratch (swap ratios)
  int32_t* Is;       // KMAX : current rows I
  int32_t* Js;       // KMAX : current columns J
  int32_t* piv;      // KMAX : row interchanges of the warm LU
  int32_t* pos;      // ldm  : 0 = unchosen, else 1 + position in the selected set
  int32_t* ulist;    // ldm  : the unchosen columns of the chunk, ascending (warm replay, back substitution)
  Cand* win;         // the winner of the last exchange
  unsigned long long* flags;
  double* bc;        // 4 doubles of broadcast scratch
  int32_t* ctl;      // small control words
  CandRed* red;      // block reduction scratch
  int32_t* Jsave;    // KMAX : selected set on entry of a mixed step
  Cert* cert;        // 33 : certificate reduction scratch
  ExchangeOut xo;    // where an exchange leaves its result
  double* M;         // the chunk (k x ldm), shared or global
};

constexpr int LOGBUF = 64;

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// lm: with the Lm region (the FP32 certified steps' multipliers and bounds);
// the FP64 steps keep their multipliers in the LU's strictly lower triangle.
__host__ __device__ inline size_t ca_smem_fixed(int k, int ldm, bool lm = true) {
  size_t b = 0;
  b += align16(sizeof(double) * (size_t)k * (k | 1)) * (lm ? 2 : 1);
  b += align16(sizeof(double) * KMAX) * 3;
  b += align16(sizeof(double) * LOGBUF);
  b += align16(sizeof(double) * (size_t)ldm);
  b += align16(sizeof(int32_t) * KMAX) * 3;
  b += align16(sizeof(int32_t) * (size_t)ldm);
  b += align16(sizeof(int32_t) * (size_t)ldm);
  b += align16(sizeof(Cand));
  b += align16(sizeof(unsigned long long));
  b += align16(sizeof(double) * 4);
  b += align16(sizeof(int32_t) * 8);
  b += align16(sizeof(CandRed));
  b += align16(sizeof(int32_t) * KMAX);
  b += align16(48 * 33);
  return b;
}

__device__ inline CaSmem ca_smem_carve(unsigned char* base, int k, int ldm, double* gchunk, bool lm = true) {
  CaSmem S;
  size_t o = 0;
  S.LU = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * (size_t)k * (k | 1));
  S.Lm = nullptr;
  if (lm) { S.Lm = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * (size_t)k * (k | 1)); }
  S.x = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * KMAX);
  S.lmul = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * KMAX);
  S.rdiag = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * KMAX);
  S.logt = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * LOGBUF);
  S.tq = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * (size_t)ldm);
  S.Is = reinterpret_cast<int32_t*>(base + o); o += align16(sizeof(int32_t) * KMAX);
  S.Js = reinterpret_cast<int32_t*>(base + o); o += align16(sizeof(int32_t) * KMAX);
  S.piv = reinterpret_cast<int32_t*>(base + o); o += align16(sizeof(int32_t) * KMAX);
  S.pos = reinterpret_cast<int32_t*>(base + o); o += align16(sizeof(int32_t) * (size_t)ldm);
  S.ulist = reinterpret_cast<int32_t*>(base + o); o += align16(sizeof(int32_t) * (size_t)ldm);
  S.win = reinterpret_cast<Cand*>(base + o); o += align16(sizeof(Cand));
  S.flags = reinterpret_cast<unsigned long long*>(base + o); o += align16(sizeof(unsigned long long));
  S.bc = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * 4);
  S.ctl = reinterpret_cast<int32_t*>(base + o); o += align16(sizeof(int32_t) * 8);
  S.red = reinterpret_cast<CandRed*>(base + o); o += align16(sizeof(CandRed));
  S.Jsave = reinterpret_cast<int32_t*>(base + o); o += align16(sizeof(int32_t) * KMAX);
  S.cert = reinterpret_cast<Cert*>(base + o); o += align16(48 * 33);
  S.xo = ExchangeOut{S.win, S.x, S.flags, &S.ctl[6], S.red};
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

// Volume bookkeeping: log|det| = sum of log|pivot| in pivot order.  Only the
// group's lead CTA keeps it; the |pivots| are buffered and their logs taken
// LOGBUF at a time in parallel, then added in order by one thread, which keeps
// the 2000-cycle FP64 log off the critical path of the pivot loop.
struct LogAcc {
  double sum;
  int cnt;
};
__device__ inline void log_flush(LogAcc& L, const CaSmem& S) {
  if (L.cnt == 0) return;
  __syncthreads();
  for (int e = threadIdx.x; e < L.cnt; e += blockDim.x) S.logt[e] = log(S.logt[e]);
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = L.sum;
    for (int e = 0; e < L.cnt; ++e) s += S.logt[e];
    S.bc[3] = s;
  }
  __syncthreads();
  L.sum = S.bc[3];
  L.cnt = 0;
  __syncthreads();
}
__device__ inline void log_push(LogAcc& L, const CaSmem& S, bool lead, double absval) {
  if (!lead) return;
  if (threadIdx.x == 0) S.logt[L.cnt] = absval;
  ++L.cnt;
  if (L.cnt == LOGBUF) log_flush(L, S);
}

// Work split of "rows x own columns" loops: the CTA's threads cover the qn
// columns; when there are fewer columns than threads, the threads of a column
// share its rows, thread g taking rows p with p % G == g (a fixed partition, so
// the same thread owns a given (row, column) entry in every loop of a step).
struct Map2D {
  int c0, cstep, g, G;
  __device__ __forceinline__ explicit Map2D(int qn) {
    const int nt = blockDim.x, tid = threadIdx.x;
    if (qn >= nt || qn == 0) { c0 = tid; cstep = nt; g = 0; G = 1; }
    else {
      G = nt / qn; g = tid / qn; c0 = tid - g * qn; cstep = qn;
      if (g >= G) c0 = qn;                 // idle thread
    }
  }
  // first row >= lo owned by this thread
  __device__ __forceinline__ int first(int lo) const {
    const int r = lo % G;
    return lo + ((g - r + G) % G);
  }
};

// Work split of the column-local phases (the warm replay and the back
// substitution, where a column needs nothing from other columns): G lanes of
// one warp share a column when there are fewer columns than threads (G a power
// of two), lane g taking rows p with p % G == g and meeting its column's other
// lanes at __syncwarp; every lane of a warp runs the same loop trip counts.
// (One thread per column with half the threads idle was measured slower.)
struct ColMap {
  int c0, cstep, g, G;
  __device__ __forceinline__ explicit ColMap(int qn) {
    const int nt = blockDim.x, tid = threadIdx.x;
    G = 1;
    if (qn > 0)
      while (G < 32 && qn * (2 * G) <= nt) G *= 2;
    g = tid & (G - 1);
    c0 = tid / G;
    cstep = nt / G;
  }
  // trips of the column loop, equal for all lanes of a warp
  __device__ __forceinline__ int trips(int qn) const {
    const int wc0 = (threadIdx.x & ~31) / G;       // first column of this warp
    return wc0 < qn ? (qn - wc0 + cstep - 1) / cstep : 0;
  }
};

// The chunk's unchosen columns (pos == 0), ascending, into S.ulist by warp 0
// (a ballot per 32 columns); returns their number to warp 0's lanes.
__device__ inline int list_unchosen_warp(const CaSmem& S, int qn) {
  const int lane = threadIdx.x & 31;
  int n = 0;
  for (int c0 = 0; c0 < qn; c0 += 32) {
    const int c = c0 + lane;
    const bool f = c < qn && S.pos[c] == 0;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (f) S.ulist[n + __popc(bal & ((1u << lane) - 1u))] = c;
    n += __popc(bal);
  }
  return n;
}

// Gather the k x qn chunk of the strip; returns nonzero if any entry is not finite.
__device__ inline int gather_chunk(const DevProblem& P, int phase, const CaSmem& S, int k, int64_t q0, int qn,
                                   int ldm, const Map2D& mp) {
  double* M = S.M;
  int bad = 0;
  for (int c = mp.c0; c < qn; c += mp.cstep)
    for (int a = mp.g; a < k; a += mp.G) {
      const double v = strip_entry(P, phase, S.Is, S.Js, a, q0 + c);
      M[(int64_t)a * ldm + c] = v;
      bad |= !bits_finite(v);
    }
  return bad;
}

// One maxvol step over the k x len strip of `phase`.  Jsel: in = warm set (ignored
// when cold), out = selected k strip columns in generator order.  seq: exchange
// round counter, advanced identically in every CTA of the group.  The
// arithmetic is that of the FP64 reference, operation for operation: LU with
// column pivoting (cold) or with row pivoting on the warm columns, multipliers
// a_p * (1/pivot), column-sweep back substitution with the reciprocals of the
// U0 diagonal, swaps t_q = C[i*][q] * (1/c*), C[p][q] = fma(-x_p, t_q, C[p][q]).
// The k x k LU is stored with the odd row stride ldl = k | 1 (no bank conflicts
// when a warp walks down one of its columns); a warm LU keeps its multipliers
// below the diagonal.  The column-local phases (replay, back substitution) run
// over the list of the unchosen columns.  kPre: the strip is already in
// the chunk M (a single CTA holding all of it, rows 0..k-1); nothing is
// gathered and the warm start reads B = M[:, Jsel].
template <class Group, bool kPre = false>
__device__ StepResult maxvol_step(const Group& grp, const CaArgs& A, const CaSmem& S, int phase, bool cold,
                                  int32_t* Jsel, unsigned long long& seq, bool lead) {
  const DevProblem& P = A.P;
  const int k = A.k, ldm = A.ldm, tid = threadIdx.x, nt = blockDim.x;
  const int ldl = k | 1;
  const int lane = tid & 31, warp = tid >> 5;
  const int64_t len = phase == 0 ? pcols(P) : P.m;
  const int chunk = phase == 0 ? A.chunk_n : A.chunk_m;
  const int64_t q0 = (int64_t)grp.rank() * chunk;
  const int qn = (int)max((int64_t)0, min((int64_t)chunk, len - q0));
  const Map2D mp(qn);
  double* M = S.M;
  double* LU = S.LU;
  StepResult res{LRA_OK, 0, 0.0};
  LogAcc L{0.0, 0};

  if (tid == 0) S.ctl[0] = 0;
  for (int c = tid; c < qn; c += nt) S.pos[c] = 0;
  __syncthreads();
  if constexpr (!kPre) {
    if (gather_chunk(P, phase, S, k, q0, qn, ldm, mp)) atomicOr(&S.ctl[0], 1);
    if (phase == 1 && A.Cstrip != nullptr) {
      __syncthreads();
      for (int it = tid; it < qn * k; it += nt) {
        const int c = it / k, a = it - c * k;
        A.Cstrip[(q0 + c) * k + a] = M[(int64_t)a * ldm + c];
      }
    }
  }
  __syncthreads();
  const unsigned long long myflags = S.ctl[0] ? FLAG_NONFINITE : 0ull;
  bool deficient = false;

  if (!cold) {
    // ---- warm start: B = strip[:, Jsel]; the pivoted LU of B is replayed by every CTA
    for (int it = tid; it < k * k; it += nt) {
      const int a = it / k, t = it - a * k;
      if constexpr (kPre) LU[a * ldl + t] = M[(int64_t)a * ldm + (Jsel[t] - q0)];
      else LU[a * ldl + t] = strip_entry(P, phase, S.Is, S.Js, a, Jsel[t]);
    }
    __syncthreads();
    int fallback = 0;
    for (int t = 0; t < k; ++t) {
      if (warp == 0) {
        // pivot row: largest |B(t)[p][t]| over p >= t, lowest p on ties; every
        // lane takes the reciprocal of its candidates while the search runs
        Cand c = cand_none();
        double rc0 = 0.0, rc1 = 0.0;
        const int p0 = t + lane, p1 = t + lane + 32;
        if (p0 < k) { const double v = LU[p0 * ldl + t]; cand_consider(c, mag_key(v), 0, p0); rc0 = 1.0 / v; }
        if (p1 < k) { const double v = LU[p1 * ldl + t]; cand_consider(c, mag_key(v), 0, p1); rc1 = 1.0 / v; }
        c = warp_best_local(c, 0);                   // rows < 64 as positions: the order of cand_better
        const int r = (c.key == 0ull) ? t : c.j;
        const double pv = LU[r * ldl + t];
        const int rl = (r - t) & 31;
        const double rsel = (r - t) < 32 ? rc0 : rc1;
        const double rp = __shfl_sync(0xffffffffu, rsel, rl);
        if (lane == 0) {
          S.piv[t] = r;
          S.ctl[1] = (pv == 0.0);
        }
        // multipliers l_p = B[p][t] * (1/pivot) of the rows below t after the
        // interchange (row r then holds row t's entry)
        double l0 = 0.0, l1 = 0.0;
        if (pv != 0.0) {
          if (t + 1 + lane < k) { const int p = t + 1 + lane; l0 = ((p == r) ? LU[t * ldl + t] : LU[p * ldl + t]) * rp; }
          if (t + 33 + lane < k) { const int p = t + 33 + lane; l1 = ((p == r) ? LU[t * ldl + t] : LU[p * ldl + t]) * rp; }
        }
        __syncwarp();
        // interchange rows t and r in columns t.. only: column t' < t keeps the
        // multipliers of step t' in the row positions of that step, the order in
        // which they are replayed on the CTA's own columns below
        if (r != t)
          for (int j = t + lane; j < k; j += 32) {
            const double tmp = LU[t * ldl + j]; LU[t * ldl + j] = LU[r * ldl + j]; LU[r * ldl + j] = tmp;
          }
        __syncwarp();
        // the multipliers go below the diagonal of column t, where the LU keeps them
        if (pv != 0.0) {
          if (t + 1 + lane < k) LU[(t + 1 + lane) * ldl + t] = l0;
          if (t + 33 + lane < k) LU[(t + 33 + lane) * ldl + t] = l1;
        }
      }
      __syncthreads();
      if (S.ctl[1]) { fallback = 1; break; }          // same decision in every CTA
      // trailing (k-t-1)^2 update, one entry per thread, consecutive threads
      // along a row: every warp of the CTA takes a share, so all four SM
      // sub-partitions' FP64 units work on it
      {
        const int w = k - t - 1;
        for (int e = tid; e < w * w; e += nt) {
          const int p = t + 1 + e / w, j = t + 1 + e % w;
          LU[p * ldl + j] = fma(-LU[p * ldl + t], LU[t * ldl + j], LU[p * ldl + j]);
        }
      }
      __syncthreads();
    }
    if (fallback) {
      cold = true;
      __syncthreads();
    } else {
      if (warp == 0) {
        for (int t = lane; t < k; t += 32) {
          const int64_t jt = Jsel[t];
          if (jt >= q0 && jt < q0 + qn) S.pos[jt - q0] = t + 1;
        }
        __syncwarp();
        const int nu = list_unchosen_warp(S, qn);
        if (lane == 0) S.ctl[5] = nu;
      }
      __syncthreads();
      // replay the row interchanges and eliminations on the unchosen columns (the
      // chosen ones become unit columns after the back substitution), one column
      // (or one group of lanes) at a time: the columns are independent
      {
        const int nu = S.ctl[5];
        const ColMap cm(nu);
        const int trips = cm.trips(nu);
        for (int u = 0; u < trips; ++u) {
          const int ix = cm.c0 + u * cm.cstep;
          const bool act = ix < nu;
          const int c = act ? S.ulist[ix] : 0;
          for (int t = 0; t < k; ++t) {
            const int r = S.piv[t];
            if (act && r != t && cm.g == 0) {
              const double tmp = M[(int64_t)t * ldm + c];
              M[(int64_t)t * ldm + c] = M[(int64_t)r * ldm + c];
              M[(int64_t)r * ldm + c] = tmp;
            }
            if (cm.G > 1) __syncwarp();
            if (act) {
              const double mt = M[(int64_t)t * ldm + c];
              int p = t + 1;
              p += (cm.g - p % cm.G + cm.G) % cm.G;
              for (; p < k; p += cm.G)
                M[(int64_t)p * ldm + c] = fma(-LU[p * ldl + t], mt, M[(int64_t)p * ldm + c]);
            }
            if (cm.G > 1) __syncwarp();
          }
        }
      }
      __syncthreads();
      for (int t = 0; t < k; ++t) log_push(L, S, lead, fabs(LU[t * ldl + t]));
    }
  }

  if (cold) {
    // ---- cold start: LU with column pivoting over the whole strip
    for (int t = 0; t < k; ++t) {
      Cand mine = cand_none();
      unsigned bhi = 0;
      for (int c = tid; c < qn; c += nt)
        if (S.pos[c] == 0) cand_take_val(mine, bhi, M[(int64_t)t * ldm + c], 0, (int32_t)(q0 + c));
      grp.template exchange<false>(seq, mine, myflags, M, ldm, q0, k, chunk, S.xo);
      ++seq;
      if (warp == 0) {
        // warp 0 holds the winner: the pivot's reciprocal, U0's column t and the
        // multipliers of this elimination step
        const Cand w = *S.win;
        const double pv = S.x[t];
        if (lane == 0) {
          Jsel[t] = w.j;
          if (w.j >= q0 && w.j < q0 + qn) S.pos[w.j - q0] = t + 1;
        }
        if (pv != 0.0) {
          const double rp = 1.0 / pv;
          for (int p = lane; p <= t; p += 32) LU[p * ldl + t] = S.x[p];
          for (int p = t + 1 + lane; p < k; p += 32) S.lmul[p] = S.x[p] * rp;
        }
      }
      __syncthreads();
      if (grp.failed(S.xo)) { res.status = LRA_ERR_TIMEOUT; return res; }
      if (*S.flags & FLAG_NONFINITE) { res.status = LRA_ERR_NONFINITE; return res; }
      const double pv = S.x[t];
      if (pv == 0.0) { deficient = true; continue; }
      for (int c = mp.c0; c < qn; c += mp.cstep) {
        if (S.pos[c]) continue;
        const double mt = M[(int64_t)t * ldm + c];
        for (int p = mp.first(t + 1); p < k; p += mp.G)
          M[(int64_t)p * ldm + c] = fma(-S.lmul[p], mt, M[(int64_t)p * ldm + c]);
      }
      log_push(L, S, lead, fabs(pv));
      __syncthreads();
    }
    if (deficient) {
      res.status = LRA_WARN_RANK_DEFICIENT;
      res.logdet = -INFINITY;
      return res;
    }
  }

  // ---- C = (I | U0^{-1} U1): column-sweep back substitution on unchosen columns.
  // The owner of row i scales it (x_i = b_i * (1/U0_ii)) right after its last
  // update, so one barrier per row suffices.
  for (int i = tid; i < k; i += nt) S.rdiag[i] = 1.0 / LU[i * ldl + i];
  if (cold && warp == 0) {              // the unchosen columns after the cold LU (warm steps listed them above)
    const int nu = list_unchosen_warp(S, qn);
    if (lane == 0) S.ctl[5] = nu;
  }
  __syncthreads();
  {
    // column by column over the unchosen columns (lanes of one column meet at
    // __syncwarp): no CTA barrier
    const int nu = S.ctl[5];
    const ColMap cm(nu);
    const int trips = cm.trips(nu);
    for (int u = 0; u < trips; ++u) {
      const int ix = cm.c0 + u * cm.cstep;
      const bool act = ix < nu;
      const int c = act ? S.ulist[ix] : 0;
      if (act && (k - 1) % cm.G == cm.g)
        M[(int64_t)(k - 1) * ldm + c] = M[(int64_t)(k - 1) * ldm + c] * S.rdiag[k - 1];
      for (int i = k - 1; i >= 1; --i) {
        if (cm.G > 1) __syncwarp();
        if (act) {
          const double xi = M[(int64_t)i * ldm + c];
          for (int p = cm.g; p < i; p += cm.G)
            M[(int64_t)p * ldm + c] = fma(-LU[p * ldl + i], xi, M[(int64_t)p * ldm + c]);
          // row i - 1 is complete: its owner scales it (one FP64 multiply per
          // row, outside the loop, where a select would cost one per entry)
          if (((i - 1) & (cm.G - 1)) == cm.g)
            M[(int64_t)(i - 1) * ldm + c] = M[(int64_t)(i - 1) * ldm + c] * S.rdiag[i - 1];
        }
      }
      if (cm.G > 1) __syncwarp();
    }
  }
  __syncthreads();
  for (int c = mp.c0; c < qn; c += mp.cstep)
    if (S.pos[c])
      for (int a = mp.g; a < k; a += mp.G) M[(int64_t)a * ldm + c] = (S.pos[c] - 1 == a) ? 1.0 : 0.0;
  __syncthreads();

  // ---- dominance swaps (Algorithm algdomin).  Only entries with |c| > h can
  // cause a swap, and the search's winner is used only when it is one of them:
  // each thread keeps its best entry above h (none if there is none), which
  // gives the same decision and the same winner as the best of all entries.
  // Each thread visits its entries column by column, rows ascending, so an
  // equal key never replaces the lower (j, i); after the first scan, the search
  // for the next swap runs inside the rank-1 update, on the values as written.
  const unsigned long long hkey = mag_key(A.h);
  const unsigned hhi = (unsigned)__double2hiint(A.h) & 0x7fffffffu;
  int nsw = 0;
  Cand mine = cand_none();
  unsigned bhi = hhi;
  for (int c = mp.c0; c < qn; c += mp.cstep) {
    if (S.pos[c]) continue;
    for (int a = mp.g; a < k; a += mp.G)
      cand_take_above(mine, bhi, M[(int64_t)a * ldm + c], a, (int32_t)(q0 + c), hkey);
  }
  for (;;) {
    grp.template exchange<false>(seq, mine, myflags, M, ldm, q0, k, chunk, S.xo);
    ++seq;
    if (warp == 0) {                              // the reciprocal of the winner, before the barrier
      const Cand w = *S.win;
      if (w.key > hkey && lane == 0) S.bc[0] = 1.0 / S.x[w.i];
    }
    __syncthreads();
    if (grp.failed(S.xo)) { res.status = LRA_ERR_TIMEOUT; return res; }
    if (*S.flags & FLAG_NONFINITE) { res.status = LRA_ERR_NONFINITE; return res; }
    const Cand w = *S.win;
    if (w.key <= hkey) break;                     // no |c| > h left (or no candidate)
    if (nsw >= A.max_swaps) { res.status = LRA_WARN_NOT_CONVERGED; break; }
    const double rcs = S.bc[0];
    // t_q = C[i*][q] * (1/c*): with one thread to a column (mp.G == 1, uniform)
    // that thread reads row i* itself before it updates the column; otherwise
    // all t_q first, then the update
    const bool own_tq = mp.G == 1;
    if (!own_tq) {
      for (int c = tid; c < qn; c += nt) S.tq[c] = M[(int64_t)w.i * ldm + c] * rcs;
      __syncthreads();
    }
    // the columns outside the selected set after this swap: the unselected ones
    // but w.j, and the column leaving position w.i
    const int64_t wjl = w.j - q0, oldl = (int64_t)Jsel[w.i] - q0;
    mine = cand_none();
    bhi = hhi;
    for (int c = mp.c0; c < qn; c += mp.cstep) {
      const double tq = own_tq ? M[(int64_t)w.i * ldm + c] * rcs : S.tq[c];
      const bool cand = (c == oldl) || (S.pos[c] == 0 && c != wjl);
      for (int p = mp.g; p < k; p += mp.G) {
        const double v = (p == w.i) ? tq : fma(-S.x[p], tq, M[(int64_t)p * ldm + c]);
        M[(int64_t)p * ldm + c] = v;
        if (cand) cand_take_above(mine, bhi, v, p, (int32_t)(q0 + c), hkey);
      }
    }
    __syncthreads();
    if (w.j >= q0 && w.j < q0 + qn)
      for (int p = tid; p < k; p += nt) M[(int64_t)p * ldm + (w.j - q0)] = (p == w.i) ? 1.0 : 0.0;
    if (tid == 0) {
      const int64_t old = Jsel[w.i];
      if (old >= q0 && old < q0 + qn) S.pos[old - q0] = 0;
      if (w.j >= q0 && w.j < q0 + qn) S.pos[w.j - q0] = w.i + 1;
      Jsel[w.i] = w.j;
    }
    log_push(L, S, lead, fabs(S.x[w.i]));
    ++nsw;
    __syncthreads();
  }
  log_flush(L, S);
  res.nswaps = nsw;
  res.logdet = L.sum;
  return res;
}

}  // namespace lra
