// lra_oversample.cu -- rectangular k x l generators for a batch of blocks
// (paper: Algorithm algrup, greedy expansions of a k x k submatrix to k x l;
// Theorem th3 bounds the CUR error of such generators), one CTA per block from a
// work queue, after a batched C-A run has produced each block's square
// generator (rows I, columns J).
//
// Per block: X = B^{-1} W'[I, :] is the C matrix of a maxvol step on the row
// strip warm-started at J with no swaps (the single-CTA maxvol arithmetic);
// then p times the column outside the generator with the largest s_j =
// ||X[:, j]||^2 joins it (the squared volume grows by 1 + s_j) and every other
// column is whitened again, X[:, q] -= gamma (x . X[:, q]) x with gamma =
// (1 - 1/sqrt(1 + sigma)) / sigma (Sherman-Morrison for (C C^T)^{-1}); the
// columns are independent, one thread each.  With pmax > 0, Section scrsorth's
// expansion/contraction cycles follow: while the generator fails the local
// h-maximality test of Corollary colclmx (1 + max s_q over the columns outside
// it <= h), a p-cycle adds p columns greedily and removes p greedily (the column
// with the smallest s_j leaves, X[:, q] += gamma' (x . X[:, q]) x with
// gamma' = (1/sqrt(1 - sigma) - 1) / sigma, Theorem th2); a cycle that changed
// the set and raised the volume is kept and p restarts at 1, otherwise X, s and
// J' are restored from a per-CTA copy and p grows.  Outputs C = W'[:, J'], the
// rectangular nucleus U of W'[I, J'] and R = W[I, :].
//
// prjvol_kernel picks the columns by r-projective volume instead (Algorithm
// algprjvlm): Algorithm alg1tor (Householder QR with column pivoting, stopped
// at the numerical rank r) reduces the strip W'[I, :] to R' (r x n) in place,
// a warm maxvol step on R' from the QR's pivots makes the r x r submatrix
// locally h-maximal (Algorithm algdomin), and Algorithm algrup's expansions
// take it to l columns; the outputs are those of oversample_kernel.
#include <algorithm>
#include <cstring>

#include "lra_ca_core.cuh"
#include "lra_internal.h"
#include "lra_nucleus.cuh"
#include "lra_profile.h"

namespace lra {

struct OvArgs {
  DevProblem base;
  const int64_t* blocks;      // nb x 4
  const int64_t* offs;        // nb x 2: offsets of C_b (nrows x l_b) and R_b (k_b x ncols) in the outputs
  const int32_t* order;
  int32_t nb, kmax, pextra, lmax;
  int32_t pmax, max_cycles;   // expansion/contraction cycles (pmax = 0: none)
  int32_t max_swaps;          // prjvol: dominance swaps on R'
  double h, rank_tol;
  const int32_t* Iin;         // nb x kmax
  const int32_t* Jin;         // nb x kmax
  const int32_t* info_in;     // nb x LRA_INFO_LEN (k used = info[6], status = info[3])
  int32_t* I;                 // nb x kmax
  int32_t* J;                 // nb x lmax
  double* C;
  double* R;
  double* U;                  // nb x lmax x kmax
  int32_t* info;              // nb x LRA_INFO_LEN
  unsigned int* counter;
  double* scratch;            // per CTA: G (kmax x lmax), if needed a strip (kmax x max_len), and with
                              // cycles a copy of X and s ((kmax + 1) x max_len)
  size_t scratch_stride;
  size_t backup_offset;       // doubles from the CTA's scratch to its copy of X and s
  size_t smem_bytes;
  int64_t max_len;
};

constexpr int PMAX = 16;     // largest p of an expansion/contraction cycle

// Key that orders candidates by the smallest |x| first (0 = no candidate, NaN never one).
__device__ __forceinline__ unsigned long long min_key(double x) {
  const unsigned long long a = mag_key(x);
  return a == 0ull ? 0ull : (INF_BITS + 2ull) - a;
}

// Whitening update of X (k x nc, leading dimension ldm) for column j entering
// (sign = +1) or leaving (sign = -1) the generator: with x = X[:, j] and
// sigma = s_j, X[:, q] <- fma(c_q, x, X[:, q]) for every column q, c_q = -+g t_q,
// t_q = x . X[:, q], g = (1 - 1/sqrt(1 + sigma)) / sigma entering and
// (1/sqrt(1 - sigma) - 1) / sigma leaving (Sherman-Morrison), then s_q is
// recomputed.  sigma = 0 changes nothing.  Called by the whole CTA.
__device__ void ov_whiten(double* M, int ldm, double* s, int k, int nc, int j, int sign, double* s_x, double* s_g) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const double sigma = s[j];
  if (sigma == 0.0) return;
  if (tid == 0)
    s_g[0] = (sign > 0) ? -((1.0 - 1.0 / sqrt(1.0 + sigma)) / sigma) : (1.0 / sqrt(1.0 - sigma) - 1.0) / sigma;
  for (int i = tid; i < k; i += nt) s_x[i] = M[(int64_t)i * ldm + j];
  __syncthreads();
  const double gs = s_g[0];
  for (int c = tid; c < nc; c += nt) {
    double t = 0.0;
    for (int i = 0; i < k; ++i) t = fma(s_x[i], M[(int64_t)i * ldm + c], t);
    const double cc = gs * t;
    double v = 0.0;
    for (int i = 0; i < k; ++i) {
      const double x = fma(cc, s_x[i], M[(int64_t)i * ldm + c]);
      M[(int64_t)i * ldm + c] = x;
      v = fma(x, x, v);
    }
    s[c] = v;
  }
  __syncthreads();
}

// Greedy expansion by up to p columns (Algorithm algrup): the column outside
// the generator with the largest s_j (lowest j on ties) is appended to Jw; none
// once the largest s_j is 0.  rho[0] *= 1 + s_j.  Returns the number added.
__device__ int ov_expand(double* M, int ldm, double* s, int32_t* pos, int32_t* Jw, int& l, int k, int nc, int p,
                         double* rho, double* s_x, double* s_g, CandRed* red) {
  int added = 0;
  for (int g = 0; g < p; ++g) {
    Cand mine = cand_none();
    for (int c = threadIdx.x; c < nc; c += blockDim.x)
      if (!pos[c]) cand_consider(mine, mag_key(s[c]), 0, c);
    unsigned long long fl = 0;
    const Cand w = block_best(mine, fl, red);
    if (w.key == 0ull || w.key == mag_key(0.0)) break;
    const int js = w.j;
    if (threadIdx.x == 0) {
      rho[0] = rho[0] * (1.0 + s[js]);
      pos[js] = 1;
      Jw[l] = js;
    }
    __syncthreads();
    ++l;
    ov_whiten(M, ldm, s, k, nc, js, +1, s_x, s_g);
    ++added;
  }
  __syncthreads();
  return added;
}

// Greedy contraction by p columns (the reverse of Algorithm algrup): the column
// inside the generator with the smallest s_j (lowest j on ties) leaves Jw, whose
// other entries keep their order.  rho[0] *= 1 - s_j.  Returns false if the
// smallest s_j is not below 1.
__device__ bool ov_contract(double* M, int ldm, double* s, int32_t* pos, int32_t* Jw, int& l, int k, int nc, int p,
                            double* rho, double* s_x, double* s_g, CandRed* red) {
  for (int g = 0; g < p; ++g) {
    Cand mine = cand_none();
    for (int c = threadIdx.x; c < nc; c += blockDim.x)
      if (pos[c]) cand_consider(mine, min_key(s[c]), 0, c);
    unsigned long long fl = 0;
    const Cand w = block_best(mine, fl, red);
    if (w.key == 0ull) return false;
    const int jr = w.j;
    if (!(s[jr] < 1.0)) return false;
    if (threadIdx.x == 0) {
      rho[0] = rho[0] * (1.0 - s[jr]);
      int a = 0;
      while (a < l && Jw[a] != jr) ++a;
      for (; a + 1 < l; ++a) Jw[a] = Jw[a + 1];
      pos[jr] = 0;
    }
    __syncthreads();
    --l;
    ov_whiten(M, ldm, s, k, nc, jr, -1, s_x, s_g);
  }
  __syncthreads();
  return true;
}

// The next block of the batch from the work queue, or -1 once it is empty (the
// same value in every thread).  Called by the whole CTA.
__device__ int ov_next_block(const OvArgs& B, int* s_b) {
  if (threadIdx.x == 0) {
    const unsigned int qh = atomicAdd(B.counter, 1u);
    *s_b = (qh < (unsigned)B.nb) ? (B.order ? B.order[qh] : (int)qh) : -1;
  }
  __syncthreads();
  const int b = *s_b;
  __syncthreads();
  return b;
}

// Block b's sub-problem: false, after writing the block's status, when its
// descriptor or its C-A run is unusable (a failed run keeps its status).
// Otherwise nr, nc, k (the run's generator size), lb = min(k + pextra, nc) and
// the maxvol arguments A for the row strip W'[I, :] (no swaps; leading
// dimension nc when cols_only, else max(nr, nc); the strip in shared memory
// when it fits, else in gstrip).
__device__ bool ov_block_begin(const OvArgs& B, int b, bool cols_only, double* gstrip, CaArgs& A, int64_t& nr,
                               int64_t& nc, int& k, int& lb) {
  int32_t* info = B.info + LRA_INFO_LEN * (size_t)b;
  const int32_t* inf0 = B.info_in + LRA_INFO_LEN * (size_t)b;
  const int64_t r0 = B.blocks[4 * (size_t)b], c0 = B.blocks[4 * (size_t)b + 2];
  nr = B.blocks[4 * (size_t)b + 1];
  nc = B.blocks[4 * (size_t)b + 3];
  const int st_in = inf0[3];
  k = inf0[6];
  if (r0 < 0 || c0 < 0 || nr < 1 || nc < 1 || r0 + nr > B.base.m || c0 + nc > B.base.n || nr > B.max_len ||
      nc > B.max_len || (st_in != LRA_OK && st_in < 16) || k < 1 || k > B.kmax || k > min(nr, nc)) {
    for (int e = threadIdx.x; e < LRA_INFO_LEN; e += blockDim.x)
      info[e] = (e == 3) ? ((st_in != LRA_OK && st_in < 16) ? st_in : LRA_ERR_INVALID_ARG) : 0;
    return false;
  }
  lb = (int)min((int64_t)(k + B.pextra), nc);
  std::memset(&A, 0, sizeof(A));
  A.P = B.base;
  A.P.m = nr;
  A.P.n = nc;
  if (A.P.src == LRA_DENSE) {
    const size_t esz = (A.P.dtype == LRA_F32) ? 4 : 8;
    A.P.W = static_cast<const unsigned char*>(B.base.W) + (size_t)(r0 * B.base.ldw + c0) * esz;
  } else {
    A.P.X = B.base.X + 3 * r0;
    A.P.Y = B.base.Y + 3 * c0;
  }
  A.k = k;
  A.max_swaps = 0;
  A.h = B.h;
  A.chunk_n = (int)nc;
  A.chunk_m = (int)nr;
  A.ldm = cols_only ? (int)nc : (int)max(nr, nc);
  A.strip_in_smem = ca_smem_fixed(k, A.ldm) + sizeof(double) * (size_t)k * A.ldm <= B.smem_bytes;
  A.gstrip = A.strip_in_smem ? nullptr : gstrip;
  return true;
}

// Outputs of block b at l columns J' = Jb: C = W'[:, J'] (nr x l), R = W[I, :]
// (k x nc), the rows I, U = the rectangular nucleus of G = W'[I, J'] (formed in
// the CTA's scratch G), and info = (rank, i1, i2, status, 0, 0, k, l), the
// status turned to LRA_WARN_RANK_DEFICIENT when it was LRA_OK and the rank is
// below k.  Called by the whole CTA.
__device__ void ov_block_finish(const OvArgs& B, int b, const CaArgs& A, int64_t nr, int64_t nc, int k, int l,
                                const int32_t* Jb, int st, int i1, int i2, double* G, unsigned char* smem) {
  const int tid = threadIdx.x, nt = blockDim.x;
  int32_t* info = B.info + LRA_INFO_LEN * (size_t)b;
  __syncthreads();
  const int32_t* Ib = B.Iin + (size_t)b * B.kmax;
  double* Cb = B.C + B.offs[2 * (size_t)b];
  double* Rb = B.R + B.offs[2 * (size_t)b + 1];
  for (int64_t it = tid; it < nr * l; it += nt) {
    const int64_t i = it / l;
    const int a = (int)(it - i * l);
    Cb[it] = c_entry(A.P, i, Jb[a]);
  }
  for (int64_t it = tid; it < (int64_t)k * nc; it += nt) {
    const int a = (int)(it / nc);
    const int64_t c = it - (int64_t)a * nc;
    Rb[it] = r_entry(A.P, Ib[a], c);
  }
  for (int it = tid; it < k * l; it += nt) {
    const int a = it / l, c = it - a * l;
    G[it] = wp_entry(A.P, Ib[a], Jb[c]);
  }
  for (int a = tid; a < k; a += nt) B.I[(size_t)b * B.kmax + a] = Ib[a];
  __syncthreads();
  const int rank = nucleus_rect_cta(G, k, l, B.rank_tol, B.U + (size_t)b * B.lmax * B.kmax, smem);
  if (tid == 0) {
    if (rank < k && st == LRA_OK) st = LRA_WARN_RANK_DEFICIENT;
    info[0] = rank; info[1] = i1; info[2] = i2; info[3] = st; info[4] = 0; info[5] = 0; info[6] = k;
    info[7] = l;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NT) oversample_kernel(OvArgs B) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_b;
  __shared__ double s_x[KMAX];
  __shared__ double s_g[2];
  __shared__ double s_rho[1];
  __shared__ int s_flag;
  __shared__ int32_t s_Jw[2 * KMAX + PMAX];   // the generator's columns during expansion and cycles
  __shared__ int32_t s_Jb[2 * KMAX];          // their copy at the start of a cycle
  double* G = B.scratch + (size_t)blockIdx.x * B.scratch_stride;
  double* gstrip = G + (size_t)B.kmax * B.lmax;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (;;) {
    const int b = ov_next_block(B, &s_b);
    if (b < 0) break;
    int32_t* info = B.info + LRA_INFO_LEN * (size_t)b;
    CaArgs A;
    int64_t nr, nc;
    int k, lb;
    if (!ov_block_begin(B, b, false, gstrip, A, nr, nc, k, lb)) continue;
    int32_t* Jb = B.J + (size_t)b * B.lmax;
    int l = k, st = LRA_OK, cycles = 0, ptried = 0;
    {
      const CaSmem S = ca_smem_carve(smem, k, A.ldm, A.gstrip);
      for (int a = tid; a < k; a += nt) {
        S.Is[a] = B.Iin[(size_t)b * B.kmax + a];
        S.Js[a] = B.Jin[(size_t)b * B.kmax + a];
      }
      __syncthreads();
      unsigned long long seq = 0;
      const StepResult sr = maxvol_step(SoloGroup{}, A, S, 0, false, S.Js, seq, true);
      __syncthreads();
      st = (sr.status == LRA_WARN_NOT_CONVERGED) ? LRA_OK : sr.status;
      if (st != LRA_OK && st < 16) {
        if (tid == 0) {
          info[0] = 0; info[1] = 0; info[2] = 0; info[3] = st; info[4] = 0; info[5] = 0; info[6] = k; info[7] = k;
        }
        __syncthreads();
        continue;
      }
      if (st == LRA_WARN_RANK_DEFICIENT) {
        // zero pivot: no expansion, the square generator as given
        for (int a = tid; a < k; a += nt) Jb[a] = B.Jin[(size_t)b * B.kmax + a];
      } else {
        for (int a = tid; a < k; a += nt) s_Jw[a] = S.Js[a];
        double* M = S.M;
        double* s = S.tq;                        // per-column s_j (ldm doubles)
        // s_j of every column, ascending rows (the generator's columns are unit vectors)
        for (int c = tid; c < nc; c += nt) {
          double v = 0.0;
          for (int i = 0; i < k; ++i) v = fma(M[(int64_t)i * A.ldm + c], M[(int64_t)i * A.ldm + c], v);
          s[c] = v;
        }
        if (tid == 0) s_rho[0] = 1.0;
        __syncthreads();
        ov_expand(M, A.ldm, s, S.pos, s_Jw, l, k, (int)nc, lb - k, s_rho, s_x, s_g, S.red);
        if (B.pmax > 0) {
          const int ltarget = l;
          double* Mb = G + B.backup_offset;
          bool converged = false;
          int pc = 1;
          for (;;) {
            Cand mine = cand_none();
            for (int c = tid; c < nc; c += nt)
              if (!S.pos[c]) cand_consider(mine, mag_key(s[c]), 0, c);
            unsigned long long fl = 0;
            const Cand w = block_best(mine, fl, S.red);
            const double smax = (w.key == 0ull) ? 0.0 : s[w.j];
            if (1.0 + smax <= B.h) { converged = true; break; }
            if (pc > B.pmax || cycles >= B.max_cycles) break;
            ptried = max(ptried, pc);
            for (int64_t it = tid; it < (int64_t)k * nc; it += nt) {
              const int i = (int)(it / nc);
              Mb[it] = M[(int64_t)i * A.ldm + (it - (int64_t)i * nc)];
            }
            for (int c = tid; c < nc; c += nt) Mb[(int64_t)k * nc + c] = s[c];
            for (int a = tid; a < ltarget; a += nt) s_Jb[a] = s_Jw[a];
            if (tid == 0) { s_rho[0] = 1.0; s_flag = 0; }
            __syncthreads();
            const int added = ov_expand(M, A.ldm, s, S.pos, s_Jw, l, k, (int)nc, pc, s_rho, s_x, s_g, S.red);
            const bool ok = added > 0 && ov_contract(M, A.ldm, s, S.pos, s_Jw, l, k, (int)nc, added, s_rho, s_x,
                                                     s_g, S.red);
            if (ok) {
              for (int a = tid; a < l; a += nt) {
                bool found = false;
                for (int e = 0; e < ltarget; ++e) found = found || (s_Jb[e] == s_Jw[a]);
                if (!found) s_flag = 1;
              }
            }
            __syncthreads();
            if (ok && s_flag != 0 && s_rho[0] > 1.0) {
              ++cycles;
              pc = 1;
            } else {
              for (int a = tid; a < l; a += nt) S.pos[s_Jw[a]] = 0;
              __syncthreads();
              for (int64_t it = tid; it < (int64_t)k * nc; it += nt) {
                const int i = (int)(it / nc);
                M[(int64_t)i * A.ldm + (it - (int64_t)i * nc)] = Mb[it];
              }
              for (int c = tid; c < nc; c += nt) s[c] = Mb[(int64_t)k * nc + c];
              for (int a = tid; a < ltarget; a += nt) {
                s_Jw[a] = s_Jb[a];
                S.pos[s_Jb[a]] = 1;
              }
              l = ltarget;
              ++pc;
            }
            __syncthreads();
          }
          if (!converged && st == LRA_OK) st = LRA_WARN_NOT_CONVERGED;
        }
        for (int a = tid; a < l; a += nt) Jb[a] = s_Jw[a];
      }
    }
    ov_block_finish(B, b, A, nr, nc, k, l, Jb, st, cycles, ptried, G, smem);
  }
}

// Algorithm alg1tor on the k x nc strip M (leading dimension ldm), stopped at
// the numerical rank: Householder QR with column pivoting in the FP64
// reference's arithmetic.  Step g: the pivot is the unchosen column with the
// largest squared norm s_c of rows g.. (lowest c on ties); the loop stops when
// that norm is 0, or (g > 0) when its square root is <= tol times the first
// pivot's; alpha = -sqrt(s) for x_0 >= 0, else +sqrt(s); v = x - alpha e_1;
// tau = 1 / (sqrt(s) (sqrt(s) + |x_0|)); every unchosen column c gets
// t = v . M[g.., c] (ascending fma chain), M[g + i][c] = fma(-(tau t), v_i,
// M[g + i][c]) and, in the same pass, its squared norm over rows g + 1.. for
// the next search; the pivot column becomes (alpha, 0, ..., 0).  s: nc
// doubles; pos: nc flags (1 + step for the pivots); J0: the pivots; v: KMAX
// doubles.  Returns r.  Called by the whole CTA.
__device__ int alg1tor_cta(double* M, int ldm, int k, int nc, double tol, double* s, int32_t* pos, int32_t* J0,
                           double* v, CandRed* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int c = tid; c < nc; c += nt) {
    double a = 0.0;
    for (int i = 0; i < k; ++i) a = fma(M[(int64_t)i * ldm + c], M[(int64_t)i * ldm + c], a);
    s[c] = a;
    pos[c] = 0;
  }
  __syncthreads();
  const int gmax = min(k, nc);
  double thr = 0.0;
  int g = 0;
  for (; g < gmax; ++g) {
    Cand mine = cand_none();
    for (int c = tid; c < nc; c += nt)
      if (!pos[c]) cand_consider(mine, mag_key(s[c]), 0, c);
    unsigned long long fl = 0;
    const Cand w = block_best(mine, fl, red);
    if (w.key == 0ull || w.key == mag_key(0.0)) break;
    const int js = w.j;
    const double nrm = sqrt(s[js]);
    if (g == 0) thr = tol * nrm;
    else if (!(nrm > thr)) break;
    const double x0 = M[(int64_t)g * ldm + js];
    const double alpha = (x0 >= 0.0) ? -nrm : nrm;
    const double tau = 1.0 / (nrm * (nrm + fabs(x0)));
    const int len = k - g;
    for (int i = tid; i < len; i += nt) v[i] = (i == 0) ? x0 - alpha : M[(int64_t)(g + i) * ldm + js];
    if (tid == 0) {
      pos[js] = g + 1;
      J0[g] = js;
    }
    __syncthreads();
    for (int c = tid; c < nc; c += nt) {
      if (pos[c]) continue;
      double t = 0.0;
      for (int i = 0; i < len; ++i) t = fma(v[i], M[(int64_t)(g + i) * ldm + c], t);
      const double cc = tau * t;
      double a = 0.0;
      for (int i = 0; i < len; ++i) {
        const double y = fma(-cc, v[i], M[(int64_t)(g + i) * ldm + c]);
        M[(int64_t)(g + i) * ldm + c] = y;
        if (i > 0) a = fma(y, y, a);
      }
      s[c] = a;
    }
    for (int i = tid; i < len; i += nt) M[(int64_t)(g + i) * ldm + js] = (i == 0) ? alpha : 0.0;
    __syncthreads();
  }
  return g;
}

__global__ void __launch_bounds__(NT) prjvol_kernel(OvArgs B) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_b;
  __shared__ double s_x[KMAX];
  __shared__ double s_g[2];
  __shared__ double s_rho[1];
  __shared__ int32_t s_Jw[2 * KMAX];
  double* G = B.scratch + (size_t)blockIdx.x * B.scratch_stride;
  double* gstrip = G + (size_t)B.kmax * B.lmax;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (;;) {
    const int b = ov_next_block(B, &s_b);
    if (b < 0) break;
    int32_t* info = B.info + LRA_INFO_LEN * (size_t)b;
    CaArgs A;
    int64_t nr, nc;
    int k, lb;
    if (!ov_block_begin(B, b, true, gstrip, A, nr, nc, k, lb)) continue;
    A.max_swaps = B.max_swaps;
    int32_t* Jb = B.J + (size_t)b * B.lmax;
    int l = k, st = LRA_OK, nsw = 0, r = 0;
    {
      const CaSmem S = ca_smem_carve(smem, k, A.ldm, A.gstrip);
      for (int a = tid; a < k; a += nt) S.Is[a] = B.Iin[(size_t)b * B.kmax + a];
      if (tid == 0) S.ctl[0] = 0;
      __syncthreads();
      // the strip W'[I, :] (k x nc)
      if (gather_chunk(A.P, 0, S, k, 0, (int)nc, A.ldm, Map2D((int)nc))) atomicOr(&S.ctl[0], 1);
      __syncthreads();
      if (S.ctl[0]) {
        for (int e = tid; e < LRA_INFO_LEN; e += nt)
          info[e] = (e == 3) ? LRA_ERR_NONFINITE : (e == 6 || e == 7) ? k : 0;
        continue;
      }
      // stage 1: R' (rows 0..r-1 of M, in place) and the pivots J0 (into S.Js)
      r = alg1tor_cta(S.M, A.ldm, k, (int)nc, B.rank_tol, S.tq, S.pos, S.Js, s_x, S.red);
      if (r == 0) {
        // a zero strip: the square generator as given
        for (int a = tid; a < k; a += nt) Jb[a] = B.Jin[(size_t)b * B.kmax + a];
        st = LRA_WARN_RANK_DEFICIENT;
      } else {
        // stage 2: dominance swaps on R' from J0, then greedy expansions to lb columns
        CaArgs A2 = A;
        A2.k = r;
        unsigned long long seq = 0;
        const StepResult sr = maxvol_step<SoloGroup, true>(SoloGroup{}, A2, S, 0, false, S.Js, seq, true);
        __syncthreads();
        st = sr.status;
        nsw = sr.nswaps;
        if (st != LRA_OK && st < 16) {
          for (int e = tid; e < LRA_INFO_LEN; e += nt) info[e] = (e == 3) ? st : (e == 6 || e == 7) ? k : 0;
          continue;
        }
        for (int a = tid; a < r; a += nt) s_Jw[a] = S.Js[a];
        double* M = S.M;
        double* s = S.tq;
        for (int c = tid; c < nc; c += nt) {
          double v = 0.0;
          for (int i = 0; i < r; ++i) v = fma(M[(int64_t)i * A.ldm + c], M[(int64_t)i * A.ldm + c], v);
          s[c] = v;
        }
        if (tid == 0) s_rho[0] = 1.0;
        __syncthreads();
        l = r;
        ov_expand(M, A.ldm, s, S.pos, s_Jw, l, r, (int)nc, lb - r, s_rho, s_x, s_g, S.red);
        for (int a = tid; a < l; a += nt) Jb[a] = s_Jw[a];
      }
    }
    ov_block_finish(B, b, A, nr, nc, k, l, Jb, st, nsw, r, G, smem);
  }
}

struct OvPlan {
  int grid;
  size_t smem, scratch_stride, backup_offset, bytes;
};

static lra_status ov_plan(bool prj, int kmax, int lmax, int64_t max_len, int pmax, OvPlan* pl) {
  const void* kern =
      prj ? reinterpret_cast<const void*>(prjvol_kernel) : reinterpret_cast<const void*>(oversample_kernel);
  DeviceInfo dev;
  lra_status st = current_device_info(&dev);
  if (st != LRA_OK) return st;
  const size_t budget = dev.smem_optin - 4096;
  const int ldm = (int)max_len;
  const size_t fixed = ca_smem_fixed(kmax, ldm), strip = sizeof(double) * (size_t)kmax * ldm;
  size_t need = std::max(fixed, nucleus_rect_smem_bytes(kmax, lmax));
  bool gstrip = true;
  if (std::max(fixed + strip, need) <= budget) { need = std::max(fixed + strip, need); gstrip = false; }
  if (need > budget) return LRA_ERR_INVALID_ARG;
  LRA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
  int occ = 0;
  LRA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, need));
  if (occ < 1) return LRA_ERR_INVALID_ARG;
  pl->grid = occ * dev.sms;
  pl->smem = need;
  pl->backup_offset = (size_t)kmax * lmax + (gstrip ? (size_t)kmax * max_len : 0);
  pl->scratch_stride = align_up(pl->backup_offset + (pmax > 0 ? (size_t)(kmax + 1) * max_len : 0), 32);
  pl->bytes = align_up(256 + sizeof(double) * pl->scratch_stride * pl->grid, 256);
  return LRA_OK;
}

static lra_status ov_check(bool prj, const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                           int32_t pextra, int32_t pmax, DevProblem* P) {
  lra_status st = make_dev_problem(base, nullptr, P);
  if (st != LRA_OK) return st;
  if (batch == nullptr || par == nullptr || batch->blocks == nullptr || batch->offsets == nullptr || batch->nb < 1 ||
      batch->max_len < 1)
    return LRA_ERR_INVALID_ARG;
  if (par->k < 1 || par->k > KMAX || pextra < 0 || pextra > KMAX || !(par->h >= 1.0) || !(par->h < 1e300) ||
      !(par->rank_tol >= 0.0) || !(par->rank_tol < 1.0))
    return LRA_ERR_INVALID_ARG;
  if (pmax < 0 || pmax > PMAX || (pmax > 0 && par->max_swaps < 0)) return LRA_ERR_INVALID_ARG;
  if (prj && (pmax != 0 || par->max_swaps < 0)) return LRA_ERR_INVALID_ARG;
  return LRA_OK;
}

static lra_status ov_run(bool prj, const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                         int32_t pextra, int32_t pmax, const lra_cur_batch* in, const lra_cur_batch* out,
                         void* workspace, size_t workspace_bytes, cudaStream_t stream) {
  DevProblem P;
  lra_status st = ov_check(prj, base, batch, par, pextra, pmax, &P);
  if (st != LRA_OK) return st;
  if (in == nullptr || out == nullptr || !in->I || !in->J || !in->info || !out->I || !out->J || !out->C || !out->U ||
      !out->R || !out->info)
    return LRA_ERR_INVALID_ARG;
  OvPlan pl;
  if ((st = ov_plan(prj, par->k, par->k + pextra, batch->max_len, pmax, &pl)) != LRA_OK) return st;
  if (workspace == nullptr || workspace_bytes < pl.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255u))
    return LRA_ERR_WORKSPACE;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  OvArgs A;
  std::memset(&A, 0, sizeof(A));
  A.base = P;
  A.blocks = batch->blocks;
  A.offs = batch->offsets;
  A.order = batch->order;
  A.nb = batch->nb;
  A.kmax = par->k;
  A.pextra = pextra;
  A.lmax = par->k + pextra;
  A.pmax = pmax;
  A.max_cycles = pmax > 0 ? par->max_swaps : 0;
  A.max_swaps = prj ? par->max_swaps : 0;
  A.h = par->h;
  A.rank_tol = par->rank_tol;
  A.Iin = in->I;
  A.Jin = in->J;
  A.info_in = in->info;
  A.I = out->I;
  A.J = out->J;
  A.C = out->C;
  A.R = out->R;
  A.U = out->U;
  A.info = out->info;
  A.counter = reinterpret_cast<unsigned int*>(ws);
  A.scratch = reinterpret_cast<double*>(ws + 256);
  A.scratch_stride = pl.scratch_stride;
  A.backup_offset = pl.backup_offset;
  A.smem_bytes = pl.smem;
  A.max_len = batch->max_len;
  LRA_CUDA_TRY(cudaMemsetAsync(ws, 0, 256, stream));
  if (prj) {
    LaunchScope ls(stream, "prjvol_kernel");
    prjvol_kernel<<<pl.grid, NT, pl.smem, stream>>>(A);
  } else {
    LaunchScope ls(stream, "oversample_kernel");
    oversample_kernel<<<pl.grid, NT, pl.smem, stream>>>(A);
  }
  return cuda_status(cudaGetLastError());
}

static lra_status ov_workspace(bool prj, const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                               int32_t pextra, int32_t pmax, size_t* bytes) {
  if (bytes == nullptr) return LRA_ERR_INVALID_ARG;
  DevProblem P;
  lra_status st = ov_check(prj, base, batch, par, pextra, pmax, &P);
  if (st != LRA_OK) return st;
  OvPlan pl;
  if ((st = ov_plan(prj, par->k, par->k + pextra, batch->max_len, pmax, &pl)) != LRA_OK) return st;
  *bytes = pl.bytes;
  return LRA_OK;
}

}  // namespace lra

using namespace lra;

extern "C" {

lra_status lra_oversample_batched_workspace_size(const lra_problem* base, const lra_batch* batch,
                                                 const lra_ca_params* par, int32_t pextra, size_t* bytes) {
  return ov_workspace(false, base, batch, par, pextra, 0, bytes);
}

lra_status lra_oversample_batched(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                                  int32_t pextra, const lra_cur_batch* in, const lra_cur_batch* out, void* workspace,
                                  size_t workspace_bytes, lra_stream_t stream) {
  return ov_run(false, base, batch, par, pextra, 0, in, out, workspace, workspace_bytes,
                reinterpret_cast<cudaStream_t>(stream));
}

lra_status lra_oversample_cycle_batched_workspace_size(const lra_problem* base, const lra_batch* batch,
                                                       const lra_ca_params* par, int32_t pextra, int32_t pmax,
                                                       size_t* bytes) {
  return ov_workspace(false, base, batch, par, pextra, pmax, bytes);
}

lra_status lra_oversample_cycle_batched(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                                        int32_t pextra, int32_t pmax, const lra_cur_batch* in,
                                        const lra_cur_batch* out, void* workspace, size_t workspace_bytes,
                                        lra_stream_t stream) {
  return ov_run(false, base, batch, par, pextra, pmax, in, out, workspace, workspace_bytes,
                reinterpret_cast<cudaStream_t>(stream));
}

lra_status lra_prjvol_batched_workspace_size(const lra_problem* base, const lra_batch* batch,
                                             const lra_ca_params* par, int32_t pextra, size_t* bytes) {
  return ov_workspace(true, base, batch, par, pextra, 0, bytes);
}

lra_status lra_prjvol_batched(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                              int32_t pextra, const lra_cur_batch* in, const lra_cur_batch* out, void* workspace,
                              size_t workspace_bytes, lra_stream_t stream) {
  return ov_run(true, base, batch, par, pextra, 0, in, out, workspace, workspace_bytes,
                reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
