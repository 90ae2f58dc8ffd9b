/*
 * lra_oracle.c -- plain, slow, FP64 CPU oracle for cross-approximation (C-A)
 * CUR low-rank approximation, written from "Superfast Accurate Low Rank
 * Approximation" (Pan, Luan, Svadlenka, Zhao, arXiv:1710.07946).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header or constant with
 * the CUDA path.
 *
 * Everything is FP64, single-threaded, written for a reader to check against
 * the paper by eye: no blocking, no fusion, no reordering.  Where a floating
 * point result feeds a discrete decision (an argmax), the operation order is
 * fixed as stated in each function so that an independent implementation can
 * reproduce the decision: every dot product is an ascending-index chain of
 * correctly rounded fma(), every division is one IEEE division, ties in an
 * argmax go to the lowest index.  Build with -ffp-contract=off.
 *
 * Paper passages followed (section / algorithm / equation names are the
 * paper's LaTeX labels):
 *   - C-A iterations: Section "CUR LRA; primitive, cynical, and
 *     cross-approximation algorithms" and the Tests 2 set-up of Section
 *     "Tests ..." (random initial rows, horizontal step then vertical step).
 *   - Dominant submatrix (maxvol): Algorithm "Computing a dominant submatrix"
 *     (algdomin) with its LUP initialisation, Algorithm "An iterative C-A
 *     algorithm by means of recursive LUP factorization" (alggos).
 *   - Nucleus: Algorithm "Canonical computation of a nucleus" (algcnnncl),
 *     with a rank-revealing QR in place of the SVD as Remark reubsc allows.
 *   - Abridged Hadamard multiplier: Appendix "Abridged Hadamard and Fourier
 *     Multipliers", equations eqrfd / eqbschf, randomised as D H P.
 *   - Sparse +-1 multiplier: Section "Pre-processing with quasi Gaussian
 *     matrices", case (i).
 *   - Back-transform of a pre-processed CUR: Algorithm alglratpsvd1, stage 4
 *     (R = R_H H^+, which is W[I,:] for an orthogonal multiplier).
 *   - Sampled a-posteriori error: Section "Superfast a posteriori error
 *     estimation for LRA of a matrix filled with i.i.d. values".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Problem description (the oracle's own; not shared with the library) */
/* ------------------------------------------------------------------ */
enum { ORC_DENSE = 0, ORC_LAPLACE = 1, ORC_GAUSSIAN = 2 };
enum { ORC_F64 = 0, ORC_F32 = 1, ORC_BF16 = 2 };
enum { ORC_MULT_NONE = 0, ORC_MULT_ARHT = 1, ORC_MULT_SPARSE = 2, ORC_MULT_BIDIAG = 3, ORC_MULT_ARFT = 4 };

typedef struct {
  int32_t src;          /* ORC_DENSE / ORC_LAPLACE / ORC_GAUSSIAN            */
  int32_t dtype;        /* dense storage type: ORC_F64 or ORC_F32             */
  int64_t m, n;         /* matrix size                                        */
  const void* W;        /* dense: row-major, leading dimension ldw            */
  int64_t ldw;
  const double* X;      /* kernel: m target points, xyz interleaved (m x 3)   */
  const double* Y;      /* kernel: n source points (n x 3)                    */
  double ell;           /* Gaussian length scale                              */
  int32_t mkind;        /* multiplier kind                                    */
  int32_t depth;        /* ARHT recursion depth d (n = 2^d s)                 */
  const int32_t* perm;  /* ARHT permutation P: column j of H P = column perm[j] of H */
  const int8_t* dsign;  /* ARHT diagonal D: +-1, length n                     */
  int32_t nnz;          /* sparse: nonzeros per column                        */
  const int32_t* srow;  /* sparse: n*nnz row indices, ascending per column    */
  const int8_t* ssign;  /* sparse: n*nnz signs (+-1)                          */
  /* bidiagonal products (mkind ORC_MULT_BIDIAG, depth = q factors; perm and
   * dsign hold q x n permutations and signs): the columns of the product,
   * expanded by orc_bidiag_columns, min(2^q, n) slots each, ascending rows, value 0
   * marking an unused slot */
  const int32_t* brow;
  const int32_t* bval;
  /* side of the multiplier (Remark re2orddmn): 0 = right, W' = W M with M
   * n x n; 1 = left, W' = M^T W with M m x m (for m > n) */
  int32_t mside;
  /* abridged randomized Fourier multiplier in real form (mkind ORC_MULT_ARFT,
   * right side only, depth = d): W' = W [Re M, Im M] with M = D Omega_{n,d} P,
   * so W' has 2n columns.  The columns of [Re M, Im M] before the scale
   * 2^(-d/2), expanded by orc_fourier_columns: 2^d slots each (ascending rows,
   * real weights). */
  const int32_t* frow;
  const double* fwt;
  const double* dre;    /* ARFT diagonal D: real and imaginary parts (n each) */
  const double* dim;
} orc_problem;

/* pi to double precision, for the roots of unity of the Fourier multiplier */
#define ORC_PI 3.14159265358979323846

/* Columns of W' (the pre-processed matrix): 2n for the real-form abridged
 * Fourier multiplier, n otherwise. */
static int64_t orc_cols(const orc_problem* p) { return p->mkind == ORC_MULT_ARFT ? 2 * p->n : p->n; }

/* x rounded to bfloat16 (8 significant bits: the upper half of the IEEE single
 * pattern), to nearest with ties to even, returned as a float.  For finite x. */
static float round_bf16(float x) {
  uint32_t u;
  memcpy(&u, &x, sizeof u);
  uint32_t keep = u >> 16;
  uint32_t rest = u & 0xFFFFu;
  if (rest > 0x8000u || (rest == 0x8000u && (keep & 1u))) keep += 1u;
  uint32_t r = keep << 16;
  float y;
  memcpy(&y, &r, sizeof y);
  return y;
}

/* Entry w_ij of the input W (no multiplier).  Kernel entries follow the
 * closed forms: Laplace 1/|x-y|, Gaussian exp(-|x-y|^2 / (2 l^2)). */
static double entry_w(const orc_problem* p, int64_t i, int64_t j) {
  if (p->src == ORC_DENSE) {
    if (p->dtype == ORC_F32) return (double)((const float*)p->W)[i * p->ldw + j];
    return ((const double*)p->W)[i * p->ldw + j];
  }
  const double* x = p->X + 3 * i;
  const double* y = p->Y + 3 * j;
  double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
  double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
  if (p->src == ORC_LAPLACE) {
    if (p->dtype == ORC_F32 || p->dtype == ORC_BF16) {
      /* FP32 entries: r2 rounded to single precision, then the IEEE single
       * square root and quotient, each correctly rounded. */
      float r2f = (float)r2;
      float sf = sqrtf(r2f);
      float ef = 1.0f / sf;
      if (p->dtype == ORC_BF16) return (double)round_bf16(ef);
      return (double)ef;
    }
    return 1.0 / sqrt(r2);
  }
  return exp(-(r2 / (2.0 * p->ell * p->ell)));
}

/* Columns of the product M = F_1 F_2 ... F_q of the paper's quasi-Gaussian
 * factors F_i = (I + D_i S) P_i (section "Approximation of a Gaussian matrix by
 * the product of random bidiagonal matrices", eq. def11): S the cyclic
 * down-shift, D_i = diag(signs[i]), column a of P_i = e_{perms[i][a]}, so that
 * F_i e_a = e_b + signs[i][b'] e_{b'} with b = perms[i][a], b' = (b + 1) mod n.
 * Column j is M e_j = F_1 (F_2 (... (F_q e_j))): a dense work vector, then its
 * nonzeros in ascending rows into min(2^q, n) slots (a column has at most that
 * many; integer values, |value| <= 2^q; 0 = unused). */
void orc_bidiag_columns(int64_t n, int32_t q, const int32_t* perms, const int8_t* signs, int32_t* rows,
                        int32_t* vals) {
  int64_t w = (1LL << q) < n ? (1LL << q) : n;
  int64_t* v = (int64_t*)calloc((size_t)n, sizeof(int64_t));
  int64_t* u = (int64_t*)calloc((size_t)n, sizeof(int64_t));
  for (int64_t j = 0; j < n; ++j) {
    memset(v, 0, sizeof(int64_t) * (size_t)n);
    v[j] = 1;
    for (int32_t f = q - 1; f >= 0; --f) {
      memset(u, 0, sizeof(int64_t) * (size_t)n);
      for (int64_t a = 0; a < n; ++a) {
        if (v[a] == 0) continue;
        int64_t b = perms[(int64_t)f * n + a];
        int64_t b1 = (b + 1) % n;
        u[b] += v[a];
        u[b1] += (int64_t)signs[(int64_t)f * n + b1] * v[a];
      }
      memcpy(v, u, sizeof(int64_t) * (size_t)n);
    }
    int64_t c = 0;
    for (int64_t a = 0; a < n; ++a)
      if (v[a] != 0 && c < w) { rows[j * w + c] = (int32_t)a; vals[j * w + c] = (int32_t)v[a]; ++c; }
    for (; c < w; ++c) { rows[j * w + c] = 0; vals[j * w + c] = 0; }
  }
  free(v); free(u);
}

/* 2^(-d/2): the scale that makes the abridged Hadamard matrix orthogonal
 * ("orthogonal up to scaling", appendix on abridged multipliers). */
static double arht_scale(int d) { return 1.0 / sqrt((double)(1LL << d)); }

static int popcount32(uint32_t v) { int c = 0; while (v) { c += (int)(v & 1u); v >>= 1; } return c; }

/* One term of a pre-processed entry: the input entry that row r of the
 * combining column of M multiplies.  Right multiplier, W' = W M: w'_ij = sum_r
 * w_ir M_rj, so column j of M combines entries of row i.  Left multiplier,
 * W' = M^T W: w'_ij = sum_r M_ri w_rj, so column i of M combines entries of
 * column j. */
static double entry_term(const orc_problem* p, int64_t i, int64_t j, int64_t r) {
  return p->mside ? entry_w(p, r, j) : entry_w(p, i, r);
}

/* Entry w'_ij of the pre-processed matrix W' = W M (or M^T W).  Below, c is
 * the column of M that combines the terms (j for the right side, i for the
 * left) and N the order of M.
 * ARHT: M = 2^(-d/2) D H_{N,d} P with H_{N,d} = H_{2^d} (x) I_s, N = 2^d s
 *   (recursion eqrfd cut at depth d with H_s = I_s).  With perm[c] = b s + t,
 *   column c of M holds 2^d nonzeros, at rows a s + t, a = 0..2^d-1, equal to
 *   2^(-d/2) D_{a s + t} (-1)^{popcount(a & b)}.  The 2^d terms are summed in
 *   ascending a, then scaled once.
 * Sparse +-1: column c of M holds nnz entries +-1/2 (for nnz = 4; in general
 *   +-1/sqrt(nnz)) at rows srow[c*nnz + t]; summed in ascending t, scaled once. */
static double entry_wp(const orc_problem* p, int64_t i, int64_t j) {
  if (p->mkind == ORC_MULT_NONE) return entry_w(p, i, j);
  int64_t c = p->mside ? i : j;
  int64_t N = p->mside ? p->m : p->n;
  if (p->mkind == ORC_MULT_ARHT) {
    int64_t s = N >> p->depth;
    int64_t pc = p->perm[c];
    int64_t b = pc / s, t = pc % s;
    double acc = 0.0;
    for (int64_t a = 0; a < (1LL << p->depth); ++a) {
      int64_t r = a * s + t;
      double v = entry_term(p, i, j, r) * (double)p->dsign[r];
      if (popcount32((uint32_t)(a & b)) & 1) acc = acc - v; else acc = acc + v;
    }
    return acc * arht_scale(p->depth);
  }
  if (p->mkind == ORC_MULT_ARFT) {
    /* the 2^d real weights of column j of [Re M, Im M] in ascending rows, each an
     * fma, then the scale 2^(-d/2) */
    int64_t w = 1LL << p->depth;
    double acc = 0.0;
    for (int64_t t = 0; t < w; ++t) acc = fma(p->fwt[j * w + t], entry_w(p, i, p->frow[j * w + t]), acc);
    return acc * arht_scale(p->depth);
  }
  if (p->mkind == ORC_MULT_BIDIAG) {
    /* nonzero slots in ascending row order, each an fma with its integer weight */
    int64_t w = (1LL << p->depth) < N ? (1LL << p->depth) : N;
    double acc = 0.0;
    for (int64_t t = 0; t < w; ++t) {
      int32_t v = p->bval[c * w + t];
      if (v == 0) continue;
      acc = fma((double)v, entry_term(p, i, j, p->brow[c * w + t]), acc);
    }
    return acc * arht_scale(p->depth);
  }
  /* sparse */
  double acc = 0.0;
  for (int t = 0; t < p->nnz; ++t) {
    int64_t r = p->srow[c * p->nnz + t];
    double v = entry_term(p, i, j, r);
    if (p->ssign[c * p->nnz + t] < 0) acc = acc - v; else acc = acc + v;
  }
  return acc * (1.0 / sqrt((double)p->nnz));
}

/* Row strip W'[I,:] (k x n', n' = orc_cols(p), row-major). */
void orc_gather_rows(const orc_problem* p, const int32_t* I, int32_t k, double* out) {
  int64_t nc = orc_cols(p);
  for (int32_t a = 0; a < k; ++a)
    for (int64_t j = 0; j < nc; ++j) out[(int64_t)a * nc + j] = entry_wp(p, I[a], j);
}

/* Column strip W'[:,J], stored transposed: out[a*m + i] = W'[i, J[a]]. */
void orc_gather_cols_t(const orc_problem* p, const int32_t* J, int32_t k, double* out) {
  for (int32_t a = 0; a < k; ++a)
    for (int64_t i = 0; i < p->m; ++i) out[(int64_t)a * p->m + i] = entry_wp(p, i, J[a]);
}

/* Original rows W[I,:] (no multiplier), k x n. */
void orc_gather_rows_orig(const orc_problem* p, const int32_t* I, int32_t k, double* out) {
  for (int32_t a = 0; a < k; ++a)
    for (int64_t j = 0; j < p->n; ++j) out[(int64_t)a * p->n + j] = entry_w(p, I[a], j);
}

/* The factors of the CUR of W from a generator (I, J) of W' = M^T W (a left
 * multiplier): W ~ W[:, J] pinv(W'[I, J]) W'[I, :], which is reading 1's
 * back-transform (C from W', R from W) applied to W^T = W^T M.  So C holds the
 * original columns (m x kJ) and R the pre-processed rows (kI x n).  Called after
 * the core W'[I, J] has been taken; a no-op for a right multiplier. */
static void left_outputs(const orc_problem* p, const int32_t* I, int32_t kI, const int32_t* J, int32_t kJ,
                         double* C, double* R) {
  if (!p->mside || p->mkind == ORC_MULT_NONE) return;
  for (int64_t i = 0; i < p->m; ++i)
    for (int32_t a = 0; a < kJ; ++a) C[i * kJ + a] = entry_w(p, i, J[a]);
  orc_gather_rows(p, I, kI, R);
}

/* ------------------------------------------------------------------ */
/* Maxvol on a k x n strip (dominant k x k submatrix)                  */
/* ------------------------------------------------------------------ */
enum { ORC_OK = 0, ORC_ERR_NONFINITE = 3, ORC_WARN_RANK_DEFICIENT = 16, ORC_WARN_NOT_CONVERGED = 17 };

static int all_finite(const double* a, int64_t cnt) {
  for (int64_t i = 0; i < cnt; ++i) if (!isfinite(a[i])) return 0;
  return 1;
}

/*
 * orc_maxvol: find k columns J of the k x n matrix A (row-major) whose k x k
 * submatrix B = A[:,J] is dominant (every entry of B^{-1} A bounded by h).
 *
 * Initialisation (Algorithm alggos, stages 1-2):
 *   cold  (Jwarm == NULL): LU factorisation with column pivoting, A P^T = L (U0 | U1).
 *         At elimination step t the pivot column is the unchosen column with the
 *         largest |A(t)[t, q]| (lowest q on ties); rows t+1.. are eliminated with
 *         multipliers l_p = A(t)[p, j_t] / A(t)[t, j_t] and
 *         A[p][q] <- fma(-l_p, A[t][q], A[p][q]) over the unchosen columns q.
 *   warm  (Jwarm given, C-A sweeps after the first): the same elimination with the
 *         pivot columns forced to Jwarm[0..k-1] in order and partial pivoting over
 *         rows (pivot row = largest |A(t)[p, j_t]|, p >= t, lowest p on ties;
 *         rows t and that row are exchanged across the whole strip).
 *   Then C = Bbar^{-1} A = (I | U0^{-1} U1) in the original column order: each
 *   unchosen column b is solved by column-sweep back substitution with U0
 *   (for i = k-1 down to 0: x_i = b_i * (1 / U0[i][i]), then
 *   b_p <- fma(-U0[p][i], x_i, b_p) for p < i); column J[i] of C is e_i.
 * Swaps (Algorithm algdomin, stages 1-2): take the entry of largest |C[i][j]|
 *   over i < k and j not in J, ties to the lowest j then the lowest i.  Stop when
 *   it is <= h.  Otherwise J[i*] <- j* and C is updated in place to the new
 *   B^{-1} A: with c* = C[i*][j*] and the old column x = C[:, j*],
 *   for every column q:  t_q = C[i*][q] * (1 / c*);  C[i*][q] = t_q;
 *   C[p][q] = fma(-x[p], t_q, C[p][q]) for p != i*; column j* is then set to
 *   e_{i*} exactly.
 *   Every division is one reciprocal per pivot (1 / pivot) followed by
 *   multiplications, the same solve with one rounding more per entry.
 *   |det B| is multiplied by |c*| at each swap (strict volume increase for h >= 1).
 * Outputs: J (position i of J is row i of C), C (k x n) if Cout != NULL,
 *   logdet = log|det A[:,J]| (LU diagonal at init, + log|c*| per swap), number of
 *   swaps; the status is ORC_WARN_RANK_DEFICIENT if a zero pivot was met (no
 *   swaps are then made) and ORC_WARN_NOT_CONVERGED if max_swaps stopped the loop.
 *   A zero warm pivot falls back to the cold start.
 */
int orc_maxvol(const double* A, int32_t k, int64_t n, const int32_t* Jwarm, double h, int32_t max_swaps,
               int32_t* J, double* Cout, double* logdet_out, int32_t* nswaps_out) {
  double* M = (double*)malloc(sizeof(double) * (size_t)k * (size_t)n);
  double* U0 = (double*)malloc(sizeof(double) * (size_t)k * (size_t)k);
  double* x = (double*)malloc(sizeof(double) * (size_t)k);
  unsigned char* chosen = (unsigned char*)calloc((size_t)n, 1);
  int status = ORC_OK;
  int warm = (Jwarm != NULL);
  double logdet = 0.0;

restart:
  memcpy(M, A, sizeof(double) * (size_t)k * (size_t)n);
  memset(chosen, 0, (size_t)n);
  logdet = 0.0;
  status = ORC_OK;
  for (int32_t t = 0; t < k; ++t) {
    int64_t jt;
    if (!warm) {
      double bv = -1.0; jt = -1;
      for (int64_t q = 0; q < n; ++q)
        if (!chosen[q] && fabs(M[t * n + q]) > bv) { bv = fabs(M[t * n + q]); jt = q; }
    } else {
      jt = Jwarm[t];
      int32_t r = t; double bv = fabs(M[(int64_t)t * n + jt]);
      for (int32_t p = t + 1; p < k; ++p)
        if (fabs(M[(int64_t)p * n + jt]) > bv) { bv = fabs(M[(int64_t)p * n + jt]); r = p; }
      if (r != t)
        for (int64_t q = 0; q < n; ++q) { double tmp = M[(int64_t)t * n + q]; M[(int64_t)t * n + q] = M[(int64_t)r * n + q]; M[(int64_t)r * n + q] = tmp; }
    }
    J[t] = (int32_t)jt;
    chosen[jt] = 1;
    double piv = M[(int64_t)t * n + jt];
    if (piv == 0.0) {
      if (warm) { warm = 0; goto restart; }
      status = ORC_WARN_RANK_DEFICIENT;
      continue;                       /* nothing to eliminate with */
    }
    logdet += log(fabs(piv));
    double rpiv = 1.0 / piv;
    for (int32_t p = t + 1; p < k; ++p) {
      double l = M[(int64_t)p * n + jt] * rpiv;
      for (int64_t q = 0; q < n; ++q)
        if (!chosen[q]) M[(int64_t)p * n + q] = fma(-l, M[(int64_t)t * n + q], M[(int64_t)p * n + q]);
    }
  }
  if (status == ORC_WARN_RANK_DEFICIENT) {
    if (Cout) memset(Cout, 0, sizeof(double) * (size_t)k * (size_t)n);
    *logdet_out = -INFINITY; *nswaps_out = 0;
    free(M); free(U0); free(x); free(chosen);
    return status;
  }
  /* U0[s][t] = final row s of pivot column J[t], s <= t */
  for (int32_t s = 0; s < k; ++s)
    for (int32_t t = 0; t < k; ++t) U0[s * k + t] = (s <= t) ? M[(int64_t)s * n + J[t]] : 0.0;
  /* C = (I | U0^{-1} U1) in original column order; reuse M column by column */
  for (int32_t i = 0; i < k; ++i) x[i] = 1.0 / U0[i * k + i];     /* reciprocals of the diagonal */
  for (int64_t q = 0; q < n; ++q) {
    if (chosen[q]) continue;
    for (int32_t i = k - 1; i >= 0; --i) {
      double xi = M[(int64_t)i * n + q] * x[i];
      M[(int64_t)i * n + q] = xi;
      for (int32_t p = 0; p < i; ++p) M[(int64_t)p * n + q] = fma(-U0[p * k + i], xi, M[(int64_t)p * n + q]);
    }
  }
  for (int32_t t = 0; t < k; ++t)
    for (int32_t i = 0; i < k; ++i) M[(int64_t)i * n + J[t]] = (i == t) ? 1.0 : 0.0;

  /* dominance swaps */
  int32_t nsw = 0;
  for (;;) {
    double bv = -1.0; int64_t bj = -1; int32_t bi = -1;
    for (int64_t q = 0; q < n; ++q) {
      if (chosen[q]) continue;
      for (int32_t i = 0; i < k; ++i)
        if (fabs(M[(int64_t)i * n + q]) > bv) { bv = fabs(M[(int64_t)i * n + q]); bj = q; bi = i; }
    }
    if (bj < 0 || !(bv > h)) break;
    if (nsw >= max_swaps) { status = ORC_WARN_NOT_CONVERGED; break; }
    double cs = M[(int64_t)bi * n + bj];
    double rcs = 1.0 / cs;
    for (int32_t p = 0; p < k; ++p) x[p] = M[(int64_t)p * n + bj];
    for (int64_t q = 0; q < n; ++q) {
      double tq = M[(int64_t)bi * n + q] * rcs;
      M[(int64_t)bi * n + q] = tq;
      for (int32_t p = 0; p < k; ++p)
        if (p != bi) M[(int64_t)p * n + q] = fma(-x[p], tq, M[(int64_t)p * n + q]);
    }
    for (int32_t p = 0; p < k; ++p) M[(int64_t)p * n + bj] = (p == bi) ? 1.0 : 0.0;  /* j* is now e_{i*} */
    chosen[J[bi]] = 0;
    chosen[bj] = 1;
    J[bi] = (int32_t)bj;
    logdet += log(fabs(cs));
    ++nsw;
  }
  if (Cout) memcpy(Cout, M, sizeof(double) * (size_t)k * (size_t)n);
  *logdet_out = logdet;
  *nswaps_out = nsw;
  free(M); free(U0); free(x); free(chosen);
  return status;
}

/* ------------------------------------------------------------------ */
/* Nucleus: U = pseudo-inverse of the rank-r truncation of G (k x k)   */
/* ------------------------------------------------------------------ */

/* Householder reflector on x[0..len-1] (stride str) in the textbook form
 * H = I - tau v v^T, v[0] = 1, H x = beta e_1 (Golub & Van Loan, Sec. 5.1).
 * Returns tau; writes beta into x[0] and v[1..] into x[1..]. */
static double house(double* x, int len, int str) {
  double alpha = x[0];
  double xn2 = 0.0;
  for (int i = 1; i < len; ++i) xn2 = fma(x[i * str], x[i * str], xn2);
  if (xn2 == 0.0) return 0.0;
  double nrm = sqrt(fma(alpha, alpha, xn2));
  double beta = (alpha >= 0.0) ? -nrm : nrm;
  double tau = (beta - alpha) / beta;
  double scal = 1.0 / (alpha - beta);
  for (int i = 1; i < len; ++i) x[i * str] = x[i * str] * scal;
  x[0] = beta;
  return tau;
}

/* Squared norm of column segment x[0..len-1] (unit stride): one ascending fma chain. */
static double sqnorm(const double* x, int len) {
  double s = 0.0;
  for (int i = 0; i < len; ++i) s = fma(x[i], x[i], s);
  return s;
}

/* Apply H = I - tau v v^T (v[0] = 1 implicit, v[1..] at vv[1..], stride vs)
 * from the left to column segment y[0..len-1] (stride ys). */
static void apply_house(const double* vv, int vs, double tau, double* y, int len, int ys) {
  if (tau == 0.0) return;
  double w = y[0];
  for (int i = 1; i < len; ++i) w = fma(vv[i * vs], y[i * ys], w);
  double c = tau * w;
  y[0] = y[0] - c;
  for (int i = 1; i < len; ++i) y[i * ys] = fma(-c, vv[i * vs], y[i * ys]);
}

/*
 * orc_nucleus: Algorithm algcnnncl with a rank-revealing factorisation in place
 * of the SVD (Remark reubsc).
 *   1. Householder QR with column pivoting (Businger-Golub): G P = Q R; at step t
 *      the column with the largest remaining squared norm (rows t.., recomputed)
 *      is moved to position t, lowest index on ties.  Every inner product of
 *      this QR (the column norms, ||x||^2 of each reflector, v^T y of each
 *      application) is one ascending fma chain.
 *   2. Numerical rank r = number of leading |R_tt| > tol |R_00|.
 *   3. U = pinv(G_r) for the truncation G_r = Q_r [R11 R12] P^T: with
 *      T = [R11 R12] (r x k) and the QR factorisation T^T = Z S,
 *      pinv(G_r) = P Z S^{-T} Q_r^T (complete orthogonal decomposition;
 *      equals P R^{-1} Q^T when r = k).
 * G and U are k x k row-major; U[j][i] maps row i of W'[:,J] ... i.e. U is the
 * l x k nucleus with l = k.  Returns r.
 */
int32_t orc_nucleus(const double* G, int32_t k, double tol, double* U) {
  /* column-major working copy: A[col*k + row] */
  double* A = (double*)malloc(sizeof(double) * (size_t)k * (size_t)k);
  double* taus = (double*)malloc(sizeof(double) * (size_t)k);
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  for (int32_t i = 0; i < k; ++i)
    for (int32_t j = 0; j < k; ++j) A[j * k + i] = G[i * k + j];
  for (int32_t j = 0; j < k; ++j) perm[j] = j;
  for (int32_t t = 0; t < k; ++t) {
    int32_t pj = t; double bn = -1.0;
    for (int32_t j = t; j < k; ++j) {
      double s = sqnorm(&A[j * k + t], k - t);
      if (s > bn) { bn = s; pj = j; }
    }
    if (pj != t) {
      for (int32_t i = 0; i < k; ++i) { double tmp = A[t * k + i]; A[t * k + i] = A[pj * k + i]; A[pj * k + i] = tmp; }
      int32_t tp = perm[t]; perm[t] = perm[pj]; perm[pj] = tp;
    }
    taus[t] = house(&A[t * k + t], k - t, 1);
    for (int32_t j = t + 1; j < k; ++j) apply_house(&A[t * k + t], 1, taus[t], &A[j * k + t], k - t, 1);
  }
  int32_t r = 0;
  double r00 = fabs(A[0]);
  if (r00 > 0.0)
    while (r < k && fabs(A[r * k + r]) > tol * r00) ++r;

  memset(U, 0, sizeof(double) * (size_t)k * (size_t)k);
  if (r == 0) { free(A); free(taus); free(perm); return 0; }

  /* Qt = Q^T = H_{k-1} ... H_0 applied to I  (column-major, k x k) */
  double* Qt = (double*)calloc((size_t)k * (size_t)k, sizeof(double));
  for (int32_t i = 0; i < k; ++i) Qt[i * k + i] = 1.0;
  for (int32_t t = 0; t < k; ++t)
    for (int32_t j = 0; j < k; ++j) apply_house(&A[t * k + t], 1, taus[t], &Qt[j * k + t], k - t, 1);

  /* T^T (k x r, column-major: column c = row c of T = R[c][0..k-1]) and its QR */
  double* Tt = (double*)calloc((size_t)k * (size_t)r, sizeof(double));
  double* tz = (double*)malloc(sizeof(double) * (size_t)r);
  for (int32_t c = 0; c < r; ++c)
    for (int32_t i = c; i < k; ++i) Tt[c * k + i] = A[i * k + c];
  if (r < k) {
    for (int32_t c = 0; c < r; ++c) {
      tz[c] = house(&Tt[c * k + c], k - c, 1);
      for (int32_t j = c + 1; j < r; ++j) apply_house(&Tt[c * k + c], 1, tz[c], &Tt[j * k + c], k - c, 1);
    }
  } else {
    for (int32_t c = 0; c < r; ++c) tz[c] = 0.0;   /* T^T is already lower -> use R directly */
  }
  /* X (k x k column-major) = Z S^{-T} Q_r^T.
   * For r = k: S^T = R^T... handle uniformly: when r == k we take Z = I and
   * S = R^T (T^T = R^T is lower triangular), i.e. solve S^T V = Q_r^T with
   * S^T = R upper triangular by back substitution. */
  double* X = (double*)calloc((size_t)k * (size_t)k, sizeof(double));
  for (int32_t col = 0; col < k; ++col) {
    /* right-hand side: column col of Q_r^T = (Qt[col*k + 0..r-1]) */
    double* v = &X[col * k];
    if (r == k) {
      /* solve R v = Qt[:,col] (back substitution, descending rows) */
      for (int32_t i = k - 1; i >= 0; --i) {
        double s = Qt[col * k + i];
        for (int32_t p = i + 1; p < k; ++p) s = fma(-A[p * k + i], v[p], s);
        v[i] = s / A[i * k + i];
      }
    } else {
      /* S is r x r upper triangular in Tt (S[i][c] = Tt[c*k + i], i <= c);
       * solve S^T v = Qt[0..r-1, col] by forward substitution */
      for (int32_t i = 0; i < r; ++i) {
        double s = Qt[col * k + i];
        for (int32_t p = 0; p < i; ++p) s = fma(-Tt[i * k + p], v[p], s);
        v[i] = s / Tt[i * k + i];
      }
      /* v (length k, zeros below r) <- Z v = H'_0 ... H'_{r-1} v */
      for (int32_t c = r - 1; c >= 0; --c) apply_house(&Tt[c * k + c], 1, tz[c], &v[c], k - c, 1);
    }
  }
  /* U = P X: row perm[i] of U is row i of X */
  for (int32_t i = 0; i < k; ++i)
    for (int32_t col = 0; col < k; ++col) U[(int64_t)perm[i] * k + col] = X[col * k + i];
  free(A); free(taus); free(perm); free(Qt); free(Tt); free(tz); free(X);
  return r;
}

/*
 * orc_nucleus_rect: the nucleus of a rectangular k x l generator G (k <= l,
 * row-major): U = pinv of the rank-r truncation of its QRP factorisation
 * (Algorithm algcnnncl with Remark reubsc's rank-revealing factorisation),
 * l x k row-major.  As orc_nucleus: Householder QR with column pivoting over
 * the l columns (k steps, column norms over rows t.. recomputed each step,
 * lowest index on ties; every inner product one ascending fma chain), r = #{|R_tt| >
 * tol |R_00|}, then the complete
 * orthogonal decomposition: T^T = (rows 0..r-1 of R)^T (l x r) = Z S, and
 * U = P Z S^{-T} Q_r^T.  Returns r.
 */
int32_t orc_nucleus_rect(const double* G, int32_t k, int32_t l, double tol, double* U) {
  double* A = (double*)malloc(sizeof(double) * (size_t)k * (size_t)l);     /* A[col*k + row] */
  double* taus = (double*)malloc(sizeof(double) * (size_t)k);
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)l);
  for (int32_t i = 0; i < k; ++i)
    for (int32_t j = 0; j < l; ++j) A[(int64_t)j * k + i] = G[(int64_t)i * l + j];
  for (int32_t j = 0; j < l; ++j) perm[j] = j;
  for (int32_t t = 0; t < k; ++t) {
    int32_t pj = t; double bn = -1.0;
    for (int32_t j = t; j < l; ++j) {
      double s = sqnorm(&A[(int64_t)j * k + t], k - t);
      if (s > bn) { bn = s; pj = j; }
    }
    if (pj != t) {
      for (int32_t i = 0; i < k; ++i) {
        double tmp = A[(int64_t)t * k + i]; A[(int64_t)t * k + i] = A[(int64_t)pj * k + i]; A[(int64_t)pj * k + i] = tmp;
      }
      int32_t tp = perm[t]; perm[t] = perm[pj]; perm[pj] = tp;
    }
    taus[t] = house(&A[(int64_t)t * k + t], k - t, 1);
    for (int32_t j = t + 1; j < l; ++j) apply_house(&A[(int64_t)t * k + t], 1, taus[t], &A[(int64_t)j * k + t], k - t, 1);
  }
  int32_t r = 0;
  double r00 = fabs(A[0]);
  if (r00 > 0.0)
    while (r < k && fabs(A[(int64_t)r * k + r]) > tol * r00) ++r;
  memset(U, 0, sizeof(double) * (size_t)l * (size_t)k);
  if (r == 0) { free(A); free(taus); free(perm); return 0; }
  double* Qt = (double*)calloc((size_t)k * (size_t)k, sizeof(double));      /* Q^T, column-major */
  for (int32_t i = 0; i < k; ++i) Qt[i * k + i] = 1.0;
  for (int32_t t = 0; t < k; ++t)
    for (int32_t j = 0; j < k; ++j) apply_house(&A[(int64_t)t * k + t], 1, taus[t], &Qt[j * k + t], k - t, 1);
  /* T^T (l x r, column-major: column c = row c of R over columns c..l-1) and its QR */
  double* Tt = (double*)calloc((size_t)l * (size_t)r, sizeof(double));
  double* tz = (double*)malloc(sizeof(double) * (size_t)r);
  for (int32_t c = 0; c < r; ++c)
    for (int32_t i = c; i < l; ++i) Tt[(int64_t)c * l + i] = A[(int64_t)i * k + c];
  for (int32_t c = 0; c < r; ++c) {
    tz[c] = house(&Tt[(int64_t)c * l + c], l - c, 1);
    for (int32_t j = c + 1; j < r; ++j) apply_house(&Tt[(int64_t)c * l + c], 1, tz[c], &Tt[(int64_t)j * l + c], l - c, 1);
  }
  /* X (l x k, column-major) = Z S^{-T} Q_r^T, one column at a time */
  double* X = (double*)calloc((size_t)l * (size_t)k, sizeof(double));
  for (int32_t col = 0; col < k; ++col) {
    double* v = &X[(int64_t)col * l];
    for (int32_t i = 0; i < r; ++i) {
      double s = Qt[col * k + i];
      for (int32_t p = 0; p < i; ++p) s = fma(-Tt[(int64_t)i * l + p], v[p], s);
      v[i] = s / Tt[(int64_t)i * l + i];
    }
    for (int32_t c = r - 1; c >= 0; --c) apply_house(&Tt[(int64_t)c * l + c], 1, tz[c], &v[c], l - c, 1);
  }
  for (int32_t i = 0; i < l; ++i)
    for (int32_t col = 0; col < k; ++col) U[(int64_t)perm[i] * k + col] = X[(int64_t)col * l + i];
  free(A); free(taus); free(perm); free(Qt); free(Tt); free(tz); free(X);
  return r;
}

/* ------------------------------------------------------------------ */
/* C-A iterations                                                      */
/* ------------------------------------------------------------------ */
/*
 * orc_ca_run: alpha C-A loops; each loop is a horizontal step (maxvol over the
 * columns of the k x n row strip W'[I,:] -> J) followed by a vertical step
 * (maxvol over the rows of the m x k column strip W'[:,J] -> I), as in the
 * Tests 2 schedule.  Loop 1 starts from the caller's rows I0 with a cold
 * column step; every later step is warm-started from the current set, so
 * |det W'[I,J]| never decreases.  The loop stops early when a whole loop made
 * no swap.  Outputs:
 *   I, J            final index sets (k each, in pivot-position order)
 *   C (m x k)       W'[:,J] row-major;  R (k x n) W[I,:] (original rows, the
 *                   back-transform of Algorithm alglratpsvd1 stage 4)
 *   U (k x k)       nucleus of G = W'[I,J] at relative tolerance rank_tol
 *   logvol[2*alpha] log|det W'[I,J]| after every step (unused slots NaN)
 *   info[4]         {rank, total swaps, loops run, status}
 * A strip holding NaN or Inf stops the run with status ORC_ERR_NONFINITE (the
 * outputs are then undefined).
 */
int orc_ca_run_warm(const orc_problem* p, int32_t k, int32_t sweeps, const int32_t* I0, const int32_t* J0,
                    double h, int32_t max_swaps, double rank_tol, int32_t* I, int32_t* J, double* C, double* U,
                    double* R, double* logvol, int32_t* info);
int orc_ca_run(const orc_problem* p, int32_t k, int32_t sweeps, const int32_t* I0, double h, int32_t max_swaps,
               double rank_tol, int32_t* I, int32_t* J, double* C, double* U, double* R, double* logvol,
               int32_t* info) {
  return orc_ca_run_warm(p, k, sweeps, I0, NULL, h, max_swaps, rank_tol, I, J, C, U, R, logvol, info);
}

/* orc_ca_run with the first column step warm-started at the columns J0 (k
 * distinct, or NULL for the cold start): resuming a run from its (I, J). */
int orc_ca_run_warm(const orc_problem* p, int32_t k, int32_t sweeps, const int32_t* I0, const int32_t* J0,
                    double h, int32_t max_swaps, double rank_tol, int32_t* I, int32_t* J, double* C, double* U,
                    double* R, double* logvol, int32_t* info) {
  int64_t m = p->m, n = orc_cols(p);          /* the strips are rows / columns of W' */
  double* Rs = (double*)malloc(sizeof(double) * (size_t)k * (size_t)n);
  double* Cs = (double*)malloc(sizeof(double) * (size_t)k * (size_t)m);
  double* G = (double*)malloc(sizeof(double) * (size_t)k * (size_t)k);
  int32_t* Jn = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  int32_t* In = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  int status = ORC_OK, total = 0, loops = 0;
  memcpy(I, I0, sizeof(int32_t) * (size_t)k);
  if (J0 != NULL) memcpy(J, J0, sizeof(int32_t) * (size_t)k);
  for (int32_t s = 0; s < 2 * sweeps; ++s) logvol[s] = NAN;
  for (int32_t s = 0; s < sweeps; ++s) {
    double ld; int32_t nsw1 = 0, nsw2 = 0;
    orc_gather_rows(p, I, k, Rs);
    if (!all_finite(Rs, (int64_t)k * n)) { status = ORC_ERR_NONFINITE; break; }
    int st = orc_maxvol(Rs, k, n, (s == 0 && J0 == NULL) ? NULL : J, h, max_swaps, Jn, NULL, &ld, &nsw1);
    if (st > status) status = st;
    memcpy(J, Jn, sizeof(int32_t) * (size_t)k);
    logvol[2 * s] = ld;
    orc_gather_cols_t(p, J, k, Cs);
    if (!all_finite(Cs, (int64_t)k * m)) { status = ORC_ERR_NONFINITE; break; }
    st = orc_maxvol(Cs, k, m, I, h, max_swaps, In, NULL, &ld, &nsw2);
    if (st > status) status = st;
    memcpy(I, In, sizeof(int32_t) * (size_t)k);
    logvol[2 * s + 1] = ld;
    total += nsw1 + nsw2;
    loops = s + 1;
    if (s > 0 && nsw1 == 0 && nsw2 == 0) break;
  }
  if (status == ORC_ERR_NONFINITE) {
    info[0] = 0; info[1] = total; info[2] = loops; info[3] = status;
    free(Rs); free(Cs); free(G); free(Jn); free(In);
    return status;
  }
  /* outputs: C = W'[:,J] (transpose of the last column strip, which used the final J) */
  for (int64_t i = 0; i < m; ++i)
    for (int32_t a = 0; a < k; ++a) C[i * k + a] = Cs[(int64_t)a * m + i];
  orc_gather_rows_orig(p, I, k, R);
  for (int32_t a = 0; a < k; ++a)
    for (int32_t b = 0; b < k; ++b) G[a * k + b] = C[(int64_t)I[a] * k + b];
  int32_t r = orc_nucleus(G, k, rank_tol, U);
  left_outputs(p, I, k, J, k, C, R);
  if (r < k && status == ORC_OK) status = ORC_WARN_RANK_DEFICIENT;
  info[0] = r; info[1] = total; info[2] = loops; info[3] = status;
  free(Rs); free(Cs); free(G); free(Jn); free(In);
  return status;
}

/*
 * orc_rhtcur: CUR LRA with Gaussian sampling (Algorithm algrhtcur), with
 * lbar = l = k (a square k x k generator):
 *  1. S = W Hbar (m x k) for the caller's n x k Gaussian Hbar (row-major),
 *     S[i][a] = sum over j ascending of fma(Hbar[j][a], w_ij, .) (the plain
 *     product; the input is W itself, no multiplier).
 *  2. The algorithms of GE96 on S: the k rows I of a k x k submatrix with
 *     locally maximal volume in S.  Taken as a one-loop C-A run on S^T
 *     (k x m) from all its k rows, whose cold first column step (LU with
 *     column pivoting, then dominance swaps while max |B^{-1} S^T| > h) picks
 *     k columns of S^T, i.e. rows of S.
 *  3. The same on W[I, :] (k x n): a one-loop C-A run from all k rows; its cold
 *     column step picks J, its row step puts the rows in generator order, and
 *     its nucleus is U = pinv of the rank-r QRP truncation of W[I, J].
 *  4. C = W[:, J] (m x k) and R = W[I, :] (k x n) in that order.
 * Outputs: I, J (k), C, U (k x k), R, logvol (2: the second run's), info:
 * rank, swaps (both runs), loops (2), status (an error of either run, else the
 * worse warning).
 */
int orc_rhtcur(const orc_problem* p, const double* Hbar, int32_t k, double h, int32_t max_swaps, double rank_tol,
               int32_t* I, int32_t* J, double* C, double* U, double* R, double* logvol, int32_t* info) {
  int64_t m = p->m, n = p->n;
  double* ST = (double*)malloc(sizeof(double) * (size_t)k * (size_t)m);
  for (int32_t a = 0; a < k; ++a)
    for (int64_t i = 0; i < m; ++i) {
      double acc = 0.0;
      for (int64_t j = 0; j < n; ++j) acc = fma(Hbar[j * k + a], entry_w(p, i, j), acc);
      ST[(int64_t)a * m + i] = acc;
    }
  int32_t* I0 = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  for (int32_t a = 0; a < k; ++a) I0[a] = a;
  orc_problem ps;
  memset(&ps, 0, sizeof(ps));
  ps.src = ORC_DENSE; ps.dtype = ORC_F64; ps.m = k; ps.n = m; ps.W = ST; ps.ldw = m; ps.mkind = ORC_MULT_NONE;
  int32_t* I1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  int32_t* J1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  double* C1 = (double*)malloc(sizeof(double) * (size_t)k * (size_t)k);
  double* U1 = (double*)malloc(sizeof(double) * (size_t)k * (size_t)k);
  double* R1 = (double*)malloc(sizeof(double) * (size_t)k * (size_t)m);
  double lv1[2];
  int32_t inf1[4], inf2[4];
  int st1 = orc_ca_run(&ps, k, 1, I0, h, max_swaps, rank_tol, I1, J1, C1, U1, R1, lv1, inf1);
  int status;
  if (st1 != ORC_OK && st1 < 16) {
    info[0] = 0; info[1] = inf1[1]; info[2] = 1; info[3] = st1;
    logvol[0] = logvol[1] = NAN;
    status = st1;
  } else {
    /* the k x n row strip W[I, :] as a dense problem of its own */
    double* R0 = (double*)malloc(sizeof(double) * (size_t)k * (size_t)n);
    orc_gather_rows_orig(p, J1, k, R0);
    orc_problem pr;
    memset(&pr, 0, sizeof(pr));
    pr.src = ORC_DENSE; pr.dtype = ORC_F64; pr.m = k; pr.n = n; pr.W = R0; pr.ldw = n; pr.mkind = ORC_MULT_NONE;
    int32_t* I2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
    double* C2 = (double*)malloc(sizeof(double) * (size_t)k * (size_t)k);
    int st2 = orc_ca_run(&pr, k, 1, I0, h, max_swaps, rank_tol, I2, J, C2, U, R, logvol, inf2);
    for (int32_t a = 0; a < k; ++a) I[a] = J1[I2[a]];
    if (st2 != ORC_OK && st2 < 16) status = st2;
    else status = st1 > st2 ? st1 : st2;
    if (!(st2 != ORC_OK && st2 < 16)) {
      double* Ct = (double*)malloc(sizeof(double) * (size_t)k * (size_t)m);
      orc_gather_cols_t(p, J, k, Ct);
      for (int64_t i = 0; i < m; ++i)
        for (int32_t a = 0; a < k; ++a) C[i * k + a] = Ct[(int64_t)a * m + i];
      free(Ct);
    }
    info[0] = inf2[0]; info[1] = inf1[1] + inf2[1]; info[2] = 2; info[3] = status;
    free(R0); free(I2); free(C2);
  }
  free(ST); free(I0); free(I1); free(J1); free(C1); free(U1); free(R1);
  return status;
}

/*
 * orc_ca_run_adaptive: C-A with the generator size fitted to the numerical
 * rank.  The paper's tests take r x r generators with r the numerical rank of
 * the input at 1e-6 (section "Numerical Experiments", Test Overview); here
 * that rank is found from the nucleus of the C-A run itself, in stages:
 *   sizes k_1 < k_2 < ... < k_S, each clipped to kmax = min(k_S, m, n);
 *   stage s: a complete C-A run (orc_ca_run) of size k_s from initial rows
 *     I_s, then the nucleus rank r_s at rank_tol;
 *   stop when r_s < k_s - margin (the core has spare room) or k_s = kmax;
 *   otherwise I_{s+1} = the stage's rows I, then the caller's initial rows
 *     I0[0 .. kmax-1] that are not in I, in their order, up to k_{s+1} rows.
 * I0 holds kmax distinct rows; I_1 = I0[0 .. k_1-1].
 * Outputs at the final size kf: I, J (kf), C (m x kf), U (kf x kf),
 * R (kf x n), logvol of the final stage; info[0] rank, info[1] swaps and
 * info[2] loops summed over the stages, info[3] the final stage's status,
 * info[4] kf, info[5] stages run.  Buffers are sized for kmax.
 */
int orc_ca_run_adaptive(const orc_problem* p, const int32_t* stages, int32_t nstages, int32_t margin,
                        int32_t sweeps, const int32_t* I0, double h, int32_t max_swaps, double rank_tol, int32_t* I,
                        int32_t* J, double* C, double* U, double* R, double* logvol, int32_t* info) {
  int64_t lim = p->m < p->n ? p->m : p->n;
  int32_t kmax = stages[nstages - 1];
  if (kmax > lim) kmax = (int32_t)lim;
  int32_t* Icur = (int32_t*)malloc(sizeof(int32_t) * (size_t)kmax);
  int32_t s = 0, k = stages[0] < kmax ? stages[0] : kmax;
  int32_t swaps = 0, loops = 0, nrun = 0, st = ORC_OK;
  int32_t inf[4];
  memcpy(Icur, I0, sizeof(int32_t) * (size_t)k);
  for (;;) {
    st = orc_ca_run(p, k, sweeps, Icur, h, max_swaps, rank_tol, I, J, C, U, R, logvol, inf);
    ++nrun;
    swaps += inf[1];
    loops += inf[2];
    if (st != ORC_OK && st < 16) break;
    if (k >= kmax || inf[0] < k - margin) break;
    /* next larger stage size */
    int32_t kn = k;
    while (s + 1 < nstages && kn <= k) {
      ++s;
      kn = stages[s] < kmax ? stages[s] : kmax;
    }
    if (kn <= k) break;
    memcpy(Icur, I, sizeof(int32_t) * (size_t)k);
    int32_t c = k;
    for (int32_t t = 0; t < kmax && c < kn; ++t) {
      int in = 0;
      for (int32_t a = 0; a < k; ++a) in |= (I[a] == I0[t]);
      if (!in) Icur[c++] = I0[t];
    }
    k = kn;
  }
  info[0] = inf[0]; info[1] = swaps; info[2] = loops; info[3] = st; info[4] = k; info[5] = nrun;
  free(Icur);
  return st;
}

/*
 * orc_cynical: the cynical CUR algorithms of the paper's tests (section
 * "Four algorithms used", Tests 3 and 4; section "CUR LRA; primitive, cynical,
 * and cross-approximation algorithms"): an r x r generator of locally maximal
 * volume inside a q x q sketch W'[K, L] (q = 4r in the paper).
 *   kind 0 (Tests 3): K and L are the caller's random index sets.
 *   kind 1 (Tests 4): L is the caller's random column set; a single C-A loop
 *     with q x q generators makes the sketch: K = the rows that maxvol
 *     (orc_maxvol, cold start) selects in the column strip W'[:, L], then
 *     L = the columns it selects in the row strip W'[K, :].
 * A C-A run (orc_ca_run, sweeps loops from the initial rows I0s: r distinct
 * indices in [0, q)) on the dense sketch S = W'[K, L] gives I', J' and the
 * nucleus of S[I', J'] = W'[I, J]; the generators are I = K[I'], J = L[J'],
 * with C = W'[:, J] (m x r), R = W[I, :] (r x n).
 * info: rank, swaps of every maxvol step, loops of the sketch C-A, status.
 * K and L (q each) are inputs and, for kind 1, receive the computed sets.
 */
int orc_cynical(const orc_problem* p, int32_t kind, int32_t r, int32_t q, int32_t* K, int32_t* L,
                const int32_t* I0s, int32_t sweeps, double h, int32_t max_swaps, double rank_tol, int32_t* I,
                int32_t* J, double* C, double* U, double* R, int32_t* info) {
  int64_t m = p->m, n = p->n;
  int status = ORC_OK, swaps = 0;
  info[0] = 0; info[1] = 0; info[2] = 0; info[3] = ORC_OK;
  if (kind == 1) {
    int32_t nsw = 0;
    double ld;
    double* Cs = (double*)malloc(sizeof(double) * (size_t)q * (size_t)m);
    orc_gather_cols_t(p, L, q, Cs);
    if (!all_finite(Cs, (int64_t)q * m)) status = ORC_ERR_NONFINITE;
    else {
      int st = orc_maxvol(Cs, q, m, NULL, h, max_swaps, K, NULL, &ld, &nsw);
      if (st > status) status = st;
      swaps += nsw;
    }
    free(Cs);
    if (status != ORC_ERR_NONFINITE) {
      double* Rs = (double*)malloc(sizeof(double) * (size_t)q * (size_t)n);
      orc_gather_rows(p, K, q, Rs);
      if (!all_finite(Rs, (int64_t)q * n)) status = ORC_ERR_NONFINITE;
      else {
        int st = orc_maxvol(Rs, q, n, NULL, h, max_swaps, L, NULL, &ld, &nsw);
        if (st > status) status = st;
        swaps += nsw;
      }
      free(Rs);
    }
    if (status == ORC_ERR_NONFINITE) {
      info[1] = swaps; info[3] = status;
      return status;
    }
  }
  /* the sketch as a dense problem of its own */
  double* S = (double*)malloc(sizeof(double) * (size_t)q * (size_t)q);
  for (int32_t a = 0; a < q; ++a)
    for (int32_t b = 0; b < q; ++b) S[(int64_t)a * q + b] = entry_wp(p, K[a], L[b]);
  orc_problem ps;
  memset(&ps, 0, sizeof(ps));
  ps.src = ORC_DENSE; ps.dtype = ORC_F64; ps.m = q; ps.n = q; ps.W = S; ps.ldw = q; ps.mkind = ORC_MULT_NONE;
  int32_t* Ii = (int32_t*)malloc(sizeof(int32_t) * (size_t)r);
  int32_t* Jj = (int32_t*)malloc(sizeof(int32_t) * (size_t)r);
  double* Cq = (double*)malloc(sizeof(double) * (size_t)q * (size_t)r);
  double* Rq = (double*)malloc(sizeof(double) * (size_t)r * (size_t)q);
  double* lv = (double*)malloc(sizeof(double) * 2 * (size_t)sweeps);
  int32_t inf[4];
  int st = orc_ca_run(&ps, r, sweeps, I0s, h, max_swaps, rank_tol, Ii, Jj, Cq, U, Rq, lv, inf);
  swaps += inf[1];
  if (st == ORC_ERR_NONFINITE || (st != ORC_OK && st < 16)) {
    status = st;
    info[1] = swaps; info[2] = inf[2]; info[3] = status;
  } else {
    if (st > status) status = st;
    for (int32_t a = 0; a < r; ++a) { I[a] = K[Ii[a]]; J[a] = L[Jj[a]]; }
    double* Ct = (double*)malloc(sizeof(double) * (size_t)r * (size_t)m);
    orc_gather_cols_t(p, J, r, Ct);
    for (int64_t i = 0; i < m; ++i)
      for (int32_t a = 0; a < r; ++a) C[i * r + a] = Ct[(int64_t)a * m + i];
    free(Ct);
    orc_gather_rows_orig(p, I, r, R);
    left_outputs(p, I, r, J, r, C, R);
    info[0] = inf[0]; info[1] = swaps; info[2] = inf[2]; info[3] = status;
  }
  free(S); free(Ii); free(Jj); free(Cq); free(Rq); free(lv);
  return status;
}

/*
 * Whitening update of X for one column entering (sign = +1) or leaving
 * (sign = -1) the generator C_g.  X = T W'[I, :] with T^T T = (C_g C_g^T)^{-1},
 * so s_q = ||X[:, q]||^2 = b_q^T (C_g C_g^T)^{-1} b_q for every column b_q.
 * With x = X[:, j] (copied first) and sigma = ||x||^2, Sherman-Morrison gives
 *   entering: T' = (I - g x x^T) T,  g = (1 - 1/sqrt(1 + sigma)) / sigma,
 *   leaving:  T' = (I + g x x^T) T,  g = (1/sqrt(1 - sigma) - 1) / sigma,
 * applied to every column q (inside the generator or not, j included):
 * t = x . X[:, q] (ascending fma chain), X[:, q] <- fma(-+g t, x, X[:, q]),
 * and s_q is recomputed (ascending fma chain).  sigma = 0 changes nothing.
 */
static void ov_whiten(double* X, double* s, double* x, int32_t k, int64_t n, int64_t j, int sign) {
  double sigma = s[j];
  if (sigma == 0.0) return;
  double g = (sign > 0) ? (1.0 - 1.0 / sqrt(1.0 + sigma)) / sigma : (1.0 / sqrt(1.0 - sigma) - 1.0) / sigma;
  double gs = (sign > 0) ? -g : g;
  for (int32_t i = 0; i < k; ++i) x[i] = X[(int64_t)i * n + j];
  for (int64_t q = 0; q < n; ++q) {
    double t = 0.0;
    for (int32_t i = 0; i < k; ++i) t = fma(x[i], X[(int64_t)i * n + q], t);
    double c = gs * t;
    double v = 0.0;
    for (int32_t i = 0; i < k; ++i) {
      X[(int64_t)i * n + q] = fma(c, x[i], X[(int64_t)i * n + q]);
      v = fma(X[(int64_t)i * n + q], X[(int64_t)i * n + q], v);
    }
    s[q] = v;
  }
}

/* Greedy expansion by up to p columns (Algorithm algrup): the column outside
 * the generator with the largest s_j (lowest j on ties) joins it, appended to
 * Jo; none joins once the largest s_j is 0.  rho is multiplied by 1 + s_j
 * (Theorem th2: the squared volume grows by that factor).  Returns the number
 * added. */
static int32_t ov_expand(double* X, double* s, double* x, unsigned char* in, int32_t* Jo, int32_t* l, int32_t k,
                         int64_t n, int32_t p, double* rho) {
  int32_t added = 0;
  for (int32_t g = 0; g < p; ++g) {
    int64_t js = -1;
    for (int64_t j = 0; j < n; ++j)
      if (!in[j] && (js < 0 || s[j] > s[js])) js = j;
    if (js < 0 || !(s[js] > 0.0)) break;
    *rho = *rho * (1.0 + s[js]);
    in[js] = 1;
    Jo[(*l)++] = (int32_t)js;
    ov_whiten(X, s, x, k, n, js, +1);
    ++added;
  }
  return added;
}

/* Greedy contraction by p columns (the reverse of Algorithm algrup): the
 * column inside the generator with the smallest s_j (lowest j on ties) leaves
 * it; Jo keeps the order of the columns that stay.  rho is multiplied by
 * 1 - s_j (Theorem th2: the squared volume shrinks by that factor).  Returns 0,
 * or -1 if the smallest s_j is not below 1 (the generator would lose rank). */
static int ov_contract(double* X, double* s, double* x, unsigned char* in, int32_t* Jo, int32_t* l, int32_t k,
                       int64_t n, int32_t p, double* rho) {
  for (int32_t g = 0; g < p; ++g) {
    int64_t jr = -1;
    for (int64_t j = 0; j < n; ++j)
      if (in[j] && !isnan(s[j]) && (jr < 0 || s[j] < s[jr])) jr = j;
    if (jr < 0 || !(s[jr] < 1.0)) return -1;
    *rho = *rho * (1.0 - s[jr]);
    int32_t a = 0;
    while (Jo[a] != (int32_t)jr) ++a;
    for (; a + 1 < *l; ++a) Jo[a] = Jo[a + 1];
    --(*l);
    in[jr] = 0;
    ov_whiten(X, s, x, k, n, jr, -1);
  }
  return 0;
}

/*
 * orc_oversample_cycle: a rectangular k x l generator (l = k + p) from the
 * rows I and columns J of a square one.
 *  1. X = B^{-1} W'[I, :], B = W'[I, J]: the C matrix of a maxvol step
 *     (orc_maxvol) on the row strip warm-started at J with no swaps; its
 *     columns J are exact unit vectors, and its selected set J0 (J unless the
 *     warm LU met a zero pivot) starts J'.  A rank-deficient strip (zero
 *     pivot) keeps J' = J; nothing is added and no cycle runs.
 *  2. Algorithm algrup: pextra greedy expansions (ov_expand), each adding the
 *     column that increases the volume of the generator C_g (sqrt det C_g C_g^T)
 *     the most; Theorem th3 bounds the CUR error of such generators.
 *  3. Section scrsorth's expansion/contraction cycles, when pmax > 0.  The
 *     generator is accepted as locally h-maximal when 1 + max s_q over the
 *     columns q outside it is at most h (Corollary colclmx with b^2 = max s_q).
 *     Otherwise a p-cycle expands by p columns and contracts back by p
 *     (ov_contract).  It is kept when it changed the set and its volume factor
 *     rho (the product of the 1 + s and 1 - s factors) is above 1, and p
 *     restarts at 1.  Otherwise X, s and J' are restored and p grows by one.
 *     The loop ends when the test passes (status unchanged), or when p passes
 *     pmax or max_cycles cycles were kept (status ORC_WARN_NOT_CONVERGED).
 *  4. U = orc_nucleus_rect of W'[I, J'] (k x l), C = W'[:, J'] (m x l), R =
 *     W[I, :] (k x n).
 * C (m x (k+pextra)) and U ((k+pextra) x k) are sized for l = k + pextra; J'
 * needs k + pextra + pmax entries (a cycle grows it by p before contracting).
 * info: rank, l (used), status (worst of the maxvol step, the cycles and the
 * nucleus), cycles kept, the largest p tried.
 */
int orc_oversample_cycle(const orc_problem* p, const int32_t* I, const int32_t* J, int32_t k, int32_t pextra,
                         int32_t pmax, int32_t max_cycles, double h, double rank_tol, int32_t* Jo, double* C,
                         double* U, double* R, int32_t* info) {
  int64_t m = p->m, n = p->n;
  int32_t l = k, cycles = 0, ptried = 0;
  double* X = (double*)malloc(sizeof(double) * (size_t)k * (size_t)n);
  double* Rs = (double*)malloc(sizeof(double) * (size_t)k * (size_t)n);
  orc_gather_rows(p, I, k, Rs);
  if (!all_finite(Rs, (int64_t)k * n)) {
    info[0] = 0; info[1] = k; info[2] = ORC_ERR_NONFINITE; info[3] = 0; info[4] = 0;
    free(X); free(Rs);
    return ORC_ERR_NONFINITE;
  }
  double ld;
  int32_t nsw = 0;
  int status = orc_maxvol(Rs, k, n, J, h, 0, Jo, X, &ld, &nsw);
  if (status == ORC_WARN_NOT_CONVERGED) status = ORC_OK;        /* no swaps wanted here */
  if (status == ORC_WARN_RANK_DEFICIENT) memcpy(Jo, J, sizeof(int32_t) * (size_t)k);   /* no expansion */
  unsigned char* in = (unsigned char*)calloc((size_t)n, 1);
  double* s = (double*)malloc(sizeof(double) * (size_t)n);
  double* x = (double*)malloc(sizeof(double) * (size_t)k);
  for (int32_t a = 0; a < k; ++a) in[Jo[a]] = 1;
  if (status != ORC_WARN_RANK_DEFICIENT) {
    for (int64_t j = 0; j < n; ++j) {
      double v = 0.0;
      for (int32_t i = 0; i < k; ++i) v = fma(X[(int64_t)i * n + j], X[(int64_t)i * n + j], v);
      s[j] = v;
    }
    double rho = 1.0;
    ov_expand(X, s, x, in, Jo, &l, k, n, pextra, &rho);
    if (pmax > 0) {
      int32_t ltarget = l;
      double* Xb = (double*)malloc(sizeof(double) * (size_t)k * (size_t)n);
      double* sb = (double*)malloc(sizeof(double) * (size_t)n);
      int32_t* Jb = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ltarget + pmax));
      int converged = 0;
      int32_t pc = 1;
      for (;;) {
        double smax = 0.0;
        for (int64_t q = 0; q < n; ++q)
          if (!in[q] && s[q] > smax) smax = s[q];
        if (1.0 + smax <= h) { converged = 1; break; }
        if (pc > pmax || cycles >= max_cycles) break;
        if (pc > ptried) ptried = pc;
        memcpy(Xb, X, sizeof(double) * (size_t)k * (size_t)n);
        memcpy(sb, s, sizeof(double) * (size_t)n);
        memcpy(Jb, Jo, sizeof(int32_t) * (size_t)ltarget);
        rho = 1.0;
        int32_t added = ov_expand(X, s, x, in, Jo, &l, k, n, pc, &rho);
        int ok = (added > 0) && ov_contract(X, s, x, in, Jo, &l, k, n, added, &rho) == 0;
        int changed = 0;
        if (ok) {
          /* the same set iff every kept column was in the old set */
          for (int32_t a = 0; a < l && !changed; ++a) {
            int found = 0;
            for (int32_t b = 0; b < ltarget; ++b) if (Jb[b] == Jo[a]) { found = 1; break; }
            if (!found) changed = 1;
          }
        }
        if (ok && changed && rho > 1.0) {
          ++cycles;
          pc = 1;
        } else {
          for (int32_t a = 0; a < l; ++a) in[Jo[a]] = 0;
          memcpy(X, Xb, sizeof(double) * (size_t)k * (size_t)n);
          memcpy(s, sb, sizeof(double) * (size_t)n);
          memcpy(Jo, Jb, sizeof(int32_t) * (size_t)ltarget);
          l = ltarget;
          for (int32_t a = 0; a < l; ++a) in[Jo[a]] = 1;
          ++pc;
        }
      }
      if (!converged && status == ORC_OK) status = ORC_WARN_NOT_CONVERGED;
      free(Xb); free(sb); free(Jb);
    }
  }
  /* outputs at l */
  double* Ct = (double*)malloc(sizeof(double) * (size_t)l * (size_t)m);
  orc_gather_cols_t(p, Jo, l, Ct);
  for (int64_t i = 0; i < m; ++i)
    for (int32_t a = 0; a < l; ++a) C[i * l + a] = Ct[(int64_t)a * m + i];
  orc_gather_rows_orig(p, I, k, R);
  double* G = (double*)malloc(sizeof(double) * (size_t)k * (size_t)l);
  for (int32_t a = 0; a < k; ++a)
    for (int32_t b = 0; b < l; ++b) G[(int64_t)a * l + b] = C[(int64_t)I[a] * l + b];
  int32_t r = orc_nucleus_rect(G, k, l, rank_tol, U);
  left_outputs(p, I, k, Jo, l, C, R);
  if (r < k && status == ORC_OK) status = ORC_WARN_RANK_DEFICIENT;
  info[0] = r; info[1] = l; info[2] = status; info[3] = cycles; info[4] = ptried;
  free(X); free(Rs); free(in); free(s); free(x); free(Ct); free(G);
  return status;
}

/* orc_oversample: orc_oversample_cycle without cycles (pmax = 0); info: rank,
 * l (used), status. */
int orc_oversample(const orc_problem* p, const int32_t* I, const int32_t* J, int32_t k, int32_t pextra,
                   double h, double rank_tol, int32_t* Jo, double* C, double* U, double* R, int32_t* info) {
  int32_t inf[5];
  int st = orc_oversample_cycle(p, I, J, k, pextra, 0, 0, h, rank_tol, Jo, C, U, R, inf);
  info[0] = inf[0]; info[1] = inf[1]; info[2] = inf[2];
  return st;
}

/* ------------------------------------------------------------------ */
/* r-projective volume: Algorithm alg1tor, then Algorithm algprjvlm     */
/* ------------------------------------------------------------------ */

/*
 * orc_alg1tor: Algorithm alg1tor (a column set grown one greedy column at a
 * time, starting from the column of largest norm) on the k x n matrix A
 * (row-major, overwritten), stopped at the numerical rank.  At step g = 0, 1, ...:
 *   1. the pivot j_g is the column outside the chosen set whose subvector of
 *      rows g..k-1 has the largest squared norm s_j (an ascending fma chain,
 *      recomputed from the current A), lowest j on ties.  The loop stops before
 *      step g when g = min(k, n), when that largest s_j is 0, or, for g > 0,
 *      when sqrt(s_{j_g}) <= tol * sqrt(s_{j_0}); the numerical rank is r = g;
 *   2. a Householder reflection on rows g..k-1 maps x = A[g.., j_g] to
 *      alpha e_1 with alpha = -sqrt(s) for x_0 >= 0 and +sqrt(s) otherwise:
 *      v = x - alpha e_1 and tau = 1 / (sqrt(s) (sqrt(s) + |x_0|)), which is
 *      2 / v^T v.  Column j_g becomes (alpha, 0, ..., 0) exactly.  Every other
 *      column c outside the chosen set gets t = v . A[g.., c] (ascending fma
 *      chain) and A[g + i][c] <- fma(-(tau t), v_i, A[g + i][c]).  The chosen
 *      columns are zero below their own row and stay unchanged.
 * This is Householder QR with column pivoting (Businger-Golub).  The leading r
 * rows of the result are R' of the rank-revealing factorisation A = Q R P in
 * stage 1 of Algorithm algprjvlm, with the columns in their original order;
 * R'[:, J0] is upper triangular in pivot order, J0 = (j_0, ..., j_{r-1}).
 * Returns r.
 */
int32_t orc_alg1tor(double* A, int32_t k, int64_t n, double tol, int32_t* J0) {
  unsigned char* chosen = (unsigned char*)calloc((size_t)n, 1);
  double* v = (double*)malloc(sizeof(double) * (size_t)k);
  int32_t g = 0;
  double thr = 0.0;
  int64_t gmax = (n < k) ? n : k;
  for (; g < gmax; ++g) {
    int64_t js = -1;
    double sbest = 0.0;
    for (int64_t c = 0; c < n; ++c) {
      if (chosen[c]) continue;
      double sc = 0.0;
      for (int32_t i = g; i < k; ++i) sc = fma(A[(int64_t)i * n + c], A[(int64_t)i * n + c], sc);
      if (js < 0 || sc > sbest) { js = c; sbest = sc; }
    }
    if (js < 0 || !(sbest > 0.0)) break;
    double nrm = sqrt(sbest);
    if (g == 0) thr = tol * nrm;
    else if (!(nrm > thr)) break;
    double x0 = A[(int64_t)g * n + js];
    double alpha = (x0 >= 0.0) ? -nrm : nrm;
    double tau = 1.0 / (nrm * (nrm + fabs(x0)));
    v[0] = x0 - alpha;
    for (int32_t i = 1; i < k - g; ++i) v[i] = A[(int64_t)(g + i) * n + js];
    chosen[js] = 1;
    J0[g] = (int32_t)js;
    for (int64_t c = 0; c < n; ++c) {
      if (chosen[c]) continue;
      double t = 0.0;
      for (int32_t i = 0; i < k - g; ++i) t = fma(v[i], A[(int64_t)(g + i) * n + c], t);
      double cc = tau * t;
      for (int32_t i = 0; i < k - g; ++i) A[(int64_t)(g + i) * n + c] = fma(-cc, v[i], A[(int64_t)(g + i) * n + c]);
    }
    A[(int64_t)g * n + js] = alpha;
    for (int32_t i = g + 1; i < k; ++i) A[(int64_t)i * n + js] = 0.0;
  }
  free(chosen); free(v);
  return g;
}

/*
 * orc_prjvol: a k x l generator of maximal r-projective volume in the row
 * strip A = W'[I, :] of a square generator's rows I (k = |I|),
 * l = min(k + pextra, n) (Algorithm algprjvlm; Lemma leprwnmp maps the volumes
 * of R' back to r-projective volumes in A):
 *  1. stage 1: orc_alg1tor on A at rank_tol gives the numerical rank r, R'
 *     (the first r rows, r x n) and J0;
 *  2. stage 2's black box for a submatrix of maximal volume in the full-rank
 *     R': the dominance swaps of Algorithm algdomin (orc_maxvol on R'
 *     warm-started at J0, threshold h, at most max_swaps swaps; R'[:, J0] is
 *     upper triangular, so the warm LU is R'[:, J0] itself), then Algorithm
 *     algrup's greedy expansions (ov_expand on X = B^{-1} R') up to l columns;
 *  3. outputs W'[:, J'] and the nucleus as orc_oversample_cycle's: C =
 *     W'[:, J'] (m x l), U = orc_nucleus_rect(W'[I, J'], k, l, rank_tol),
 *     R = W[I, :] (k x n).
 * A zero strip (r = 0) keeps J' = J and l = k.  C (m x (k + pextra)) and U
 * ((k + pextra) x k) are sized for l = k + pextra.  info: nucleus rank, l,
 * status (worst of the swaps and the nucleus: ORC_WARN_NOT_CONVERGED when
 * max_swaps stopped the swaps, ORC_WARN_RANK_DEFICIENT when the nucleus rank
 * is below k or r = 0), swaps, r.
 */
int orc_prjvol(const orc_problem* p, const int32_t* I, const int32_t* J, int32_t k, int32_t pextra, double h,
               int32_t max_swaps, double rank_tol, int32_t* Jo, double* C, double* U, double* R, int32_t* info) {
  int64_t m = p->m, n = p->n;
  int32_t lt = (k + pextra < n) ? k + pextra : (int32_t)n;
  double* A = (double*)malloc(sizeof(double) * (size_t)k * (size_t)n);
  orc_gather_rows(p, I, k, A);
  if (!all_finite(A, (int64_t)k * n)) {
    info[0] = 0; info[1] = k; info[2] = ORC_ERR_NONFINITE; info[3] = 0; info[4] = 0;
    free(A);
    return ORC_ERR_NONFINITE;
  }
  int32_t* J0 = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  int32_t r = orc_alg1tor(A, k, n, rank_tol, J0);
  int status = ORC_OK;
  int32_t l = k, nsw = 0;
  if (r == 0) {
    memcpy(Jo, J, sizeof(int32_t) * (size_t)k);
    status = ORC_WARN_RANK_DEFICIENT;
  } else {
    double* X = (double*)malloc(sizeof(double) * (size_t)r * (size_t)n);
    double* s = (double*)malloc(sizeof(double) * (size_t)n);
    double* x = (double*)malloc(sizeof(double) * (size_t)r);
    unsigned char* in = (unsigned char*)calloc((size_t)n, 1);
    double ld;
    /* A's first r rows are R' (row-major, leading dimension n) */
    status = orc_maxvol(A, r, n, J0, h, max_swaps, Jo, X, &ld, &nsw);
    l = r;
    for (int32_t a = 0; a < r; ++a) in[Jo[a]] = 1;
    for (int64_t j = 0; j < n; ++j) {
      double v = 0.0;
      for (int32_t i = 0; i < r; ++i) v = fma(X[(int64_t)i * n + j], X[(int64_t)i * n + j], v);
      s[j] = v;
    }
    double rho = 1.0;
    ov_expand(X, s, x, in, Jo, &l, r, n, lt - r, &rho);
    free(X); free(s); free(x); free(in);
  }
  double* Ct = (double*)malloc(sizeof(double) * (size_t)l * (size_t)m);
  orc_gather_cols_t(p, Jo, l, Ct);
  for (int64_t i = 0; i < m; ++i)
    for (int32_t a = 0; a < l; ++a) C[i * l + a] = Ct[(int64_t)a * m + i];
  orc_gather_rows_orig(p, I, k, R);
  double* G = (double*)malloc(sizeof(double) * (size_t)k * (size_t)l);
  for (int32_t a = 0; a < k; ++a)
    for (int32_t b = 0; b < l; ++b) G[(int64_t)a * l + b] = C[(int64_t)I[a] * l + b];
  int32_t rk = orc_nucleus_rect(G, k, l, rank_tol, U);
  left_outputs(p, I, k, Jo, l, C, R);
  if (rk < k && status == ORC_OK) status = ORC_WARN_RANK_DEFICIENT;
  info[0] = rk; info[1] = l; info[2] = status; info[3] = nsw; info[4] = r;
  free(A); free(J0); free(Ct); free(G);
  return status;
}

/* ------------------------------------------------------------------ */
/* Leverage-score sampling inside C-A (DMM08 Algorithm 1 on sketches)   */
/* ------------------------------------------------------------------ */
#define ORC_JAC_SWEEPS 10
#define ORC_LEV_EIG_TOL 1e-12

/* Pair i of round t of the round-robin (circle) schedule over kp (even)
 * indices: index 0 meets 1 + t, and 1 + ((t + i) mod (kp - 1)) meets
 * 1 + ((t - i) mod (kp - 1)); every pair meets once in kp - 1 rounds. */
static void jac_pair(int32_t kp, int32_t t, int32_t i, int32_t* p, int32_t* q) {
  int32_t a = (i == 0) ? 0 : 1 + (t + i) % (kp - 1);
  int32_t b = 1 + (t + kp - 1 - i) % (kp - 1);
  *p = a < b ? a : b;
  *q = a < b ? b : a;
}

/*
 * orc_jacobi_eig: eigen-decomposition of a symmetric k x k G (row-major, in
 * place) by at most ORC_JAC_SWEEPS sweeps of Jacobi rotations in the round-robin
 * order (k rounded up to even kp; pairs with an index >= k are skipped).  In
 * each round every rotation is computed from G as it stands at the round's
 * start (the pairs are disjoint): for G[p][q] != 0, tau = (G[q][q] -
 * G[p][p]) / (2 G[p][q]), t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
 * c = 1 / sqrt(1 + t^2), s = t c (the classical symmetric Schur rotation that
 * zeroes G[p][q]); then all row pairs (row p <- c row_p - s row_q, row q <-
 * s row_p + c row_q), then all column pairs the same way, then the columns of
 * Q (Q starts as I).  After each sweep the iteration stops when the largest
 * |G[p][q]|, p < q, is at most 2^-48 times the largest |G[p][p]| (a maximum of
 * absolute values, the same in any order of evaluation).  On return G is
 * diagonal to rounding and G_in = Q G Q^T.
 */
void orc_jacobi_eig(double* G, double* Q, int32_t k) {
  int32_t kp = k + (k & 1);
  int32_t half = kp / 2;
  double* cs = (double*)malloc(sizeof(double) * 2 * (size_t)(half > 0 ? half : 1));
  for (int32_t i = 0; i < k; ++i)
    for (int32_t j = 0; j < k; ++j) Q[i * k + j] = (i == j) ? 1.0 : 0.0;
  for (int32_t sw = 0; sw < ORC_JAC_SWEEPS; ++sw) {
    for (int32_t t = 0; t < kp - 1; ++t) {
      for (int32_t i = 0; i < half; ++i) {
        int32_t p, q;
        jac_pair(kp, t, i, &p, &q);
        double c = 1.0, sn = 0.0;
        if (q < k && G[p * k + q] != 0.0) {
          double tau = (G[q * k + q] - G[p * k + p]) / (2.0 * G[p * k + q]);
          double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + tt * tt);
          sn = tt * c;
        }
        cs[2 * i] = c; cs[2 * i + 1] = sn;
      }
      for (int32_t i = 0; i < half; ++i) {
        int32_t p, q;
        jac_pair(kp, t, i, &p, &q);
        if (q >= k) continue;
        double c = cs[2 * i], sn = cs[2 * i + 1];
        for (int32_t j = 0; j < k; ++j) {
          double x = G[p * k + j], y = G[q * k + j];
          G[p * k + j] = c * x - sn * y;
          G[q * k + j] = sn * x + c * y;
        }
      }
      for (int32_t i = 0; i < half; ++i) {
        int32_t p, q;
        jac_pair(kp, t, i, &p, &q);
        if (q >= k) continue;
        double c = cs[2 * i], sn = cs[2 * i + 1];
        for (int32_t j = 0; j < k; ++j) {
          double x = G[j * k + p], y = G[j * k + q];
          G[j * k + p] = c * x - sn * y;
          G[j * k + q] = sn * x + c * y;
        }
        for (int32_t j = 0; j < k; ++j) {
          double x = Q[j * k + p], y = Q[j * k + q];
          Q[j * k + p] = c * x - sn * y;
          Q[j * k + q] = sn * x + c * y;
        }
      }
    }
    double off = 0.0, dmax = 0.0;
    for (int32_t p = 0; p < k; ++p) {
      if (fabs(G[p * k + p]) > dmax) dmax = fabs(G[p * k + p]);
      for (int32_t q = p + 1; q < k; ++q)
        if (fabs(G[p * k + q]) > off) off = fabs(G[p * k + q]);
    }
    if (off <= ldexp(1.0, -48) * dmax) break;
  }
  free(cs);
}

/*
 * orc_lev_scores: SVD-based leverage scores (eq. eqlevsc with beta = 1) of the
 * columns of a k x n sketch A (row-major): v_j = ||row j of V^(r)||^2, with
 * V^(r) the top-r right singular vectors of A, from the Gram matrix:
 *  1. G = A A^T, G[a][b] = ascending fma chain over j, for a <= b, mirrored;
 *  2. orc_jacobi_eig(G) -> eigenvalues d_a = G[a][a], eigenvectors Q[:, a];
 *  3. the r largest eigenvalues (largest first, lowest index on ties) that are
 *     >= ORC_LEV_EIG_TOL times the largest and positive (sigma >= 1e-6 sigma_max);
 *  4. v_j = sum over them, in that order, of w / d_t with w = e^2, e the
 *     ascending fma chain of Q[:, t] . A[:, j] (v_j = (a_j . u_t)^2 / sigma_t^2).
 * The scores p_j = v_j / sum v are the sampling probabilities.  Returns the
 * number of eigenpairs used (0 when A has no positive eigenvalue).
 */
int32_t orc_lev_scores(const double* A, int32_t k, int64_t n, int32_t r, double* v) {
  double* G = (double*)malloc(sizeof(double) * (size_t)k * (size_t)k);
  double* Q = (double*)malloc(sizeof(double) * (size_t)k * (size_t)k);
  int32_t* sel = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  unsigned char* used = (unsigned char*)calloc((size_t)k, 1);
  for (int32_t a = 0; a < k; ++a)
    for (int32_t b = a; b < k; ++b) {
      double acc = 0.0;
      for (int64_t j = 0; j < n; ++j) acc = fma(A[(int64_t)a * n + j], A[(int64_t)b * n + j], acc);
      G[a * k + b] = acc;
      G[b * k + a] = acc;
    }
  orc_jacobi_eig(G, Q, k);
  int32_t re = 0;
  double dmax = 0.0;
  for (int32_t t = 0; t < r && t < k; ++t) {
    int32_t best = -1;
    for (int32_t a = 0; a < k; ++a)
      if (!used[a] && (best < 0 || G[a * k + a] > G[best * k + best])) best = a;
    if (best < 0 || !(G[best * k + best] > 0.0)) break;
    if (t == 0) dmax = G[best * k + best];
    else if (G[best * k + best] < ORC_LEV_EIG_TOL * dmax) break;
    used[best] = 1;
    sel[re++] = best;
  }
  for (int64_t j = 0; j < n; ++j) {
    double acc = 0.0;
    for (int32_t t = 0; t < re; ++t) {
      int32_t c = sel[t];
      double e = 0.0;
      for (int32_t a = 0; a < k; ++a) e = fma(Q[a * k + c], A[(int64_t)a * n + j], e);
      double w = e * e;
      acc = acc + w / G[c * k + c];
    }
    v[j] = acc;
  }
  free(G); free(Q); free(sel); free(used);
  return re;
}

/*
 * orc_lev_sample: DMM08's sampling of l indices out of n by the scores v
 * (probabilities p_j = v_j / total, total = the ascending sum of v):
 *  kind 0, Exactly(l) (Algorithm algsmplex): for t = 0..l-1 the smallest j with
 *    cum_j > u_t * total (cum_j the ascending running sum of v; if none, the
 *    last j with v_j > 0): l indices in draw order, repeats allowed;
 *  kind 1, Expected(l) (Algorithm algsmplexp): j ascending is picked when u_j <
 *    min(1, (l v_j) / total), at most l picks.
 * u: l (kind 0) or n (kind 1) uniform draws in [0, 1).  With total <= 0 (no
 * scores) the first min(l, n) indices are taken.  A kind-1 scan that picks
 * nothing takes the index of the largest v_j (lowest on ties).  Returns the
 * number of indices written to out.
 */
int32_t orc_lev_sample(const double* v, int64_t n, int32_t l, int32_t kind, const double* u, int32_t* out) {
  double* cum = (double*)malloc(sizeof(double) * (size_t)n);
  double c = 0.0;
  int64_t last = -1;
  for (int64_t j = 0; j < n; ++j) {
    c = c + v[j];
    cum[j] = c;
    if (v[j] > 0.0) last = j;
  }
  double total = c;
  int32_t cnt = 0;
  if (!(total > 0.0) || last < 0) {
    for (int64_t j = 0; j < n && cnt < l; ++j) out[cnt++] = (int32_t)j;
  } else if (kind == 0) {
    for (int32_t t = 0; t < l; ++t) {
      double target = u[t] * total;
      int64_t lo = 0, hi = n;                 /* smallest j with cum[j] > target */
      while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (cum[mid] > target) hi = mid; else lo = mid + 1;
      }
      out[cnt++] = (int32_t)(lo < n ? lo : last);
    }
  } else {
    for (int64_t j = 0; j < n && cnt < l; ++j) {
      double pr = ((double)l * v[j]) / total;
      if (pr > 1.0) pr = 1.0;
      if (u[j] < pr) out[cnt++] = (int32_t)j;
    }
    if (cnt == 0) {
      int64_t best = 0;
      for (int64_t j = 1; j < n; ++j) if (v[j] > v[best]) best = j;
      out[cnt++] = (int32_t)best;
    }
  }
  free(cum);
  return cnt;
}

/*
 * orc_ca_lev: C-A iterations whose steps select by DMM08 Algorithm 1 on the
 * sketches (the C-A lines of the tables "LRA errors of Cross-Approximation
 * tests incorporating [DMM08, Algorithm 1]"): from the rows I0 (k of them),
 * iters times
 *   horizontal step: the scores of the columns of W'[I, :] (kI x n, rank r) ->
 *     orc_lev_sample(l = k) with the draws u_{2s} -> J (kJ indices);
 *   vertical step: the scores of the rows, i.e. of the columns of W'[:, J]^T
 *     (kJ x m) -> orc_lev_sample with u_{2s+1} -> I (kI indices);
 * then U = pinv of the rank-r QRP truncation of G = W'[I, J] (kI x kJ; the
 * rectangular nucleus, of G^T when kI > kJ, transposed back), C = W'[:, J]
 * (m x kJ), R = W[I, :] (kI x n).  Repeated indices (Exactly) stay in the sets.
 * kind: bit 0 selects the sampling (0 Exactly, 1 Expected); bit 1 replaces the
 * SVD-based scores by uniform ones (lev_uniform), so kind 2 and 3 sample with
 * probabilities 1/n.
 * draws: 2 iters steps of max(m, n) uniforms each.  Outputs sized for k.
 * info: rank, kI, kJ, status (ORC_WARN_RANK_DEFICIENT when a sketch had no
 * positive eigenvalue or the nucleus rank is below min(kI, kJ)).
 */
/* Uniform scores v_j = 1 (probabilities 1/n): the leverage scores of a perturbed
 * factor-Gaussian input with r << n are nearly equal (the chi-square argument of
 * the section on superfast leverage scores, Lemma lmchitail and its corollary),
 * so the SVD stage is skipped. */
static void lev_uniform(double* v, int64_t n) {
  for (int64_t j = 0; j < n; ++j) v[j] = 1.0;
}

int orc_ca_lev(const orc_problem* p, int32_t k, int32_t r, int32_t iters, int32_t kind, const double* draws,
               const int32_t* I0, double rank_tol, int32_t* I, int32_t* J, double* C, double* U, double* R,
               int32_t* info) {
  int64_t m = p->m, n = p->n, L = m > n ? m : n;
  double* S = (double*)malloc(sizeof(double) * (size_t)k * (size_t)L);
  double* v = (double*)malloc(sizeof(double) * (size_t)L);
  int32_t kI = k, kJ = 0;
  int status = ORC_OK;
  memcpy(I, I0, sizeof(int32_t) * (size_t)k);
  for (int32_t it = 0; it < iters; ++it) {
    orc_gather_rows(p, I, kI, S);
    if (!all_finite(S, (int64_t)kI * n)) { status = ORC_ERR_NONFINITE; break; }
    if (kind & 2) lev_uniform(v, n);
    else if (orc_lev_scores(S, kI, n, r < kI ? r : kI, v) == 0) status = ORC_WARN_RANK_DEFICIENT;
    kJ = orc_lev_sample(v, n, k, kind & 1, draws + (size_t)(2 * it) * L, J);
    orc_gather_cols_t(p, J, kJ, S);
    if (!all_finite(S, (int64_t)kJ * m)) { status = ORC_ERR_NONFINITE; break; }
    if (kind & 2) lev_uniform(v, m);
    else if (orc_lev_scores(S, kJ, m, r < kJ ? r : kJ, v) == 0) status = ORC_WARN_RANK_DEFICIENT;
    kI = orc_lev_sample(v, m, k, kind & 1, draws + (size_t)(2 * it + 1) * L, I);
  }
  if (status == ORC_ERR_NONFINITE) {
    info[0] = 0; info[1] = kI; info[2] = kJ; info[3] = status;
    free(S); free(v);
    return status;
  }
  double* Ct = (double*)malloc(sizeof(double) * (size_t)kJ * (size_t)m);
  orc_gather_cols_t(p, J, kJ, Ct);
  for (int64_t i = 0; i < m; ++i)
    for (int32_t a = 0; a < kJ; ++a) C[i * kJ + a] = Ct[(int64_t)a * m + i];
  orc_gather_rows_orig(p, I, kI, R);
  double* G = (double*)malloc(sizeof(double) * (size_t)kI * (size_t)kJ);
  int32_t rank;
  if (kI <= kJ) {
    for (int32_t a = 0; a < kI; ++a)
      for (int32_t b = 0; b < kJ; ++b) G[(int64_t)a * kJ + b] = C[(int64_t)I[a] * kJ + b];
    rank = orc_nucleus_rect(G, kI, kJ, rank_tol, U);               /* kJ x kI */
  } else {
    double* Ut = (double*)malloc(sizeof(double) * (size_t)kI * (size_t)kJ);
    for (int32_t b = 0; b < kJ; ++b)
      for (int32_t a = 0; a < kI; ++a) G[(int64_t)b * kI + a] = C[(int64_t)I[a] * kJ + b];
    rank = orc_nucleus_rect(G, kJ, kI, rank_tol, Ut);              /* kI x kJ = pinv(G^T) */
    for (int32_t b = 0; b < kJ; ++b)
      for (int32_t a = 0; a < kI; ++a) U[(int64_t)b * kI + a] = Ut[(int64_t)a * kJ + b];
    free(Ut);
  }
  left_outputs(p, I, kI, J, kJ, C, R);
  if (rank < (kI < kJ ? kI : kJ) && status == ORC_OK) status = ORC_WARN_RANK_DEFICIENT;
  info[0] = rank; info[1] = kI; info[2] = kJ; info[3] = status;
  free(S); free(v); free(Ct); free(G);
  return status;
}

/* ------------------------------------------------------------------ */
/* CUR apply and sampled residual                                      */
/* ------------------------------------------------------------------ */
/* Y = C (U (R X)): C m x k, U k x k, R k x n, X n x nrhs, Y m x nrhs, all
 * row-major; each inner product an ascending fma chain. */
void orc_cur_apply(const double* C, const double* U, const double* R, int64_t m, int64_t n, int32_t k,
                   const double* X, int32_t nrhs, double* Y) {
  double* T1 = (double*)malloc(sizeof(double) * (size_t)k * (size_t)nrhs);
  double* T2 = (double*)malloc(sizeof(double) * (size_t)k * (size_t)nrhs);
  for (int32_t a = 0; a < k; ++a)
    for (int32_t c = 0; c < nrhs; ++c) {
      double s = 0.0;
      for (int64_t j = 0; j < n; ++j) s = fma(R[(int64_t)a * n + j], X[j * nrhs + c], s);
      T1[a * nrhs + c] = s;
    }
  for (int32_t a = 0; a < k; ++a)
    for (int32_t c = 0; c < nrhs; ++c) {
      double s = 0.0;
      for (int32_t b = 0; b < k; ++b) s = fma(U[a * k + b], T1[b * nrhs + c], s);
      T2[a * nrhs + c] = s;
    }
  for (int64_t i = 0; i < m; ++i)
    for (int32_t c = 0; c < nrhs; ++c) {
      double s = 0.0;
      for (int32_t a = 0; a < k; ++a) s = fma(C[i * k + a], T2[a * nrhs + c], s);
      Y[i * nrhs + c] = s;
    }
  free(T1); free(T2);
}

/*
 * orc_residual_sample: the q x s submatrix E[Q,S] of E = W - C U R (rows Q,
 * columns S given), and its statistics
 *   stats[0] mean of e,  stats[1] variance (1/K) sum (e - mean)^2,
 *   stats[2] mean of |e|, stats[3] max |e| (Chebyshev norm of the sample),
 *   stats[4] ||E[Q,S]||_F / ||W[Q,S]||_F (Frobenius-ratio estimate).
 * The paper tests the sample mean and variance of K = qs >= 100 i.i.d.
 * entries; the sums here run in ascending (row, column) order.
 * E (q x s) is written if Eout != NULL.
 */
void orc_residual_sample_rect(const orc_problem* p, const double* C, const double* U, const double* R, int32_t k,
                              int32_t l, const int32_t* Q, int32_t q, const int32_t* S, int32_t s, double* stats,
                              double* Eout);
void orc_residual_sample(const orc_problem* p, const double* C, const double* U, const double* R, int32_t k,
                         const int32_t* Q, int32_t q, const int32_t* S, int32_t s, double* stats, double* Eout) {
  orc_residual_sample_rect(p, C, U, R, k, k, Q, q, S, s, stats, Eout);
}

/* The same for a rectangular generator: C m x l, U l x k, R k x n. */
void orc_residual_sample_rect(const orc_problem* p, const double* C, const double* U, const double* R, int32_t k,
                              int32_t l, const int32_t* Q, int32_t q, const int32_t* S, int32_t s, double* stats,
                              double* Eout) {
  double* cu = (double*)malloc(sizeof(double) * (size_t)k);
  double* e = (double*)malloc(sizeof(double) * (size_t)q * (size_t)s);
  int64_t n = p->n;
  double sw2 = 0.0;
  for (int32_t a = 0; a < q; ++a) {
    /* row Q[a] of C U */
    for (int32_t b = 0; b < k; ++b) {
      double t = 0.0;
      for (int32_t c = 0; c < l; ++c) t = fma(C[(int64_t)Q[a] * l + c], U[c * k + b], t);
      cu[b] = t;
    }
    for (int32_t c = 0; c < s; ++c) {
      double t = 0.0;
      for (int32_t b = 0; b < k; ++b) t = fma(cu[b], R[(int64_t)b * n + S[c]], t);
      double w = entry_w(p, Q[a], S[c]);
      e[(int64_t)a * s + c] = w - t;
      sw2 = fma(w, w, sw2);
    }
  }
  double K = (double)q * (double)s;
  double sum = 0.0, sabs = 0.0, mx = 0.0, se2 = 0.0;
  for (int64_t t = 0; t < (int64_t)q * s; ++t) {
    sum += e[t]; sabs += fabs(e[t]); se2 = fma(e[t], e[t], se2);
    if (fabs(e[t]) > mx) mx = fabs(e[t]);
  }
  double mean = sum / K, var = 0.0;
  for (int64_t t = 0; t < (int64_t)q * s; ++t) { double d = e[t] - mean; var = fma(d, d, var); }
  stats[0] = mean; stats[1] = var / K; stats[2] = sabs / K; stats[3] = mx;
  stats[4] = (sw2 > 0.0) ? sqrt(se2) / sqrt(sw2) : 0.0;
  if (Eout) memcpy(Eout, e, sizeof(double) * (size_t)q * (size_t)s);
  free(cu); free(e);
}

/* ------------------------------------------------------------------ */
/* Test helpers: brute force, dense multipliers, Jacobi SVD            */
/* ------------------------------------------------------------------ */

/* |det| of a k x k matrix by Gaussian elimination with partial pivoting. */
static double absdet(double* B, int k) {
  double d = 1.0;
  for (int t = 0; t < k; ++t) {
    int r = t;
    for (int p = t + 1; p < k; ++p) if (fabs(B[p * k + t]) > fabs(B[r * k + t])) r = p;
    if (B[r * k + t] == 0.0) return 0.0;
    if (r != t) for (int q = 0; q < k; ++q) { double tmp = B[t * k + q]; B[t * k + q] = B[r * k + q]; B[r * k + q] = tmp; }
    d *= fabs(B[t * k + t]);
    for (int p = t + 1; p < k; ++p) {
      double l = B[p * k + t] / B[t * k + t];
      for (int q = t; q < k; ++q) B[p * k + q] -= l * B[t * k + q];
    }
  }
  return d;
}

/* Exhaustive search over all k-subsets of the n columns of A (k x n): the
 * maximal |det A[:,J]| (the definition of maximal volume, eqvol).  Returns
 * the max; best J (ascending) in Jbest. */
double orc_brute_maxvol(const double* A, int32_t k, int32_t n, int32_t* Jbest) {
  int32_t* c = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  double* B = (double*)malloc(sizeof(double) * (size_t)k * (size_t)k);
  for (int32_t i = 0; i < k; ++i) c[i] = i;
  double best = -1.0;
  for (;;) {
    for (int32_t a = 0; a < k; ++a)
      for (int32_t b = 0; b < k; ++b) B[a * k + b] = A[(int64_t)a * n + c[b]];
    double d = absdet(B, k);
    if (d > best) { best = d; memcpy(Jbest, c, sizeof(int32_t) * (size_t)k); }
    int32_t i = k - 1;
    while (i >= 0 && c[i] == n - k + i) --i;
    if (i < 0) break;
    ++c[i];
    for (int32_t j = i + 1; j < k; ++j) c[j] = c[j - 1] + 1;
  }
  free(c); free(B);
  return best;
}

/* Dense n x n H_{n,d} built by the recursion of equation eqrfd,
 * H_{2q} = [[H_q, H_q], [H_q, -H_q]], started from H_s = I_s (n = 2^d s). */
void orc_hadamard_abridged(int64_t n, int32_t d, double* H) {
  int64_t s = n >> d;
  memset(H, 0, sizeof(double) * (size_t)n * (size_t)n);
  for (int64_t i = 0; i < s; ++i) H[i * n + i] = 1.0;
  for (int64_t q = s; q < n; q *= 2) {
    for (int64_t i = 0; i < q; ++i)
      for (int64_t j = 0; j < q; ++j) {
        double v = H[i * n + j];
        H[i * n + (j + q)] = v;
        H[(i + q) * n + j] = v;
        H[(i + q) * n + (j + q)] = -v;
      }
  }
}

/* Dense complex Omega_{n,d} (re, im: n x n row-major) by the decimation-in-
 * frequency recursion of equation eqfd, cut at depth d: Omega_s = I_s (n = 2^d s)
 * and, for q = s, 2s, ..., n/2,
 *   Omega_{2q} = Phat [[Omega_q, Omega_q], [Omega_q Dhat_q, -Omega_q Dhat_q]],
 * Dhat_q = diag(w_{2q}^j), j = 0..q-1, w_N = exp(2 pi sqrt(-1) / N).  Phat puts
 * row i of the upper block on row 2i and row i of the lower block on row 2i + 1
 * (the even / odd interleaving under which the recursion at d = log2 n gives the
 * DFT matrix of equation eqdft). */
void orc_fourier_abridged(int64_t n, int32_t d, double* re, double* im) {
  int64_t s = n >> d;
  double* tr = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double* ti = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  memset(re, 0, sizeof(double) * (size_t)n * (size_t)n);
  memset(im, 0, sizeof(double) * (size_t)n * (size_t)n);
  for (int64_t i = 0; i < s; ++i) re[i * n + i] = 1.0;
  for (int64_t q = s; q < n; q *= 2) {
    /* the q x q block Omega_q sits in the top-left corner of (re, im) */
    for (int64_t i = 0; i < q; ++i)
      for (int64_t j = 0; j < q; ++j) {
        double ar = re[i * n + j], ai = im[i * n + j];
        double phi = (2.0 * ORC_PI * (double)j) / (double)(2 * q);
        double cr = cos(phi), ci = sin(phi);
        double br = ar * cr - ai * ci, bi = ar * ci + ai * cr;     /* (Omega_q Dhat_q)[i][j] */
        tr[(2 * i) * n + j] = ar;           ti[(2 * i) * n + j] = ai;
        tr[(2 * i) * n + j + q] = ar;       ti[(2 * i) * n + j + q] = ai;
        tr[(2 * i + 1) * n + j] = br;       ti[(2 * i + 1) * n + j] = bi;
        tr[(2 * i + 1) * n + j + q] = -br;  ti[(2 * i + 1) * n + j + q] = -bi;
      }
    for (int64_t i = 0; i < 2 * q; ++i)
      for (int64_t j = 0; j < 2 * q; ++j) { re[i * n + j] = tr[i * n + j]; im[i * n + j] = ti[i * n + j]; }
  }
  free(tr); free(ti);
}

/* Nonzeros of column c of Omega_{n,d}: 2^d (row, exponent e) pairs, the entry
 * being w_n^e.  By the recursion above, column c of Omega_{2q} is column
 * c' = c mod q of Omega_q on the even rows and the same column times
 * +-w_{2q}^{c'} (sign - when c >= q) on the odd rows; w_{2q} = w_n^{n/(2q)} and
 * -1 = w_n^{n/2}.  Returned in the order the recursion produces them. */
static void fourier_column(int64_t n, int32_t d, int64_t c, int64_t* rows, int64_t* ex) {
  int64_t s = n >> d;
  int64_t cs[32];                 /* the column index at each level, size 2^h s */
  int64_t q = n;
  for (int32_t h = d; h >= 0; --h) { cs[h] = c; if (h > 0) { q /= 2; c = c % q; } }
  /* level 0: column cs[0] of I_s */
  int64_t cnt = 1;
  rows[0] = cs[0]; ex[0] = 0;
  q = s;
  for (int32_t h = 1; h <= d; ++h) {
    int64_t cp = cs[h] % q, neg = cs[h] >= q;
    int64_t tw = (cp * (n / (2 * q)) + (neg ? n / 2 : 0)) % n;
    for (int64_t t = 0; t < cnt; ++t) {
      rows[cnt + t] = 2 * rows[t] + 1; ex[cnt + t] = (ex[t] + tw) % n;
      rows[t] = 2 * rows[t];
    }
    cnt *= 2;
    q *= 2;
  }
}

/* The 2n columns of [Re M, Im M] for M = D Omega_{n,d} P (before the scale
 * 2^(-d/2)): column j of M is D times column perm[j] of Omega_{n,d}, with
 * D = diag(dre + sqrt(-1) dim) (random points of the complex unit circle).  Column
 * j of the real form (j < n) holds Re(D_r w_n^e), column n + j holds
 * Im(D_r w_n^e), at the rows r of column perm[j], in ascending rows (2^d slots
 * per column). */
void orc_fourier_columns(int64_t n, int32_t d, const int32_t* perm, const double* dre, const double* dim,
                         int32_t* rows, double* wts) {
  int64_t w = 1LL << d;
  int64_t* rr = (int64_t*)malloc(sizeof(int64_t) * (size_t)w);
  int64_t* ee = (int64_t*)malloc(sizeof(int64_t) * (size_t)w);
  for (int64_t j = 0; j < n; ++j) {
    fourier_column(n, d, perm[j], rr, ee);
    /* ascending rows (insertion sort: 2^d is small) */
    for (int64_t a = 1; a < w; ++a)
      for (int64_t b = a; b > 0 && rr[b - 1] > rr[b]; --b) {
        int64_t t = rr[b]; rr[b] = rr[b - 1]; rr[b - 1] = t;
        t = ee[b]; ee[b] = ee[b - 1]; ee[b - 1] = t;
      }
    for (int64_t t = 0; t < w; ++t) {
      int64_t r = rr[t];
      double phi = (2.0 * ORC_PI * (double)ee[t]) / (double)n;
      double cr = cos(phi), ci = sin(phi);
      rows[j * w + t] = (int32_t)r;
      wts[j * w + t] = dre[r] * cr - dim[r] * ci;
      rows[(n + j) * w + t] = (int32_t)r;
      wts[(n + j) * w + t] = dre[r] * ci + dim[r] * cr;
    }
  }
  free(rr); free(ee);
}

/* Dense multiplier M (N x N, N = n for a right multiplier, m for a left one)
 * of the problem, assembled from its definition: ARHT M = 2^(-d/2) D H_{N,d} P
 * (H from the recursion above, P moving column perm[j] of D H to position j);
 * sparse: M[srow][j] = ssign / sqrt(nnz). */
void orc_multiplier_dense(const orc_problem* p, double* M) {
  int64_t n = p->mside ? p->m : p->n;
  if (p->mkind == ORC_MULT_ARFT) {
    /* the n x 2n real form [Re M, Im M] of M = 2^(-d/2) D Omega_{n,d} P, from the
     * dense recursion (not from the column lists the gathers use) */
    double* re = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double* im = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    orc_fourier_abridged(n, p->depth, re, im);
    double sc = arht_scale(p->depth);
    for (int64_t r = 0; r < n; ++r)
      for (int64_t j = 0; j < n; ++j) {
        double ar = re[r * n + p->perm[j]], ai = im[r * n + p->perm[j]];
        M[r * 2 * n + j] = sc * (p->dre[r] * ar - p->dim[r] * ai);
        M[r * 2 * n + n + j] = sc * (p->dre[r] * ai + p->dim[r] * ar);
      }
    free(re); free(im);
    return;
  }
  memset(M, 0, sizeof(double) * (size_t)n * (size_t)n);
  if (p->mkind == ORC_MULT_NONE) { for (int64_t i = 0; i < n; ++i) M[i * n + i] = 1.0; return; }
  if (p->mkind == ORC_MULT_SPARSE) {
    double v = 1.0 / sqrt((double)p->nnz);
    for (int64_t j = 0; j < n; ++j)
      for (int t = 0; t < p->nnz; ++t) M[(int64_t)p->srow[j * p->nnz + t] * n + j] = p->ssign[j * p->nnz + t] * v;
    return;
  }
  if (p->mkind == ORC_MULT_BIDIAG) {
    /* M = F_1 ... F_q built left to right: column a of M F = M e_b + s M e_b' */
    double* T = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    for (int64_t i = 0; i < n; ++i) M[i * n + i] = 1.0;
    for (int32_t f = 0; f < p->depth; ++f) {
      for (int64_t a = 0; a < n; ++a) {
        int64_t b = p->perm[(int64_t)f * n + a], b1 = (b + 1) % n;
        double sg = (double)p->dsign[(int64_t)f * n + b1];
        for (int64_t i = 0; i < n; ++i) T[i * n + a] = M[i * n + b] + sg * M[i * n + b1];
      }
      memcpy(M, T, sizeof(double) * (size_t)n * (size_t)n);
    }
    double sc = arht_scale(p->depth);
    for (int64_t i = 0; i < n * n; ++i) M[i] *= sc;
    free(T);
    return;
  }
  double* H = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  orc_hadamard_abridged(n, p->depth, H);
  double sc = arht_scale(p->depth);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) M[i * n + j] = sc * (double)p->dsign[i] * H[i * n + p->perm[j]];
  free(H);
}

/* One-sided Jacobi SVD (Hestenes) of A (m x n row-major, m >= n): A = Uo diag(s) V^T.
 * Columns are rotated until every pair is orthogonal to relative tolerance 1e-15.
 * Singular values sorted descending.  Uo m x n, s n, V n x n (row-major). */
int orc_jacobi_svd(const double* A, int32_t m, int32_t n, double* Uo, double* s, double* V) {
  double* B = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
  memcpy(B, A, sizeof(double) * (size_t)m * (size_t)n);
  for (int32_t i = 0; i < n; ++i) for (int32_t j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  int sweep;
  for (sweep = 0; sweep < 100; ++sweep) {
    int rotated = 0;
    for (int32_t p = 0; p < n - 1; ++p)
      for (int32_t q = p + 1; q < n; ++q) {
        double al = 0, be = 0, ga = 0;
        for (int32_t i = 0; i < m; ++i) {
          al += B[i * n + p] * B[i * n + p];
          be += B[i * n + q] * B[i * n + q];
          ga += B[i * n + p] * B[i * n + q];
        }
        if (fabs(ga) <= 1e-15 * sqrt(al * be) || ga == 0.0) continue;
        rotated = 1;
        double zeta = (be - al) / (2.0 * ga);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
        for (int32_t i = 0; i < m; ++i) {
          double bp = B[i * n + p], bq = B[i * n + q];
          B[i * n + p] = c * bp - sn * bq; B[i * n + q] = sn * bp + c * bq;
        }
        for (int32_t i = 0; i < n; ++i) {
          double vp = V[i * n + p], vq = V[i * n + q];
          V[i * n + p] = c * vp - sn * vq; V[i * n + q] = sn * vp + c * vq;
        }
      }
    if (!rotated) break;
  }
  for (int32_t j = 0; j < n; ++j) {
    double nr = 0; for (int32_t i = 0; i < m; ++i) nr += B[i * n + j] * B[i * n + j];
    s[j] = sqrt(nr);
  }
  /* sort descending (selection sort, permuting columns) */
  for (int32_t a = 0; a < n; ++a) {
    int32_t b = a;
    for (int32_t c = a + 1; c < n; ++c) if (s[c] > s[b]) b = c;
    if (b != a) {
      double t = s[a]; s[a] = s[b]; s[b] = t;
      for (int32_t i = 0; i < m; ++i) { t = B[i * n + a]; B[i * n + a] = B[i * n + b]; B[i * n + b] = t; }
      for (int32_t i = 0; i < n; ++i) { t = V[i * n + a]; V[i * n + a] = V[i * n + b]; V[i * n + b] = t; }
    }
  }
  for (int32_t j = 0; j < n; ++j)
    for (int32_t i = 0; i < m; ++i) Uo[i * n + j] = (s[j] > 0) ? B[i * n + j] / s[j] : 0.0;
  free(B);
  return sweep;
}

/* ------------------------------------------------------------------ */
/* Differentiable CUR apply with a Gaussian kernel (no counterpart in   */
/* the paper; the FMM stage (iii) product y = C U R x with C, R and the */
/* core G = W[I,J] sampled from K(x, y) = exp(-|x - y|^2 / (2 l^2)) at  */
/* fixed pivots, U = G^{-1})                                            */
/* ------------------------------------------------------------------ */
static double gauss_k(const double* x, const double* y, double ell, double* d2out) {
  double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
  double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
  if (d2out) *d2out = r2;
  return exp(-(r2 / (2.0 * ell * ell)));
}

/* y = C U R x for one block: X (m x 3), Y (n x 3), pivots I (k rows of X),
 * J (k rows of Y), x (n x nrhs), y (m x nrhs); U = G^{-1} by orc_nucleus with
 * tolerance 0 (G is assumed nonsingular).  t1 = R x and t2 = U t1 (k x nrhs)
 * are returned for the backward when non-NULL. */
void orc_gauss_cur_apply(const double* X, int64_t m, const double* Y, int64_t n, const int32_t* I, const int32_t* J,
                         int32_t k, double ell, const double* x, int32_t nrhs, double* y, double* Uout, double* t1o,
                         double* t2o) {
  double* G = (double*)malloc(sizeof(double) * (size_t)k * k);
  double* U = (double*)malloc(sizeof(double) * (size_t)k * k);
  double* t1 = (double*)calloc((size_t)k * nrhs, sizeof(double));
  double* t2 = (double*)calloc((size_t)k * nrhs, sizeof(double));
  for (int32_t a = 0; a < k; ++a)
    for (int32_t b = 0; b < k; ++b) G[a * k + b] = gauss_k(X + 3 * (int64_t)I[a], Y + 3 * (int64_t)J[b], ell, NULL);
  orc_nucleus(G, k, 0.0, U);
  for (int32_t a = 0; a < k; ++a)
    for (int64_t j = 0; j < n; ++j) {
      double r = gauss_k(X + 3 * (int64_t)I[a], Y + 3 * j, ell, NULL);
      for (int32_t c = 0; c < nrhs; ++c) t1[a * nrhs + c] = fma(r, x[j * nrhs + c], t1[a * nrhs + c]);
    }
  for (int32_t a = 0; a < k; ++a)
    for (int32_t c = 0; c < nrhs; ++c) {
      double s = 0.0;
      for (int32_t b = 0; b < k; ++b) s = fma(U[a * k + b], t1[b * nrhs + c], s);
      t2[a * nrhs + c] = s;
    }
  for (int64_t i = 0; i < m; ++i)
    for (int32_t c = 0; c < nrhs; ++c) y[i * nrhs + c] = 0.0;
  for (int64_t i = 0; i < m; ++i)
    for (int32_t a = 0; a < k; ++a) {
      double cv = gauss_k(X + 3 * i, Y + 3 * (int64_t)J[a], ell, NULL);
      for (int32_t c = 0; c < nrhs; ++c) y[i * nrhs + c] = fma(cv, t2[a * nrhs + c], y[i * nrhs + c]);
    }
  if (Uout) memcpy(Uout, U, sizeof(double) * (size_t)k * k);
  if (t1o) memcpy(t1o, t1, sizeof(double) * (size_t)k * nrhs);
  if (t2o) memcpy(t2o, t2, sizeof(double) * (size_t)k * nrhs);
  free(G); free(U); free(t1); free(t2);
}

/* Backward of y = C U R x at fixed pivots, given dy = dL/dy (m x nrhs):
 *   s1 = C^T dy, s2 = U^T s1, dx = R^T s2,
 *   dC = dy t2^T (m x k), dR = s2 x^T (k x n), dG = -s2 t2^T (k x k)  (U = G^{-1}),
 *   dl = sum of dC, dR, dG against dK/dl = K |x - y|^2 / l^3 over their entries.
 * Any of dC, dR, dG may be NULL. */
void orc_gauss_cur_backward(const double* X, int64_t m, const double* Y, int64_t n, const int32_t* I,
                            const int32_t* J, int32_t k, double ell, const double* x, const double* dy, int32_t nrhs,
                            double* dx, double* dC, double* dR, double* dG, double* dell) {
  double* U = (double*)malloc(sizeof(double) * (size_t)k * k);
  double* t1 = (double*)malloc(sizeof(double) * (size_t)k * nrhs);
  double* t2 = (double*)malloc(sizeof(double) * (size_t)k * nrhs);
  double* yv = (double*)malloc(sizeof(double) * (size_t)m * nrhs);
  double* s1 = (double*)calloc((size_t)k * nrhs, sizeof(double));
  double* s2 = (double*)calloc((size_t)k * nrhs, sizeof(double));
  orc_gauss_cur_apply(X, m, Y, n, I, J, k, ell, x, nrhs, yv, U, t1, t2);
  const double l3 = ell * ell * ell;
  double dl = 0.0;
  for (int64_t i = 0; i < m; ++i)
    for (int32_t a = 0; a < k; ++a) {
      double d2, cv = gauss_k(X + 3 * i, Y + 3 * (int64_t)J[a], ell, &d2);
      double g = 0.0;
      for (int32_t c = 0; c < nrhs; ++c) {
        s1[a * nrhs + c] = fma(cv, dy[i * nrhs + c], s1[a * nrhs + c]);
        g = fma(dy[i * nrhs + c], t2[a * nrhs + c], g);
      }
      if (dC) dC[i * k + a] = g;
      dl = fma(g, cv * d2 / l3, dl);
    }
  for (int32_t a = 0; a < k; ++a)
    for (int32_t c = 0; c < nrhs; ++c) {
      double s = 0.0;
      for (int32_t b = 0; b < k; ++b) s = fma(U[b * k + a], s1[b * nrhs + c], s);
      s2[a * nrhs + c] = s;
    }
  for (int64_t j = 0; j < n; ++j)
    for (int32_t c = 0; c < nrhs; ++c) dx[j * nrhs + c] = 0.0;
  for (int32_t a = 0; a < k; ++a)
    for (int64_t j = 0; j < n; ++j) {
      double d2, r = gauss_k(X + 3 * (int64_t)I[a], Y + 3 * j, ell, &d2);
      double g = 0.0;
      for (int32_t c = 0; c < nrhs; ++c) {
        dx[j * nrhs + c] = fma(r, s2[a * nrhs + c], dx[j * nrhs + c]);
        g = fma(s2[a * nrhs + c], x[j * nrhs + c], g);
      }
      if (dR) dR[(int64_t)a * n + j] = g;
      dl = fma(g, r * d2 / l3, dl);
    }
  for (int32_t a = 0; a < k; ++a)
    for (int32_t b = 0; b < k; ++b) {
      double d2, gv = gauss_k(X + 3 * (int64_t)I[a], Y + 3 * (int64_t)J[b], ell, &d2);
      double g = 0.0;
      for (int32_t c = 0; c < nrhs; ++c) g = fma(-s2[a * nrhs + c], t2[b * nrhs + c], g);
      if (dG) dG[a * k + b] = g;
      dl = fma(g, gv * d2 / l3, dl);
    }
  *dell = dl;
  free(U); free(t1); free(t2); free(yv); free(s1); free(s2);
}
