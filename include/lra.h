/*
 * lra.h -- C ABI of a GB300 (sm_103a) library for superfast cross-approximation
 * (C-A) CUR low-rank approximation, after Pan, Luan, Svadlenka, Zhao,
 * "Superfast Accurate Low Rank Approximation" (arXiv:1710.07946).
 *
 * Conventions for every entry point:
 *  - Pointers documented as "device" point to CUDA device memory of the current
 *    device; "host" pointers to ordinary host memory.  All matrices are row-major.
 *  - The caller owns every buffer it passes (inputs, outputs, workspace).  The
 *    library allocates device memory only in lra_precondition (the multiplier
 *    descriptor, freed by lra_multiplier_destroy); the compute calls allocate
 *    nothing: scratch comes from the caller's workspace, sized by the matching
 *    *_workspace_size query.
 *  - Calls are asynchronous on the given stream (0 = legacy default stream).  The
 *    returned status covers host-side validation and launch errors only; problems
 *    detected on the device (zero pivots, non-finite strips, an unfinished swap
 *    loop, an expired wait) are written to the device status word named in each
 *    call and are visible after the stream is synchronised.
 *  - No call aborts, traps or prints.  Every device-side wait is bounded in time
 *    and reports LRA_ERR_TIMEOUT instead of hanging.
 */
#ifndef LRA_H
#define LRA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* lra_stream_t;   /* a cudaStream_t */

typedef enum {
  LRA_OK = 0,
  LRA_ERR_INVALID_ARG = 1,      /* bad sizes, pointers, index sets or options       */
  LRA_ERR_CUDA = 2,             /* a CUDA runtime call or launch failed             */
  LRA_ERR_NONFINITE = 3,        /* a gathered strip held NaN or Inf                 */
  LRA_ERR_TIMEOUT = 4,          /* a bounded device-side wait expired               */
  LRA_ERR_WORKSPACE = 5,        /* workspace missing or smaller than the query      */
  LRA_WARN_RANK_DEFICIENT = 16, /* a zero pivot (strip rank < k) or core rank < k   */
  LRA_WARN_NOT_CONVERGED = 17   /* max_swaps stopped a maxvol swap loop             */
} lra_status;

typedef enum { LRA_F64 = 0, LRA_F32 = 1, LRA_BF16 = 2 } lra_dtype;

/* Input access (paper: the m x n input W, accessed either as a whole or entry by
 * entry; "superfast" algorithms touch only O((m+n)k) of its entries). */
typedef enum {
  LRA_DENSE = 0,            /* W stored densely                                    */
  LRA_KERNEL_LAPLACE = 1,   /* w_ij = 1 / |x_i - y_j|, evaluated on demand         */
  LRA_KERNEL_GAUSSIAN = 2   /* w_ij = exp(-|x_i - y_j|^2 / (2 l^2)), on demand      */
} lra_source;

typedef struct {
  int32_t src;           /* lra_source                                               */
  int32_t dtype;         /* dense: storage type, LRA_F64 or LRA_F32.  Laplace kernel:
                            LRA_F64 (w = 1/sqrt(r2), FP64) or LRA_F32 (w = fl32(1 /
                            sqrt(fl32(r2))), each FP32 operation correctly rounded,
                            r2 the FP64 squared distance; relative distance to the
                            FP64 entry <= 1.5 * 2^-23) or LRA_BF16 (that FP32
                            entry rounded to bfloat16, to nearest even: relative
                            distance <= 2^-8 + 1.5 * 2^-23).  Gaussian kernel:
                            LRA_F64.
                            Any other value is LRA_ERR_INVALID_ARG.                  */
  int64_t m, n;          /* rows, columns; 1 <= m, n < 2^31                          */
  const void* W;         /* dense: device, m x n row-major, leading dimension ldw    */
  int64_t ldw;           /* dense: >= n                                              */
  const double* X;       /* kernel: device, m target points, 3 doubles each          */
  const double* Y;       /* kernel: device, n source points, 3 doubles each          */
  double length_scale;   /* Gaussian kernel l > 0                                    */
} lra_problem;

/* ------------------------------------------------------------------------- */
/* Randomised pre-processing (multipliers)                                    */
/* ------------------------------------------------------------------------- */
typedef enum {
  LRA_MULT_NONE = 0,
  LRA_MULT_ARHT = 1,        /* abridged randomized Hadamard 2^{-d/2} D H_{n,d} P     */
  LRA_MULT_SPARSE_PM1 = 2,  /* sparse +-1/sqrt(nnz) multiplier, nnz entries / column */
  LRA_MULT_BIDIAG = 3,      /* 2^{-q/2} prod_{i=1..q} (I + D_i S) P_i, quasi-Gaussian */
  LRA_MULT_ARFT = 4         /* real form [Re M, Im M], M = 2^{-d/2} D Omega_{n,d} P     */
} lra_mult_kind;

typedef struct lra_multiplier_s* lra_multiplier;   /* opaque, library-owned */

/* Which side the multiplier is applied on (paper: Remark re2orddmn -- for
 * m > n pre-multiply instead of post-multiplying). */
typedef enum {
  LRA_SIDE_RIGHT = 0,       /* W' = W M, M n x n: C = W'[:, J], R = W[I, :]          */
  LRA_SIDE_LEFT = 1         /* W' = M^T W, M m x m: C = W[:, J], R = W'[I, :]        */
} lra_mult_side;

/*
 * lra_precondition -- describe the multiplier M of the pre-processed matrix
 * W' = W M (side LRA_SIDE_RIGHT, M n x n) or W' = M^T W (side LRA_SIDE_LEFT,
 * M m x m, for m > n), which C-A then approximates (paper: Section
 * "Pre-processing with matrices of abridged Hadamard and Fourier transforms";
 * Appendix "Abridged Hadamard and Fourier Multipliers", eqs. eqrfd / eqbschf;
 * Section "Pre-processing with quasi Gaussian matrices", case (i); Remark
 * re2orddmn for the left side).  M is never formed: the strip gathers evaluate
 * the needed entries of W' on the fly.  Below, n is the order of M (the
 * problem's n for the right side, its m for the left side).  With a left
 * multiplier, w'_ij combines entries of column j of W with the weights of
 * column i of M, in the order stated for the right side, and the CUR of W from
 * the generator (I, J) of W' is C = W[:, J], U = pinv(W'[I, J]), R = W'[I, :]
 * (the right-side back-transform applied to W^T).  Left multipliers serve
 * lra_ca_run, lra_ca_run_warm, lra_ca_run_noalloc and lra_multiplier_apply;
 * certified-FP32 mode runs them in FP64.
 *
 *   kind = LRA_MULT_ARHT: M = 2^{-d/2} D H_{n,d} P, depth_or_nnz = d (1..10),
 *     n = 2^d s.  H_{n,d} = H_{2^d} (x) I_s is the d-step abridged Hadamard
 *     recursion, D = diag(signs) with signs[i] = +-1 (n host int8),
 *     P the permutation taking column perm[j] of D H to position j
 *     (perm_or_rows: n host int32, a permutation of 0..n-1).
 *   kind = LRA_MULT_SPARSE_PM1: column j of M holds depth_or_nnz (1..16)
 *     entries signs[j*nnz+t] / sqrt(nnz) in the rows perm_or_rows[j*nnz+t],
 *     strictly ascending in t (host arrays of n*nnz int32 / int8).
 *   kind = LRA_MULT_BIDIAG (Section "Approximation of a Gaussian matrix by the
 *     product of random bidiagonal matrices", eq. def11): M = 2^{-q/2} F_1 ...
 *     F_q, q = depth_or_nnz (1..30), F_i = (I + D_i S) P_i with S the cyclic
 *     down-shift, D_i = diag(signs[i*n .. i*n+n)) (+-1) and column a of P_i equal
 *     to e_b, b = perm_or_rows[i*n + a] (host arrays of q*n int32 / int8, each
 *     row of perm_or_rows a permutation of 0..n-1).  Column j of M has at most
 *     min(2^q, n) nonzeros, integer multiples of 2^{-q/2} (|integer| <= 2^q);
 *     w'_ij adds them in ascending rows, each as fma(value, w, sum), and scales
 *     once.  The handle holds n * min(2^q, n) (row, int32 weight) slots, built on
 *     the host in O(n q min(2^q, n)) time; small q keeps the gathers superfast,
 *     and the paper's 20-factor products make every column dense.  2 <= n < 2^31.
 * The random draws (signs, permutation, positions) are inputs, so that runs are
 * reproducible.  The descriptor is copied to device memory owned by the handle;
 * the host arrays may be freed on return.  The copy is synchronous.
 * Errors: LRA_ERR_INVALID_ARG (bad kind or side, sizes, out-of-range or
 * unsorted indices, signs not +-1), LRA_ERR_CUDA.  A call that uses the handle
 * with a problem whose m (left) or n (right) differs from the handle's n
 * returns LRA_ERR_INVALID_ARG.
 */
lra_status lra_precondition(lra_multiplier* out, int32_t kind, int32_t side, int64_t n, int32_t depth_or_nnz,
                            const int32_t* perm_or_rows, const int8_t* signs);

/*
 * lra_precondition_fourier -- the abridged randomized Fourier multiplier
 * (paper: Appendix "Abridged Hadamard and Fourier Multipliers", eq. eqfd; the
 * ARFT of the pre-processing tests) in real form, for real inputs: a right
 * multiplier M' = [Re M, Im M] (n x 2n) with M = 2^{-d/2} D Omega_{n,d} P, so
 * the pre-processed W' = W M' has 2n columns and C-A selects J among them.
 *   Omega_{n,d}: the DIF recursion Omega_{2q} = Phat [[Omega_q, Omega_q],
 *     [Omega_q Dhat_q, -Omega_q Dhat_q]] from Omega_s = I_s (n = 2^d s), with
 *     Dhat_q = diag(w_{2q}^j), j < q, w_N = exp(2 pi sqrt(-1) / N), and Phat
 *     placing row i of the upper block on row 2i, of the lower on row 2i + 1
 *     (at d = log2 n this is the DFT matrix).  Every column has 2^d nonzeros.
 *   D = diag(diag[2r] + sqrt(-1) diag[2r+1]): n host (cos, sin) pairs of
 *     random points on the complex unit circle (|D_r| = 1 within 1e-12);
 *   P: column j of M is D times column perm[j] of Omega_{n,d} (perm: n host
 *     int32, a permutation of 0..n-1).
 * Column j < n of M' holds Re(D_r w_n^e) and column n + j holds Im(D_r w_n^e)
 * at the rows r of column perm[j] of Omega_{n,d} (entries w_n^e); the weights
 * are formed on the host (cos and sin of 2 pi e / n, then the complex product)
 * and w'_ij adds its 2^d terms in ascending rows, each as fma(weight, w, sum),
 * then scales by 2^{-d/2}.  M' has orthonormal rows, so the CUR of W from the
 * generator (I, J) of W' is C = W'[:, J], U = pinv(W'[I, J]), R = W[I, :]
 * (Algorithm alglratpsvd1 with H = M').  depth 1..10, n a multiple of 2^d,
 * 2 <= n < 2^30.  Serves lra_ca_run, lra_ca_run_warm, lra_ca_run_noalloc and
 * lra_multiplier_apply (W' m x 2n); certified-FP32 mode runs it in FP64.
 * Errors: LRA_ERR_INVALID_ARG (sizes, perm not a permutation, |D_r| != 1),
 * LRA_ERR_CUDA.
 */
lra_status lra_precondition_fourier(lra_multiplier* out, int64_t n, int32_t depth, const int32_t* perm,
                                    const double* diag);

/* Free a multiplier handle (NULL is accepted). */
lra_status lra_multiplier_destroy(lra_multiplier mult);

/*
 * lra_multiplier_apply -- the pre-processed input W' = W M (or M^T W for a
 * left multiplier) written out as a
 * dense FP64 matrix (paper: the bidiagonal pre-processing tests multiply each
 * input by the factors before C-A; the CUR of W from generators of W' is
 * C = W'[:, J], U = pinv(W'[I, J]), R = W[I, :], as for lra_ca_run with a
 * multiplier).  Entry (i, j) is formed exactly as the C-A gathers form w'_ij
 * (same terms, same order, same rounding), so a C-A run on the dense W' with no
 * multiplier selects the same I and J and returns the same C and U as a run on
 * (W, M); its R is W'[I, :], and lra_gather_rows gives R = W[I, :].
 * prob: W (dense F64/F32, or kernel entries), m x n.  mult: a handle for n
 * columns, or NULL (W' = W).  Wp: caller-owned device buffer, m x n' row-major,
 * leading dimension ldwp >= n' (n' = 2n for LRA_MULT_ARFT, n otherwise).  Cost: m n times the nonzeros of a column of M
 * fused multiply-adds (n for the 20-factor bidiagonal products).  Entries of W
 * must be finite.  Asynchronous on the stream.
 * Errors: LRA_ERR_INVALID_ARG (bad problem, sizes, n of the handle), LRA_ERR_CUDA.
 */
lra_status lra_multiplier_apply(const lra_problem* prob, lra_multiplier mult, double* Wp, int64_t ldwp,
                                lra_stream_t stream);

/*
 * lra_gather_rows -- R = W[I, :] (k x n FP64, row-major, caller-owned device
 * buffer) read from the original input (paper: the row factor of the CUR LRA,
 * Section "CUR LRA"; for a pre-processed input it is taken from W, not W').
 * I: k device int32 row indices.  A row index outside [0, m) fills its row of R
 * with NaN and sets *status_dev (device int32, may be NULL; the caller zeroes it)
 * to LRA_ERR_INVALID_ARG.  Asynchronous on the stream.
 * Errors: LRA_ERR_INVALID_ARG (bad problem, k < 1, NULL buffers), LRA_ERR_CUDA.
 */
lra_status lra_gather_rows(const lra_problem* prob, const int32_t* I, int32_t k, double* R, int32_t* status_dev,
                           lra_stream_t stream);

/* ------------------------------------------------------------------------- */
/* Cross-approximation                                                        */
/* ------------------------------------------------------------------------- */
typedef enum {
  LRA_MODE_FP64 = 0,        /* every gather, pivot and nucleus step in FP64, in the
                               operation order of the FP64 reference (bit-exact
                               pivots)                                              */
  LRA_MODE_MIXED = 1        /* each maxvol step first runs in FP32 with a rigorous
                               bound on every entry's distance to the FP64 reference;
                               a step whose every decision (pivot, swap, stop) the
                               bounds certify is kept, any other step is redone in
                               FP64.  Index sets, swap counts, C, R and U equal those
                               of LRA_MODE_FP64; logvol is then computed from the FP32
                               pivots (relative accuracy ~1e-6).  It runs on one CTA:
                               every block of a batch, and lra_ca_run inputs with
                               max(m, n) <= 2048; larger single runs, Gaussian
                               kernels and FP32 Laplace entries run in FP64.  After
                               a step falls back, the rest of that run (or block)
                               skips the FP32 attempt.                              */
} lra_mode;

typedef struct {
  int32_t k;             /* target rank = generator size, 1 <= k <= min(m, n, 64)    */
  int32_t sweeps;        /* C-A loops alpha >= 1 (one loop = column step + row step) */
  double h;              /* dominance threshold >= 1 (swap while max |B^{-1}A| > h)  */
  double rank_tol;       /* relative QRP truncation tolerance of the nucleus         */
  int32_t max_swaps;     /* cap on swaps per maxvol step (>= 0)                      */
  int32_t mode;          /* lra_mode                                                 */
  /* Generator size fitted to the numerical rank (batched runs only; lra_ca_run
     rejects nstages != 0).  The paper's tests size the generators at the
     numerical rank of the input at 1e-6; here it comes from the nucleus of the
     run itself.  nstages = 0: one run of size k.  Otherwise sizes
     k_stages[0] < ... < k_stages[nstages-1] = k, each clipped to the block's
     min(rows, cols): a complete C-A run of size k_s then its nucleus rank r_s;
     stop when r_s < k_s - rank_margin or at the largest size, else the next
     stage starts from the stage's rows I followed by the block's initial rows
     not in I (in order).  info[1], info[2] sum over the stages.               */
  int32_t nstages;       /* 0 .. LRA_MAX_STAGES                                      */
  int32_t rank_margin;   /* >= 0                                                     */
  int32_t k_stages[8];   /* LRA_MAX_STAGES entries, the first nstages used           */
  /* CTAs sharing one lra_ca_run / _warm / _noalloc (its strips split into that
     many column chunks, one pivot exchange among them per elimination step and
     swap): 0 = the library's choice (one per SM, at most one per 32 strip
     columns), else a count clipped to the number of SMs (raised if a chunk's
     scratch cannot fit a CTA's shared memory; mixed-mode runs of strips up to
     2048 columns always take one CTA).  The pivots and outputs do not depend on
     it.  A smaller grid leaves SMs to other work on the GPU; the default was
     the fastest on every single-run workload measured.  Batched calls ignore
     it.  Negative: LRA_ERR_INVALID_ARG.                                       */
  int32_t ctas;
} lra_ca_params;

#define LRA_MAX_STAGES 8

/* Outputs of one C-A CUR approximation W ~ C U R (all device, caller-owned). */
typedef struct {
  int32_t* I;            /* k row indices, in generator order                        */
  int32_t* J;            /* k column indices of W' (in [0, n'), n' = 2n for
                            LRA_MULT_ARFT, n otherwise), in generator order        */
  double* C;             /* m x k: W'[:, J] (right multiplier), W[:, J] (left)        */
  double* U;             /* k x k: nucleus, pinv of the rank-r truncation of W'[I,J] */
  double* R;             /* k x n: W[I, :] (original rows: for an orthogonal M this is
                            the back-transform R_H M^T of Algorithm alglratpsvd1);
                            W'[I, :] with a left multiplier                          */
  double* logvol;        /* 2*sweeps: log|det W'[I,J]| after each step (NaN if unrun) */
  int32_t* info;         /* LRA_INFO_LEN ints: numerical rank r, total swaps, loops run,
                            status, maxvol steps decided in FP32 (mixed mode), maxvol
                            steps run in FP64, generator rows k (rows of R, columns of
                            U), generator columns l (columns of C, rows of U; l = k
                            for square generators)                                  */
} lra_cur;

#define LRA_INFO_LEN 8

/*
 * lra_ca_workspace_size -- bytes of device workspace lra_ca_run needs for this
 * problem and these parameters (256-byte aligned start required).
 * Errors: LRA_ERR_INVALID_ARG.
 */
lra_status lra_ca_workspace_size(const lra_problem* prob, const lra_ca_params* par, lra_multiplier mult,
                                 size_t* bytes);

/*
 * lra_ca_run -- C-A CUR approximation of W' = W M (paper: Section "CUR LRA;
 * primitive, cynical, and cross-approximation algorithms", the C-A loops of
 * Figure fig4 in the Tests 2 schedule; Algorithms algdomin and alggos for each
 * step; Algorithm algcnnncl with Remark reubsc for the nucleus).
 *
 * Starting from the k rows I0 (device int32, distinct, in [0, m)), each loop
 * takes the row strip W'[I,:], finds k columns J whose k x k submatrix is
 * dominant in it (LUP initialisation with column pivoting in the first loop,
 * warm start from the current J afterwards, then volume-increasing swaps while
 * some |(W'[I,J])^{-1} W'[I,:]| entry exceeds h), then does the same on the
 * column strip W'[:,J] to update I.  The loop stops after `sweeps` loops or when
 * a loop makes no swap.  Finally C = W'[:,J], R = W[I,:], and U is the
 * pseudo-inverse of the rank-r truncation of W'[I,J] obtained from Householder
 * QR with column pivoting, r = #{t : |R_tt| > rank_tol |R_00|}.
 * In LRA_MODE_FP64 the index sets equal those of a sequential FP64 evaluation of
 * the same steps bit for bit (ties go to the lowest column, then row, index).
 * mult may be NULL (M = I).  workspace: device, >= the size query, 256-byte
 * aligned.  Device status (out->info[3]): LRA_OK, LRA_WARN_*, LRA_ERR_NONFINITE,
 * LRA_ERR_TIMEOUT or LRA_ERR_INVALID_ARG (I0 not distinct / out of range).
 * Host errors: LRA_ERR_INVALID_ARG, LRA_ERR_WORKSPACE, LRA_ERR_CUDA.
 */
lra_status lra_ca_run(const lra_problem* prob, const lra_ca_params* par, lra_multiplier mult, const int32_t* I0,
                      const lra_cur* out, void* workspace, size_t workspace_bytes, lra_stream_t stream);

/*
 * lra_ca_run_warm -- lra_ca_run with the first column step warm-started at the
 * columns J0 (device, k distinct indices in [0, n'), or NULL for the cold
 * start): resuming a run from its output (I, J) as (I0, J0) continues the
 * volume-increasing swaps, so the core's volume never decreases across the
 * restart (checkpoint / resume; the paper's C-A loops are defined by their
 * current (I, J)).  Invalid J0 gives status LRA_ERR_INVALID_ARG in info.
 * Arguments, workspace and errors otherwise as lra_ca_run.
 */
lra_status lra_ca_run_warm(const lra_problem* prob, const lra_ca_params* par, lra_multiplier mult, const int32_t* I0,
                           const int32_t* J0, const lra_cur* out, void* workspace, size_t workspace_bytes,
                           lra_stream_t stream);

/*
 * lra_rhtcur_run -- CUR LRA with Gaussian sampling (paper: Algorithm algrhtcur,
 * "Computation of a CUR LRA with Gaussian sampling"), with lbar = l = k:
 *   1. S = W Hbar (m x k): Hbar is the caller's n x k Gaussian matrix (device,
 *      FP64, row-major; the random draws are inputs), each entry of S the fma
 *      chain over the columns j of W in ascending order.  W is read as given
 *      (no multiplier); m n k fused multiply-adds, the step the paper marks as
 *      not superfast.
 *   2. Rows I: the algorithms of GE96 on S, here the maxvol selection of a
 *      k x k submatrix of locally maximal volume in S -- a one-loop C-A run on
 *      S^T from all k rows, whose cold first column step (LU with column
 *      pivoting, then swaps while max |B^{-1} S^T| > par->h) picks them.
 *   3. Columns J: a one-loop C-A run on the row strip W[I, :] from all k rows:
 *      its cold column step picks J, its row step orders I, its nucleus is U.
 *   4. C = W[:, J] (m x k), R = W[I, :] (k x n).
 * par: k (1..min(m, n, 64)), h, rank_tol, max_swaps as for lra_ca_run; sweeps
 * and mode are ignored (one loop each, FP64); nstages must be 0.
 * out: as lra_ca_run (logvol holds 2 doubles: the second run's).  info: rank,
 * swaps of both runs, loops 2, status (an error of either run first, else the
 * worse warning), 0, FP64 maxvol steps, k, k.
 * The workspace (lra_rhtcur_workspace_size) holds S^T (k x m), the row strip
 * (k x n) and the two runs' buffers.  Asynchronous on the stream.
 * Errors: LRA_ERR_INVALID_ARG, LRA_ERR_WORKSPACE, LRA_ERR_CUDA.
 */
lra_status lra_rhtcur_workspace_size(const lra_problem* prob, const lra_ca_params* par, size_t* bytes);
lra_status lra_rhtcur_run(const lra_problem* prob, const double* Hbar, const lra_ca_params* par, const lra_cur* out,
                          void* workspace, size_t workspace_bytes, lra_stream_t stream);

/*
 * lra_ca_run_noalloc -- lra_ca_run without a caller-supplied workspace, for
 * callers that cannot allocate device memory themselves: for instance a plug-in
 * running inside a host application whose own allocator owns the whole device
 * and forbids further cudaMalloc calls, or a program that only receives
 * pre-placed device buffers for its inputs and outputs.  The paper has no
 * counterpart: this is a deployment variant of lra_ca_run, with the same
 * arguments (minus the workspace), results and device status.
 *
 * Scratch: one static device array of LRA_NOALLOC_SCRATCH_BYTES (256 KiB) per
 * device, held by every device that loads the library until the process
 * exits.  Problems whose lra_ca_workspace_size exceeds it are rejected with
 * LRA_ERR_WORKSPACE before anything is launched (this happens when a strip
 * chunk does not fit in shared memory, e.g. k = 64 with n = 65536).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  The call allocates no device memory.  All calls on a
 * device share the one array: calls whose executions overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * The array keeps the last call's contents; every call clears the parts that
 * must start at zero.  The looked-up address belongs to the device's current
 * context: after a cudaDeviceReset the array may move, so do not call this
 * entry point again in that process until a call has returned LRA_ERR_CUDA
 * (which drops the cached address, so the next call looks it up afresh).
 */
#define LRA_NOALLOC_SCRATCH_BYTES (256u * 1024u)
lra_status lra_ca_run_noalloc(const lra_problem* prob, const lra_ca_params* par, lra_multiplier mult,
                              const int32_t* I0, const lra_cur* out, lra_stream_t stream);

/* ------------------------------------------------------------------------- */
/* Batches of independent blocks (HSS / FMM generators)                       */
/* ------------------------------------------------------------------------- */
/* A batch of nb submatrices W[row0 : row0+nrows, col0 : col0+ncols] of one
 * input (paper: Section "Application: HSS / FMM" -- the generators of the
 * neutered block columns are low-rank approximations of such off-diagonal
 * blocks, and C-A computes each of them superfast).  All arrays are device
 * memory, so a batched call can be captured in a CUDA graph. */
typedef struct {
  const int64_t* blocks;   /* nb x 4: row0, nrows, col0, ncols (nrows, ncols >= 1)      */
  const int64_t* offsets;  /* nb x 2: offsets, in doubles, of C_b in C and R_b in R      */
  const int32_t* order;    /* optional (NULL = 0..nb-1): the order in which blocks are
                              taken from the work queue; largest first balances the tail */
  int32_t nb;              /* number of blocks >= 1                                       */
  int64_t max_len;         /* >= max over blocks of max(nrows, ncols); sizes the scratch  */
  int32_t cta_threads;     /* CTA shape of the batched kernel: threads per CTA and CTAs  */
  int32_t ctas_per_sm;     /* per SM, one of lra_ca_batched_shapes (0, 0: the library's
                              default 512 x 1; lra_ca_batched_tune picks the fastest)    */
  int32_t pair_blocks;     /* 0 .. nb: lra_ca_run_batched runs the first pair_blocks
                              entries of the order each on a pair of CTAs that split its
                              strips (the shapes with 512 or 256 threads; FP64 mode), the
                              rest on one CTA each: large blocks then keep a short
                              critical path while small ones fill the SMs.  The results
                              do not depend on it.  Other batched calls ignore it.       */
} lra_batch;

/* Outputs of a batch (device, caller-owned).  Block b has slots for k_b =
 * min(k, nrows, ncols) generators and uses kf_b = info[b*LRA_INFO_LEN+6] of
 * them (kf_b = k_b without stages); its C_b (nrows x kf_b) and R_b (kf_b x
 * ncols) are row-major at the block's offsets (slots of nrows x k_b and
 * k_b x ncols); the other arrays have one fixed-size slot per block. */
typedef struct {
  int32_t* I;              /* nb x k: rows (block-local), first kf_b used                 */
  int32_t* J;              /* nb x k: columns (block-local)                               */
  double* C;               /* packed C_b, or NULL together with R: lra_ca_run_batched then
                              keeps only I, J, U, logvol and info (the factors' entries
                              are recomputed where they are used, e.g. by a
                              matrix-free lra_hmatvec); other batched calls need C, R  */
  double* U;               /* nb x k x k: U_b (kf_b x kf_b, row-major) at the slot start   */
  double* R;               /* packed R_b (NULL with C)                                    */
  double* logvol;          /* nb x 2*sweeps                                               */
  int32_t* info;           /* nb x LRA_INFO_LEN (as lra_cur.info)                          */
  double* work;            /* nb, or NULL: lra_ca_run_batched writes the algorithmic flops
                              of each block's run (every stage's maxvol steps -- LU,
                              back substitution, swaps, entries, fma = 2 -- and 5 k^3
                              per nucleus), for roofline accounting                    */
} lra_cur_batch;

/* Workspace bytes of lra_ca_run_batched (params: par->k is the largest rank),
 * enough for every CTA shape that can hold the batch. */
lra_status lra_ca_batched_workspace_size(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                                         size_t* bytes);

/*
 * lra_ca_run_batched -- lra_ca_run on every block of the batch, in one
 * persistent launch: each CTA takes the next block from a device work queue
 * and runs that block's C-A loop and nucleus alone, so the per-block results
 * are those of lra_ca_run on the block (same pivots, bit for bit).  k_b =
 * min(par->k, nrows, ncols); U_b truncates the core at par->rank_tol (adaptive
 * rank, info[0] of the block).  With par->nstages > 0 the generator size of
 * each block is staged up to k_b as lra_ca_params describes (info[6] = the
 * size used; the stages run follow from it).  Only dense and kernel inputs without
 * multipliers.
 * I0: device, nb x par->k block-local initial rows (first k_b of each slot
 * used, distinct).  A block outside the input or larger than max_len gets
 * status LRA_ERR_INVALID_ARG in its info slot; the others still run.
 * Errors: LRA_ERR_INVALID_ARG, LRA_ERR_WORKSPACE, LRA_ERR_CUDA.
 */
lra_status lra_ca_run_batched(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                              const int32_t* I0, const lra_cur_batch* out, void* workspace, size_t workspace_bytes,
                              lra_stream_t stream);

/*
 * lra_cynical_run_batched -- the cynical CUR algorithms on every block of a
 * batch (paper: Section "CUR LRA; primitive, cynical, and cross-approximation
 * algorithms"; the tests' Tests 3 and Tests 4), one CTA per block from a work
 * queue.  Block b's r x r generator (r = par->k) is taken inside a q x q sketch
 * W_b[K_b, L_b] (q = 4r in the paper, r <= q <= 64, q <= min(nrows, ncols)):
 *   kind 0 (Tests 3): K_b, L_b are the caller's (random) row and column sets;
 *   kind 1 (Tests 4): L_b is the caller's; one C-A loop with q x q generators
 *     makes the sketch (a cold maxvol step on the column strip W_b[:, L_b]
 *     picks K_b, one on the row strip W_b[K_b, :] picks L_b) and both sets are
 *     written back to K and L.
 * A C-A run of size r (par->sweeps loops, par->h, par->max_swaps) on the dense
 * sketch from its initial rows I0s[b] (r distinct indices in [0, q)) picks I',
 * J'; the outputs are I_b = K_b[I'], J_b = L_b[J'], C_b = W_b[:, J_b], R_b =
 * W_b[I_b, :] and U_b = the nucleus of W_b[I_b, J_b] at par->rank_tol, in the
 * layout of lra_cur_batch with k = r; info as lra_ca_run_batched (swaps of
 * every maxvol step, loops of the sketch run).  The results equal the FP64
 * reference's operation for operation.  par->mode must be LRA_MODE_FP64 and
 * par->nstages 0.  K, L: device nb x q int32 (block-local; for kind 1, K is
 * output only); I0s: device nb x r.  A block with invalid sets or smaller than
 * q gets status LRA_ERR_INVALID_ARG in its info slot.  The CTA shape is the
 * batch's cta_threads x ctas_per_sm (one of lra_ca_batched_shapes; 0, 0 =
 * for kind 0 the smallest CTAs whose shared-memory share holds the run, the
 * sketch runs having little work per barrier; for kind 1 512 x 1, its q-wide
 * maxvol steps being C-A steps).  The workspace query covers every shape that
 * fits.
 * Errors: LRA_ERR_INVALID_ARG, LRA_ERR_WORKSPACE, LRA_ERR_CUDA.
 */
lra_status lra_cynical_batched_workspace_size(const lra_problem* base, const lra_batch* batch,
                                              const lra_ca_params* par, int32_t kind, int32_t q, size_t* bytes);
lra_status lra_cynical_run_batched(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                                   int32_t kind, int32_t q, int32_t* K, int32_t* L, const int32_t* I0s,
                                   const lra_cur_batch* out, void* workspace, size_t workspace_bytes,
                                   lra_stream_t stream);

/*
 * lra_cynical_batched_tune -- autotuner of lra_cynical_run_batched for kind 0
 * (Tests 3; kind 1 rewrites its inputs and is rejected): times every CTA shape
 * as lra_ca_batched_tune does and returns the fastest in *cta_threads,
 * *ctas_per_sm, with the times in ms (-1 for shapes that do not fit) when ms is
 * not NULL.  Blocks the calling thread; not capturable.
 */
lra_status lra_cynical_batched_tune(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                                    int32_t kind, int32_t q, int32_t* K, int32_t* L, const int32_t* I0s,
                                    const lra_cur_batch* out, void* workspace, size_t workspace_bytes,
                                    lra_stream_t stream, int32_t reps, int32_t* cta_threads, int32_t* ctas_per_sm,
                                    float* ms);

/*
 * lra_oversample_batched -- rectangular generators for every block of a batch
 * that lra_ca_run_batched has processed (paper: Algorithm algrup, greedy
 * expansions of a k x k submatrix to k x l; Theorem th3 for the error bound of
 * k x l generators), one CTA per block from a work queue.  Block b's square
 * generator (rows in->I, columns in->J, size k_b = in->info[6]) grows by up to
 * pextra columns, l_b = min(k_b + pextra, ncols):
 *   X = B^{-1} W'[I, :] (B = W'[I, J]) is the C matrix of a maxvol step on the
 *   row strip warm-started at J with no swaps (its set J0 starts J'; a zero
 *   pivot keeps J' = J and adds nothing); then, pextra times, the column outside
 *   J' with the largest s_j = ||X[:, j]||^2 (lowest j on ties) joins J' (the
 *   squared volume of the generator grows by 1 + s_j) and every other column is
 *   whitened again, X[:, q] -= gamma (x . X[:, q]) x with gamma = (1 - 1/sqrt(1 +
 *   sigma)) / sigma, sigma = s_j; no column is added once the largest s_j is 0.
 * Outputs (out, layout of lra_cur_batch with these slots): I (nb x par->k),
 * J' (nb x (par->k + pextra)), C_b = W'[:, J'] (nrows x l_b) and R_b = W[I, :]
 * (k_b x ncols) packed at batch->offsets (which must size the slots for
 * min(par->k + pextra, ncols) and par->k), U_b (l_b x k_b, row-major) at the
 * start of an (par->k + pextra) x par->k slot: the pinv of the rank-r QRP
 * truncation of W'[I, J'] at par->rank_tol (r = info[0]); info[3] status,
 * info[6] = k_b, info[7] = l_b, info[1] = info[2] = 0.  Blocks whose C-A run
 * failed keep its status.
 * par->k: the C-A run's largest size; par->h: the maxvol threshold.
 * Errors: LRA_ERR_INVALID_ARG (also when the rectangular nucleus of par->k x
 * (par->k + pextra) does not fit in shared memory), LRA_ERR_WORKSPACE,
 * LRA_ERR_CUDA.
 */
lra_status lra_oversample_batched_workspace_size(const lra_problem* base, const lra_batch* batch,
                                                 const lra_ca_params* par, int32_t pextra, size_t* bytes);
lra_status lra_oversample_batched(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                                  int32_t pextra, const lra_cur_batch* in, const lra_cur_batch* out, void* workspace,
                                  size_t workspace_bytes, lra_stream_t stream);

/*
 * lra_oversample_cycle_batched -- lra_oversample_batched followed by the
 * expansion/contraction cycles of Section scrsorth (QRP-based greedy iterative
 * search for locally maximal volume).  After the greedy expansion to l_b:
 *   while the generator fails Corollary colclmx's test of local
 *   par->h-maximality, 1 + max s_q over the columns q outside J' <= par->h,
 *   a p-cycle (p starts at 1) expands J' greedily by p columns and contracts it
 *   greedily by p: the column of J' with the smallest s_j (lowest j on ties;
 *   it must be below 1) leaves, the others keep their order, and X[:, q] +=
 *   gamma' (x . X[:, q]) x for every column with gamma' = (1/sqrt(1 - sigma)
 *   - 1) / sigma (Theorem th2: the squared volume shrinks by 1 - s_j).  The
 *   cycle is kept when it changed the set and the product of its 1 + s and
 *   1 - s factors is above 1 (p restarts at 1); otherwise the state before it
 *   is restored and p grows by one.  The loop ends when the test passes, p
 *   exceeds pmax, or par->max_swaps cycles were kept.
 * Arguments, outputs and errors as lra_oversample_batched, plus: pmax (0..16;
 * 0 = lra_oversample_batched), par->max_swaps >= 0 (largest number of kept
 * cycles).  info[1] = cycles kept, info[2] = largest p tried; info[3] is
 * LRA_WARN_NOT_CONVERGED when the test did not pass (the generator is still
 * valid).  The workspace adds (par->k + 1) x batch->max_len doubles per CTA for
 * the copy of X and s.
 */
lra_status lra_oversample_cycle_batched_workspace_size(const lra_problem* base, const lra_batch* batch,
                                                       const lra_ca_params* par, int32_t pextra, int32_t pmax,
                                                       size_t* bytes);
lra_status lra_oversample_cycle_batched(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                                        int32_t pextra, int32_t pmax, const lra_cur_batch* in,
                                        const lra_cur_batch* out, void* workspace, size_t workspace_bytes,
                                        lra_stream_t stream);

/*
 * lra_prjvol_batched -- k_b x l_b generators of maximal r-projective volume
 * for every block of a batch that lra_ca_run_batched has processed (paper:
 * Algorithm algprjvlm, which turns the search into a volume maximisation in the
 * r x n factor R' of a rank-revealing QR; Algorithm alg1tor for that QR;
 * Theorem coc-avlm for the C-A steps built on it), one CTA per block from a
 * work queue.  For block b with rows I = in->I (k_b = in->info[6] of them) and
 * l_b = min(k_b + pextra, ncols):
 *   1. Algorithm alg1tor on the strip A = W'[I, :] (k_b x ncols): Householder
 *      QR with column pivoting (pivot = the column outside the chosen set with
 *      the largest squared norm of the remaining rows, an ascending fma chain,
 *      lowest index on ties), stopped at the numerical rank r_b: the first step
 *      whose pivot norm is <= par->rank_tol times the first pivot's, or
 *      min(k_b, ncols).  Its first r_b rows are R' (r_b x ncols), the pivots J0;
 *   2. Algorithm algdomin on R' warm-started at J0 (R'[:, J0] is upper
 *      triangular): swaps while some |(R'[:, J])^{-1} R'| > par->h, at most
 *      par->max_swaps of them, in lra_ca_run's maxvol arithmetic;
 *   3. Algorithm algrup's greedy expansions from those r_b columns to l_b,
 *      as in lra_oversample_batched.
 *   A zero strip (r_b = 0) keeps J' = in->J (k_b columns).
 * Outputs (out, layout of lra_oversample_batched): I, J' (l_b entries of an
 * (par->k + pextra) slot), C_b = W'[:, J'], R_b = W[I, :], U_b = pinv of the
 * rank-r QRP truncation of W'[I, J'] at par->rank_tol; info[0] = nucleus rank,
 * info[1] = swaps made on R', info[2] = r_b, info[3] = status
 * (LRA_WARN_NOT_CONVERGED when max_swaps stopped the swaps,
 * LRA_WARN_RANK_DEFICIENT when the nucleus rank is below k_b or r_b = 0,
 * LRA_ERR_NONFINITE for a strip holding NaN or Inf), info[6] = k_b,
 * info[7] = l_b.  Blocks whose C-A run failed keep its status.
 * With par->max_swaps = 0 and pextra = 0, J'[0..r_b) are Algorithm alg1tor's
 * pivots (the status then says whether a swap was wanted).
 * Errors: LRA_ERR_INVALID_ARG (also par->max_swaps < 0, and a rectangular
 * nucleus of par->k x (par->k + pextra) that does not fit in shared memory),
 * LRA_ERR_WORKSPACE, LRA_ERR_CUDA.
 */
lra_status lra_prjvol_batched_workspace_size(const lra_problem* base, const lra_batch* batch,
                                             const lra_ca_params* par, int32_t pextra, size_t* bytes);
lra_status lra_prjvol_batched(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                              int32_t pextra, const lra_cur_batch* in, const lra_cur_batch* out, void* workspace,
                              size_t workspace_bytes, lra_stream_t stream);

/*
 * lra_ca_lev_batched -- C-A iterations whose steps select by DMM08 Algorithm 1
 * on the sketches (paper: the tests of C-A incorporating [DMM08, Algorithm 1],
 * with SVD-based leverage scores, eq. eqlevsc with beta = 1, and the sampling of
 * Algorithms algsmplex / algsmplexp), one CTA per block of the batch.  Per
 * block, from the rows I0 (k of them), iters times:
 *   horizontal: the k_I x n sketch A = W[I, :]; G = A A^T (ascending fma
 *   chains); at most 10 sweeps of round-robin Jacobi rotations (all angles of a
 *   round from G at its start, then the row pairs, then the column pairs and Q;
 *   stop after a sweep that leaves every off-diagonal |G| at most 2^-48 times
 *   the largest diagonal |G|); the
 *   r' = min(r, k_I) largest eigenvalues (lowest index on ties) that are
 *   positive and >= 1e-12 of the largest; scores v_j = sum_t (Q_t . a_j)^2 / d_t;
 *   then l = k columns: kind 0 Exactly(l) -- draw t picks the smallest j with
 *   cum_j > u_t * total (ascending running sums; none: the last j with v_j > 0),
 *   repeats allowed; kind 1 Expected(l) -- j ascending is kept when u_j <
 *   min(1, (l v_j) / total), at most l, none kept: the largest v_j.  No
 *   positive score: the first l indices.
 *   vertical: the same on W[:, J]^T (k_J x m) for the rows.
 *   kind 2 and 3: Exactly(l) and Expected(l) with uniform scores v_j = 1 in
 *   place of the SVD-based ones (the paper's superfast route for perturbed
 *   factor-Gaussian inputs with r << n, whose leverage scores are nearly equal
 *   by the chi-square concentration of Lemma lmchitail): no Gram matrix and no
 *   Jacobi sweeps; r is then unused (but must still be valid).
 * Then U = pinv of the rank-r QRP truncation of W[I, J] (k_I x k_J; of its
 * transpose when k_I > k_J, transposed back), C = W[:, J], R = W[I, :].
 * k: 1..64, <= every block's rows and columns; r: 1..k; iters >= 1; I0: nb x k
 * block-local rows; draws: nb x (2 iters) x batch->max_len uniforms in [0, 1)
 * (step s of block b at (b * 2 iters + s) * max_len; Exactly reads k of them,
 * Expected one per index).  Outputs (lra_cur_batch): I, J (nb x k: the first
 * k_I, k_J used), C_b (nrows x k_J) and R_b (k_I x ncols) at batch->offsets
 * (slots nrows x k and k x ncols), U (nb x k x k, the first k_J x k_I row-major),
 * info: rank, 0, iters, status (LRA_WARN_RANK_DEFICIENT when a sketch had no
 * positive eigenvalue or the rank is below min(k_I, k_J); LRA_ERR_NONFINITE;
 * LRA_ERR_INVALID_ARG for a bad block), 0, 0, k_I, k_J.  logvol is not used.
 * Errors: LRA_ERR_INVALID_ARG, LRA_ERR_WORKSPACE, LRA_ERR_CUDA.
 */
lra_status lra_ca_lev_batched_workspace_size(const lra_problem* base, const lra_batch* batch, int32_t k, int32_t r,
                                             int32_t iters, int32_t kind, size_t* bytes);
lra_status lra_ca_lev_batched(const lra_problem* base, const lra_batch* batch, int32_t k, int32_t r, int32_t iters,
                              int32_t kind, double rank_tol, const int32_t* I0, const double* draws,
                              const lra_cur_batch* out, void* workspace, size_t workspace_bytes,
                              lra_stream_t stream);

/*
 * lra_hmatvec -- y = M x for the kernel matrix M = K(P, P) (n x n, M_ii = 0)
 * held as far blocks with C-A generators plus a dense near field (paper: the
 * FMM's stage (iii), multiplying generators and diagonal blocks by subvectors;
 * section "Application: HSS / FMM").  The far blocks are the interaction-list
 * pairs of every octree level, their generators C_b U_b R_b the outputs of
 * lra_ca_run_batched on them; the near blocks are the touching leaf pairs,
 * whose entries are formed on the fly (the diagonal i = j skipped).
 * Per far block t_b = U_b (R_b x[cols]) (R_b x by a warp per row: lane-strided
 * fma partial sums and a fixed butterfly; U_b t1 by ascending fma chains); per
 * (level, target box) group, row i of the box gets y_lev[i] = sum over the
 * group's blocks in order of sum_a C_b[i][a] t_b[a] (one fma chain); per near
 * group (target leaf) y_near[i] = the sum over its blocks in order, columns j
 * ascending, of w_ij x_j with w_ij = rsqrt(|x_i - x_j|^2) (within an ulp of
 * 1/|x_i - x_j|), in two interleaved accumulators added at the end; finally
 * y = y_near + y_2 + ... + y_L in that order (rows in no group of a level add
 * 0).  The order of every sum is fixed: repeated calls give identical bits.
 * Blocks whose generator run ended in an error contribute nothing.
 * prob: a Laplace kernel problem (X = Y, m = n).  H (device arrays, caller-owned):
 * far (nfar x 4: row0, nrows, col0, ncols), far_offsets (nfar x 2: offsets of
 * C_b and R_b in C and R), C, U (nfar x kmax x kmax, kf_b x kf_b used), R,
 * info (nfar x LRA_INFO_LEN; kf_b = info[6]) -- the batch's outputs;
 * far_groups (ngroups x 5: level (2..levels), row0, nrows, first block,
 * block count; the blocks of a group contiguous); near (nnear x 4), near_groups
 * (nnear_groups x 4: row0, nrows, first block, count).  x, y: n doubles
 * (device).  The workspace holds t (nfar x kmax) and (levels - 1 + 1) partial
 * vectors of n doubles.  Asynchronous on the stream.
 * Matrix-free form (C = R = NULL, I and J the batch's generator rows and
 * columns, a batch run without stored factors): every entry of C_b and R_b is
 * evaluated from prob's points exactly as the batch's gathers evaluated it
 * (FP32 or FP64 entries, as prob's dtype), so y equals the stored form's bit for
 * bit while the device holds only I, J and U (the stored C and R of 2^20
 * uniform points would take about 250 GB).  Cost: the entries are recomputed
 * on every call.
 * Errors: LRA_ERR_INVALID_ARG, LRA_ERR_WORKSPACE, LRA_ERR_CUDA.
 */
typedef struct {
  int64_t n;
  int32_t levels;
  int32_t kmax;
  int32_t nfar, nfar_groups, nnear, nnear_groups;
  const int64_t* far;
  const int64_t* far_offsets;
  const double* C;
  const double* U;
  const double* R;
  const int32_t* info;
  const int64_t* far_groups;
  const int64_t* near;
  const int64_t* near_groups;
  const int32_t* I;        /* nfar x kmax generator rows (block-local): with C = R = NULL */
  const int32_t* J;        /* nfar x kmax generator columns (block-local)                */
} lra_hmatrix;

lra_status lra_hmatvec_workspace_size(const lra_hmatrix* H, size_t* bytes);
lra_status lra_hmatvec(const lra_problem* prob, const lra_hmatrix* H, const double* x, double* y, void* workspace,
                       size_t workspace_bytes, lra_stream_t stream);

/*
 * lra_ca_batched_shapes -- the CTA shapes the batched kernel is built for:
 * writes up to cap (threads per CTA, CTAs per SM) pairs and returns their
 * number.  Each shape holds 16 warps per SM (128 registers a thread); they
 * trade parallelism inside one block for overlap between blocks.
 */
int32_t lra_ca_batched_shapes(int32_t* threads, int32_t* ctas_per_sm, int32_t cap);

/*
 * lra_ca_batched_tune -- autotuner of lra_ca_run_batched (no counterpart in the
 * paper): runs the whole batch reps times in each CTA shape, timing each launch
 * with CUDA events on the stream, and returns the fastest shape in
 * *cta_threads, *ctas_per_sm (store them in lra_batch for later calls) and, if
 * ms is not NULL, the fastest time of every shape (lra_ca_batched_shapes
 * order; -1 for a shape whose shared-memory share cannot hold the batch's
 * largest block at par->k, which is skipped).  Every shape computes the same
 * results, left in out.  Blocks the
 * calling thread until the stream has run the launches; not capturable.
 * Arguments and errors as lra_ca_run_batched; reps >= 1.
 */
lra_status lra_ca_batched_tune(const lra_problem* base, const lra_batch* batch, const lra_ca_params* par,
                               const int32_t* I0, const lra_cur_batch* out, void* workspace, size_t workspace_bytes,
                               lra_stream_t stream, int32_t reps, int32_t* cta_threads, int32_t* ctas_per_sm,
                               float* ms);

/*
 * lra_ca_batched_tune_stages -- autotuner of the staged generator sizes, i.e. of
 * the strip widths the C-A runs of a batch go through (no counterpart in the
 * paper, which fixes no sizes): for each candidate schedule it runs the whole
 * batch reps times, timing each launch with CUDA events on the stream, then
 * samples every block's error with lra_residual_sample_batched on `exact` (the
 * same input with FP64 entries; NULL: base itself) at rows Q and columns S as
 * that call takes them.  A schedule qualifies when every block's status is
 * LRA_OK or a warning and every sampled relative Frobenius error (stats column
 * 4) is <= tol.  *best receives the index of the fastest qualifying schedule,
 * whose results are left in out; ms[i] (optional) the fastest time of schedule
 * i and err[i] (optional) its largest sampled error (NaN if a block failed).
 * schedules: host, nsched rows of 2 + LRA_MAX_STAGES int32 -- nstages,
 * rank_margin, then the ascending sizes, the last equal to par->k; par's own
 * stage fields are ignored.  out must hold C and R; stats: device scratch of
 * nb x 5 doubles.  Blocks the calling thread; not capturable.  Errors: as
 * lra_ca_run_batched and lra_residual_sample_batched; LRA_ERR_INVALID_ARG also
 * when a schedule is malformed (every schedule is checked on the host before
 * the first launch) or none qualifies.
 */
lra_status lra_ca_batched_tune_stages(const lra_problem* base, const lra_problem* exact, const lra_batch* batch,
                                      const lra_ca_params* par, const int32_t* I0, const lra_cur_batch* out,
                                      void* workspace, size_t workspace_bytes, const int32_t* Q, int32_t q,
                                      const int32_t* S, int32_t s, double* stats, double tol,
                                      const int32_t* schedules, int32_t nsched, int32_t reps, lra_stream_t stream,
                                      int32_t* best, float* ms, double* err);

/*
 * lra_residual_sample_batched -- the a-posteriori sample of lra_residual_sample
 * for every block of a batch, in one launch: for block b, rows Q[b*q .. b*q+q)
 * and columns S[b*s .. b*s+s) (block-local, device int32) of W_b - C_b U_b R_b;
 * stats (device, nb x 5) as in lra_residual_sample (NaN for failed blocks, and
 * for blocks with a sample position outside 0 <= Q < nrows, 0 <= S < ncols,
 * which is caught before any entry is read).
 * kmax: the par->k of the batched run.  8 (q k + 2 q s) bytes must fit in
 * shared memory.  Errors: LRA_ERR_INVALID_ARG, LRA_ERR_CUDA.
 */
lra_status lra_residual_sample_batched(const lra_problem* base, const lra_batch* batch, int32_t kmax,
                                       const lra_cur_batch* cur, const int32_t* Q, int32_t q, const int32_t* S,
                                       int32_t s, double* stats, lra_stream_t stream);

/*
 * lra_residual_sample_batched_rect -- the same for rectangular generators (the
 * outputs of lra_oversample_batched): block b's C_b is nrows x l_b, U_b l_b x
 * k_b at the start of an lmax x kmax slot, R_b k_b x ncols, with k_b =
 * info[6] and l_b = info[7].  kmax <= lmax <= 128.
 */
lra_status lra_residual_sample_batched_rect(const lra_problem* base, const lra_batch* batch, int32_t kmax,
                                            int32_t lmax, const lra_cur_batch* cur, const int32_t* Q, int32_t q,
                                            const int32_t* S, int32_t s, double* stats, lra_stream_t stream);

/* ------------------------------------------------------------------------- */
/* Differentiable CUR apply on Gaussian-kernel blocks (fixed pivots)          */
/* ------------------------------------------------------------------------- */
/* nb independent blocks of equal shape: block b has targets X[b] (m x 3) and
 * sources Y[b] (n x 3), kernel K(x, y) = exp(-|x - y|^2 / (2 l^2)), and fixed
 * pivots I[b] (k rows of X[b]) and J[b] (k rows of Y[b]), e.g. from
 * lra_ca_run_batched.  All pointers device. */
typedef struct {
  const double* X;          /* nb x m x 3 */
  const double* Y;          /* nb x n x 3 */
  const int32_t* I;         /* nb x k, block-local */
  const int32_t* J;         /* nb x k, block-local */
  int32_t nb, m, n, k;      /* 1 <= k <= min(m, n, 64) */
  double length_scale;      /* l > 0 */
} lra_gauss_blocks;

/*
 * lra_gauss_cur_forward -- y[b] = C U R x[b] per block (paper: FMM stage (iii)
 * product with the generators; the gradient machinery has no counterpart in the
 * paper), with C = K(X, Y_J), R = K(X_I, Y), U = K(X_I, Y_J)^{-1} (FP64
 * Gauss-Jordan with partial pivoting).  C and R are evaluated on the fly in FP32
 * and never stored; R x is accumulated in FP32, U (R x) in FP64, C (U R x) in
 * FP32.  x: nb x n x nrhs FP32, y: nb x m x nrhs FP32 (1 <= nrhs <= 256).
 * ctx: nb x (k*k + 2*k*nrhs) FP64 written for the backward (U, R x, U R x).
 * A singular core gives NaN outputs for its block.  A pivot outside
 * 0 <= I[b][a] < m or 0 <= J[b][a] < n is caught on the device before any point
 * is read through it: the block's y and ctx are then NaN.  Errors:
 * LRA_ERR_INVALID_ARG, LRA_ERR_CUDA.
 */
lra_status lra_gauss_cur_forward(const lra_gauss_blocks* g, const float* x, int32_t nrhs, float* y, double* ctx,
                                 lra_stream_t stream);

/*
 * lra_gauss_cur_backward -- gradients of a scalar loss through y = C U R x at
 * fixed pivots, given dy = dL/dy (nb x m x nrhs FP32) and the forward's ctx:
 *   dx = R^T U^T C^T dy (nb x n x nrhs FP32);
 *   dell[b] = dL/dl of block b (FP64; the entries of C, R and the core all depend
 *             on l through dK/dl = K |x - y|^2 / l^3);
 *   optional (may be NULL): dC = dy (U R x)^T (nb x m x k), dR = U^T C^T dy x^T
 *   (nb x k x n), dG = -U^T C^T dy (U R x)^T (nb x k x k), the gradients with
 *   respect to the sampled kernel entries (FP32).
 * A block whose pivots are out of range (as in the forward) gets NaN gradients
 * and reads no point through them.  Errors: LRA_ERR_INVALID_ARG, LRA_ERR_CUDA.
 */
lra_status lra_gauss_cur_backward(const lra_gauss_blocks* g, const float* x, const float* dy, int32_t nrhs,
                                  const double* ctx, float* dx, double* dell, float* dC, float* dR, float* dG,
                                  lra_stream_t stream);

/*
 * lra_cur_apply -- Y = C (U (R X)) for one CUR triple (paper: FMM / HSS stage
 * (iii), multiplication with the generators of the neutered block columns).
 * C m x k and R k x n (as written by lra_ca_run, or rounded copies of them),
 * U k x k FP64, X n x nrhs and Y m x nrhs FP64, all device row-major.  dtype is
 * the storage type of C and R:
 *   LRA_F64: every product accumulated in FP64 (1 <= nrhs <= 1024);
 *   LRA_F32 / LRA_BF16 (1 <= nrhs <= 64): C and R streamed at 4 / 2 bytes an
 *     entry (half / a quarter of the FP64 HBM bytes; rows of R 16-byte aligned
 *     take vector loads).  Products in FP32, accumulated in FP32 over runs of at
 *     most 512 terms of R X and k terms of C T2, the runs in FP64; U T1 in FP64.
 *     One refinement step: the FP64 vector operand (X, then T2 = U T1) is split
 *     into an FP32 head and an FP32 tail, and both are multiplied by the same
 *     stored entries, so the result carries only the storage rounding of C and
 *     R (2^-24 or 2^-9 relative per entry) and the FP32 accumulation.
 * Errors: LRA_ERR_INVALID_ARG (sizes, dtype), LRA_ERR_WORKSPACE, LRA_ERR_CUDA.
 */
lra_status lra_cur_apply(const void* C, const double* U, const void* R, int64_t m, int64_t n, int32_t k,
                         const double* X, int32_t nrhs, double* Y, int32_t dtype, void* workspace,
                         size_t workspace_bytes, lra_stream_t stream);
/* Workspace bytes of lra_cur_apply for an n-column R, rank k and nrhs right-hand sides (any dtype). */
lra_status lra_cur_apply_workspace_size(int64_t n, int32_t k, int32_t nrhs, size_t* bytes);

/*
 * lra_residual_sample -- a-posteriori error estimate from a q x s submatrix of
 * E = W - C U R (paper: Section "Superfast a posteriori error estimation for LRA
 * of a matrix filled with i.i.d. values of a single variable").  Q (q device
 * int32 rows) and S (s device int32 columns) are the random sample positions;
 * q*s >= 1.  stats (device, 5 doubles): mean of e, variance (1/K) sum (e-mean)^2,
 * mean |e|, max |e|, ||E[Q,S]||_F / ||W[Q,S]||_F with K = q s.  E (device q x s,
 * optional, may be NULL) receives the sampled errors.  W is read through prob
 * (original matrix, no multiplier).  Every Q[a] must lie in 0 <= Q[a] < m and
 * every S[c] in 0 <= S[c] < n: the device checks each index before it reads
 * through it, and a bad one makes all five statistics NaN (the entry is not
 * read).  Errors: LRA_ERR_INVALID_ARG, LRA_ERR_CUDA.
 */
lra_status lra_residual_sample(const lra_problem* prob, const double* C, const double* U, const double* R,
                               int32_t k, const int32_t* Q, int32_t q, const int32_t* S, int32_t s, double* stats,
                               double* E, void* workspace, size_t workspace_bytes, lra_stream_t stream);
/* Workspace bytes of lra_residual_sample for rank k and a q x s sample. */
lra_status lra_residual_sample_workspace_size(int32_t k, int32_t q, int32_t s, size_t* bytes);

/* ------------------------------------------------------------------------- */
/* Instrumentation (no counterpart in the paper: benchmark support)           */
/* ------------------------------------------------------------------------- */
#define LRA_PROFILE_NAME_LEN 32

/* Number of kernels the library has launched in this process (all devices). */
int64_t lra_launch_count(void);

/* on != 0: bracket every subsequent kernel launch with two CUDA events recorded
 * on the launch's stream (host cost: two event creations per launch).  Do not
 * enable while capturing a CUDA graph.  Never fails. */
lra_status lra_profile_enable(int32_t on);

/* Wait for the events recorded since the last collect and report, per kernel
 * name, the summed elapsed milliseconds and the launch count; the records are
 * then discarded.  names: max_kernels * LRA_PROFILE_NAME_LEN host chars (or
 * NULL), total_ms / launches: max_kernels entries (or NULL).  *n_out receives
 * the number of distinct kernels seen (entries beyond max_kernels are dropped).
 * Errors: LRA_ERR_INVALID_ARG, LRA_ERR_CUDA (an event failed). */
lra_status lra_profile_collect(int32_t max_kernels, char* names, double* total_ms, int64_t* launches,
                               int32_t* n_out);

/* Library version string, for diagnostics. */
const char* lra_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LRA_H */
