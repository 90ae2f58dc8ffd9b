// lra_batched_kernel.cuh -- the persistent C-A kernel over a batch of blocks.
//
// Each CTA takes blocks from a device work queue (one atomic counter; the
// caller's processing order, largest blocks first for a balanced tail) and
// runs the whole C-A loop of a block, then its nucleus, on its own: the block's
// strips sit in the CTA's shared memory when they fit, otherwise in the CTA's
// slice of a global scratch area.  The per-block arithmetic is the single-CTA
// path of lra_ca_run, operation for operation.  Optionally the first blocks
// of the order run first, each on a pair of CTAs that split its strips and
// meet through the grid exchange of lra_ca_run (a separate instantiation,
// launched cooperatively).  The kernel is built in one translation unit per
// CTA shape (lra_batched_k*.cu).
#pragma once

#include "lra_ca_loop.cuh"
#include "lra_nucleus.cuh"

namespace lra {

struct BatchArgs {
  DevProblem base;
  const int64_t* blocks;    // nb x 4: row0, nrows, col0, ncols
  const int64_t* offs;      // nb x 2: offsets (in doubles) of C_b and R_b
  const int32_t* order;     // processing order (nb) or null
  int32_t nb, kmax, sweeps, max_swaps;
  double h, rank_tol;
  const int32_t* I0;        // nb x kmax initial rows (block-local)
  int32_t* I;               // nb x kmax
  int32_t* J;               // nb x kmax
  double* C;                // packed
  double* R;                // packed
  double* U;                // nb x kmax x kmax (k_b x k_b at the start of each slot)
  double* logvol;           // nb x 2 sweeps
  int32_t* info;            // nb x LRA_INFO_LEN
  double* work;             // nb: algorithmic flops of each block's run, or null
  unsigned int* counter;    // work queue head
  double* scratch;          // per CTA: G (kmax^2) then, if needed, a strip (kmax x max_len)
  size_t scratch_stride;    // doubles per CTA
  size_t smem_bytes;        // dynamic shared memory per CTA: a stage's strip is kept
                            // there when it fits with the fixed part
  int64_t max_len;          // largest block dimension the scratch was sized for
  int32_t mixed;
  int32_t nstages, margin;  // staged generator sizes (0: one run of size k_b)
  int32_t stages[LRA_MAX_STAGES];
  int32_t nteam;            // the first nteam entries of the order are each run by a pair of CTAs (0: none)
  double* tslots;           // per pair: [2][2][SLOT] exchange slots (zeroed before the launch)
  unsigned int* tabort;     // per pair: its abort word (zeroed before the launch)
};

// A round of the group's exchange with no candidate: the CTAs of a pair then
// see each other's earlier global writes (the lead's G, I, J and status).  A
// single CTA has nothing to wait for.
__device__ __forceinline__ void group_sync(const SoloGroup&, const CaSmem&, unsigned long long*, int) {}
__device__ __forceinline__ void group_sync(const GridGroup& g, const CaSmem& S, unsigned long long* seq, int k) {
  __threadfence();
  g.exchange<true>(*seq, cand_none(), 0ull, S.M, 1, 0, k, 1, S.xo);
  ++*seq;
}

// One block of the batch by a group of CTAs (one CTA, or a pair that splits the
// strips' columns between them): every stage's C-A run and nucleus, then the
// outputs.  Each CTA of a pair runs the nucleus on the lead's core G (only the
// lead writes U: Uown takes the other's copy), so that both take the same
// stage decisions; the lead writes the block's statistics.
template <class Group, bool MIXED, int NPARTS>
__device__ __forceinline__ void run_block(const Group& grp, const BatchArgs& B, int b, double* G, double* gstrip,
                          double* Uown, unsigned char* smem, int32_t* s_I0, double& s_work,
                          unsigned long long* seq) {
  const int rk = grp.rank();
  const bool lead = rk == 0;
  int32_t* info = B.info + LRA_INFO_LEN * (size_t)b;
  const int64_t r0 = B.blocks[4 * (size_t)b], nr = B.blocks[4 * (size_t)b + 1];
  const int64_t c0 = B.blocks[4 * (size_t)b + 2], nc = B.blocks[4 * (size_t)b + 3];
  if (r0 < 0 || c0 < 0 || nr < 1 || nc < 1 || r0 + nr > B.base.m || c0 + nc > B.base.n || nr > B.max_len ||
      nc > B.max_len) {
    if (lead)
      for (int e = threadIdx.x; e < LRA_INFO_LEN; e += blockDim.x) info[e] = (e == 3) ? LRA_ERR_INVALID_ARG : 0;
    return;
  }
  CaArgs A;
  memset(&A, 0, sizeof(A));
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
  const int kb = (int)min((int64_t)B.kmax, min(nr, nc));
  A.sweeps = B.sweeps;
  A.max_swaps = B.max_swaps;
  A.h = B.h;
  A.I0 = B.I0 + (size_t)b * B.kmax;
  A.I = B.I + (size_t)b * B.kmax;
  A.J = B.J + (size_t)b * B.kmax;
  // the factors are written once, after the last stage (null: not stored)
  double* const Cb = B.C ? B.C + B.offs[2 * (size_t)b] : nullptr;
  double* const Rb = B.R ? B.R + B.offs[2 * (size_t)b + 1] : nullptr;
  A.C = nullptr;
  A.R = nullptr;
  A.logvol = B.logvol + (size_t)b * 2 * B.sweeps;
  A.info = info;
  A.G = G;
  A.chunk_n = (int)((nc + NPARTS - 1) / NPARTS);
  A.chunk_m = (int)((nr + NPARTS - 1) / NPARTS);
  A.ldm = max(A.chunk_n, A.chunk_m);
  A.mixed = B.mixed;
  A.seq = seq;
  if (threadIdx.x == 0) s_work = 0.0;
  A.work = B.work ? &s_work : nullptr;
  // without a multiplier the row steps' strips are C itself (each CTA its rows):
  // the last one stays as the output
  A.Cstrip = (Cb != nullptr && A.P.mkind == LRA_MULT_NONE) ? Cb : nullptr;
  if (B.mixed && A.P.src == LRA_KERNEL_LAPLACE) {
    A.P.X32 = B.base.X32 + 3 * r0;
    A.P.Y32 = B.base.Y32 + 3 * c0;
  }
  // Generator sizes: the caller's stages clipped to kb (one run of size kb
  // without stages).  Each stage is a complete C-A run and nucleus; the next
  // stage starts from this stage's rows, then the block's unused initial rows.
  const int32_t* I0b = B.I0 + (size_t)b * B.kmax;
  int stage = 0, k = B.nstages > 0 ? min(B.stages[0], kb) : kb;
  int swaps = 0, loops = 0, n32 = 0, n64 = 0, nrun = 0, r = 0, st = LRA_OK;
  for (;;) {
    A.k = k;
    A.I0 = (nrun == 0) ? I0b : s_I0;
    A.strip_in_smem = ca_smem_fixed(k, A.ldm, MIXED) + sizeof(double) * (size_t)k * A.ldm <= B.smem_bytes;
    A.gstrip = A.strip_in_smem ? nullptr : gstrip;
    const CaSmem S = ca_smem_carve(smem, k, A.ldm, A.gstrip, MIXED);
    ca_loop<Group, MIXED>(grp, A, S);
    __syncthreads();
    group_sync(grp, S, seq, k);
    ++nrun;
    st = info[3];
    swaps += info[1]; loops += info[2]; n32 += info[4]; n64 += info[5];
    if (st != LRA_OK && st < 16) break;
    // a stage whose rank sends the block on to a larger size needs only the rank
    int knext = k;
    for (int sx = stage; sx + 1 < B.nstages && knext <= k;) knext = min(B.stages[++sx], kb);
    const int rank_only = (k < kb && knext > k) ? k - B.margin : KMAX + 1;
    double* const Ub = lead ? B.U + (size_t)b * B.kmax * B.kmax : Uown;
    r = nucleus_cta(G, k, B.rank_tol, Ub, smem, max(rank_only, 0));
    if (threadIdx.x == 0) s_work += 5.0 * k * k * k;          // the nucleus, nominal
    if (r < k && st == LRA_OK) st = LRA_WARN_RANK_DEFICIENT;
    if (k >= kb || r < k - B.margin) break;
    int kn = k;
    while (stage + 1 < B.nstages && kn <= k) kn = min(B.stages[++stage], kb);
    if (kn <= k) break;
    if (threadIdx.x == 0) {           // next initial rows: I, then unused I0b rows in order
      for (int a = 0; a < k; ++a) s_I0[a] = A.I[a];
      int c = k;
      for (int t = 0; t < kb && c < kn; ++t) {
        const int32_t v = I0b[t];
        bool in = false;
        for (int a = 0; a < k; ++a) in |= (s_I0[a] == v);
        if (!in) s_I0[c++] = v;
      }
    }
    __syncthreads();
    k = kn;
  }
  __syncthreads();
  if (Cb != nullptr && Rb != nullptr && !(st != LRA_OK && st < 16)) {
    // C_b = W'[:, J] (nr x k) and R_b = W[I, :] (k x nc) at the final size, from
    // the final I, J that the last C-A run stored; each CTA its rows of C and
    // columns of R
    const int64_t cr0 = (int64_t)rk * A.chunk_m, cc0 = (int64_t)rk * A.chunk_n;
    const int rn = (int)max((int64_t)0, min((int64_t)A.chunk_m, nr - cr0));
    const int cn = (int)max((int64_t)0, min((int64_t)A.chunk_n, nc - cc0));
    if (A.Cstrip == nullptr)
      for (int it = threadIdx.x; it < rn * k; it += blockDim.x) {
        const int c = it / k, a = it - c * k;
        Cb[(cr0 + c) * k + a] = c_entry(A.P, cr0 + c, A.J[a]);
      }
    for (int it = threadIdx.x; it < k * cn; it += blockDim.x) {
      const int a = it / cn, c = it - a * cn;
      Rb[(int64_t)a * nc + cc0 + c] = r_entry(A.P, A.I[a], cc0 + c);
    }
  }
  if (lead && threadIdx.x == 0) {
    info[0] = (st != LRA_OK && st < 16) ? 0 : r;
    info[1] = swaps; info[2] = loops; info[3] = st;
    info[4] = n32; info[5] = n64; info[6] = k; info[7] = k;
    if (B.work) B.work[b] = s_work;
  }
  __syncthreads();
}

// A pair's block, out of line: the single-CTA path keeps the kernel's registers.
static __device__ __noinline__ void run_pair_block(const GridGroup& grp, const BatchArgs& B, int b, double* G,
                                                   double* gstrip, double* Uown, unsigned char* smem,
                                                   int32_t* s_I0, double& s_work, unsigned long long* seq) {
  run_block<GridGroup, false, 2>(grp, B, b, G, gstrip, Uown, smem, s_I0, s_work, seq);
}

// NTB threads per CTA, MINB CTAs per SM (NTB * MINB = 512: 128 registers a thread).
// PAIRS: the first B.nteam blocks of the order go to CTA pairs (2t, 2t + 1), pair
// t taking blocks t, t + pairs, ... (a separate instantiation, so that the
// single-CTA path keeps its registers); then every CTA takes the remaining
// blocks from the work queue on its own.
template <bool MIXED, int NTB, int MINB, bool PAIRS = false>
__global__ void __launch_bounds__(NTB, MINB) ca_batched_kernel(BatchArgs B) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_b;
  __shared__ int32_t s_I0[KMAX];
  __shared__ double s_work;
  double* const G = B.scratch + (size_t)blockIdx.x * B.scratch_stride;
  double* const gstrip = G + (size_t)B.kmax * B.kmax;
  if constexpr (PAIRS && !MIXED) {
    const int pairs = (int)(gridDim.x >> 1), t = (int)(blockIdx.x >> 1);
    if (B.nteam > 0 && t < pairs) {
      unsigned long long seq = 0;         // the pair's exchange rounds (the same count in both CTAs)
      GridGroup grp{B.tslots + (size_t)t * 4 * SLOT, B.tabort + t, 2, 2 * t};
      double* const Glead = B.scratch + (size_t)(2 * t) * B.scratch_stride;
      for (int q = t; q < B.nteam; q += pairs) {
        const int b = B.order ? B.order[q] : q;
        run_pair_block(grp, B, b, Glead, gstrip, G, smem, s_I0, s_work, &seq);
      }
    }
  }
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned int q = atomicAdd(B.counter, 1u) + (unsigned)B.nteam;
      s_b = (q < (unsigned)B.nb) ? (B.order ? B.order[q] : (int)q) : -1;
    }
    __syncthreads();
    const int b = s_b;
    __syncthreads();
    if (b < 0) break;
    int32_t* info = B.info + LRA_INFO_LEN * (size_t)b;
    const int64_t r0 = B.blocks[4 * (size_t)b], nr = B.blocks[4 * (size_t)b + 1];
    const int64_t c0 = B.blocks[4 * (size_t)b + 2], nc = B.blocks[4 * (size_t)b + 3];
    if (r0 < 0 || c0 < 0 || nr < 1 || nc < 1 || r0 + nr > B.base.m || c0 + nc > B.base.n || nr > B.max_len ||
        nc > B.max_len) {
      for (int e = threadIdx.x; e < LRA_INFO_LEN; e += blockDim.x) info[e] = (e == 3) ? LRA_ERR_INVALID_ARG : 0;
      continue;
    }
    CaArgs A;
    memset(&A, 0, sizeof(A));
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
    const int kb = (int)min((int64_t)B.kmax, min(nr, nc));
    A.sweeps = B.sweeps;
    A.max_swaps = B.max_swaps;
    A.h = B.h;
    A.I0 = B.I0 + (size_t)b * B.kmax;
    A.I = B.I + (size_t)b * B.kmax;
    A.J = B.J + (size_t)b * B.kmax;
    // the factors are written once, after the last stage (null: not stored)
    double* const Cb = B.C ? B.C + B.offs[2 * (size_t)b] : nullptr;
    double* const Rb = B.R ? B.R + B.offs[2 * (size_t)b + 1] : nullptr;
    A.C = nullptr;
    A.R = nullptr;
    A.logvol = B.logvol + (size_t)b * 2 * B.sweeps;
    A.info = info;
    A.G = G;
    A.chunk_n = (int)nc;
    A.chunk_m = (int)nr;
    A.ldm = (int)max(nr, nc);
    A.mixed = B.mixed;
    if (threadIdx.x == 0) s_work = 0.0;
    A.work = B.work ? &s_work : nullptr;
    // without a multiplier the row steps' strips are C itself: the last one stays as the output
    A.Cstrip = (Cb != nullptr && A.P.mkind == LRA_MULT_NONE) ? Cb : nullptr;
    if (B.mixed && A.P.src == LRA_KERNEL_LAPLACE) {
      A.P.X32 = B.base.X32 + 3 * r0;
      A.P.Y32 = B.base.Y32 + 3 * c0;
    }
    // Generator sizes: the caller's stages clipped to kb (one run of size kb
    // without stages).  Each stage is a complete C-A run and nucleus; the next
    // stage starts from this stage's rows, then the block's unused initial rows.
    const int32_t* I0b = B.I0 + (size_t)b * B.kmax;
    int stage = 0, k = B.nstages > 0 ? min(B.stages[0], kb) : kb;
    int swaps = 0, loops = 0, n32 = 0, n64 = 0, nrun = 0, r = 0, st = LRA_OK;
    for (;;) {
      A.k = k;
      A.I0 = (nrun == 0) ? I0b : s_I0;
      A.strip_in_smem = ca_smem_fixed(k, A.ldm, MIXED) + sizeof(double) * (size_t)k * A.ldm <= B.smem_bytes;
      A.gstrip = A.strip_in_smem ? nullptr : gstrip;
      const CaSmem S = ca_smem_carve(smem, k, A.ldm, A.gstrip, MIXED);
      ca_loop<SoloGroup, MIXED>(SoloGroup{}, A, S);
      __syncthreads();
      ++nrun;
      st = info[3];
      swaps += info[1]; loops += info[2]; n32 += info[4]; n64 += info[5];
      if (st != LRA_OK && st < 16) break;
      // a stage whose rank sends the block on to a larger size needs only the rank
      int knext = k;
      for (int sx = stage; sx + 1 < B.nstages && knext <= k;) knext = min(B.stages[++sx], kb);
      const int rank_only = (k < kb && knext > k) ? k - B.margin : KMAX + 1;
      r = nucleus_cta(G, k, B.rank_tol, B.U + (size_t)b * B.kmax * B.kmax, smem, max(rank_only, 0));
      if (threadIdx.x == 0) s_work += 5.0 * k * k * k;          // the nucleus, nominal
      if (r < k && st == LRA_OK) st = LRA_WARN_RANK_DEFICIENT;
      if (k >= kb || r < k - B.margin) break;
      int kn = k;
      while (stage + 1 < B.nstages && kn <= k) kn = min(B.stages[++stage], kb);
      if (kn <= k) break;
      if (threadIdx.x == 0) {           // next initial rows: I, then unused I0b rows in order
        for (int a = 0; a < k; ++a) s_I0[a] = A.I[a];
        int c = k;
        for (int t = 0; t < kb && c < kn; ++t) {
          const int32_t v = I0b[t];
          bool in = false;
          for (int a = 0; a < k; ++a) in |= (s_I0[a] == v);
          if (!in) s_I0[c++] = v;
        }
      }
      __syncthreads();
      k = kn;
    }
    __syncthreads();
    if (Cb != nullptr && Rb != nullptr && !(st != LRA_OK && st < 16)) {
      // C_b = W'[:, J] (nr x k) and R_b = W[I, :] (k x nc) at the final size, from
      // the final I, J that the last C-A run stored
      if (A.Cstrip == nullptr)
        for (int it = threadIdx.x; it < (int)nr * k; it += blockDim.x) {
          const int c = it / k, a = it - c * k;
          Cb[(int64_t)c * k + a] = c_entry(A.P, c, A.J[a]);
        }
      for (int it = threadIdx.x; it < k * (int)nc; it += blockDim.x) {
        const int a = it / (int)nc, c = it - a * (int)nc;
        Rb[(int64_t)a * nc + c] = r_entry(A.P, A.I[a], c);
      }
    }
    if (threadIdx.x == 0) {
      info[0] = (st != LRA_OK && st < 16) ? 0 : r;
      info[1] = swaps; info[2] = loops; info[3] = st;
      info[4] = n32; info[5] = n64; info[6] = k; info[7] = k;
      if (B.work) B.work[b] = s_work;
    }
    __syncthreads();
  }
}

// Kernel entry of one CTA shape (defined in lra_batched_k<threads>.cu).
void* batched_kernel_512(bool mixed, bool pairs);
void* batched_kernel_256(bool mixed, bool pairs);
void* batched_kernel_128(bool mixed);
void* batched_kernel_64(bool mixed);

}  // namespace lra
