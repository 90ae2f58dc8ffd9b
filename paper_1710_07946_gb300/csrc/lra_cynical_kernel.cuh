// lra_cynical_kernel.cuh -- the cynical CUR kernel over a batch of blocks (the
// tests' Tests 3 and Tests 4), built in one translation unit per CTA shape
// (lra_cynical_k*.cu); launch plan and entry points in lra_cynical.cu.
//
// A block's r x r generator is taken inside a q x q sketch W[K, L] (q = 4r in
// the paper): Tests 3 uses the caller's random K and L; Tests 4 makes the
// sketch with one C-A loop of q x q generators from the caller's random L (a
// cold maxvol step on the column strip W[:, L] picks K, one on the row strip
// W[K, :] picks L).  A C-A run of size r on the sketch, held as a small dense
// matrix, then picks I', J' and the nucleus of W[K[I'], L[J']]; the outputs are
// C = W[:, J], U, R = W[I, :] with I = K[I'], J = L[J'].  Every step is the
// single-CTA arithmetic of the C-A kernels, operation for operation.
#pragma once

#include <cstring>

#include "lra_ca_loop.cuh"
#include "lra_nucleus.cuh"

namespace lra {

struct CynArgs {
  DevProblem base;
  const int64_t* blocks;    // nb x 4: row0, nrows, col0, ncols
  const int64_t* offs;      // nb x 2: offsets (in doubles) of C_b and R_b
  const int32_t* order;
  int32_t nb, kind, r, q, sweeps, max_swaps;
  double h, rank_tol;
  int32_t* K;               // nb x q (in; out for Tests 4)
  int32_t* L;               // nb x q (in; out for Tests 4)
  const int32_t* I0s;       // nb x r initial rows of the sketch C-A (in [0, q))
  int32_t* I;               // nb x r
  int32_t* J;               // nb x r
  double* C;                // packed
  double* R;                // packed
  double* U;                // nb x r x r
  double* logvol;           // nb x 2 sweeps
  int32_t* info;            // nb x LRA_INFO_LEN
  unsigned int* counter;    // work queue head
  double* scratch;          // per CTA: see cyn_scratch_doubles
  size_t scratch_stride;    // doubles per CTA
  size_t smem_bytes;
  int64_t max_len;
};

// Per-CTA scratch: sketch (q^2), sketch C (q r), sketch R (r q), core G (r^2),
// then, when the q x len strips of Tests 4 do not fit in shared memory, a strip.
__host__ __device__ inline size_t cyn_fixed_doubles(int r, int q) {
  return (size_t)q * q + 2 * (size_t)q * r + (size_t)r * r;
}

// NTB threads per CTA, MINB CTAs per SM (NTB * MINB = 512: 128 registers a thread).
template <int NTB, int MINB>
__global__ void __launch_bounds__(NTB, MINB) cynical_batched_kernel(CynArgs B) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_b;
  double* sk = B.scratch + (size_t)blockIdx.x * B.scratch_stride;   // q x q sketch
  double* skC = sk + (size_t)B.q * B.q;                              // q x r
  double* skR = skC + (size_t)B.q * B.r;                             // r x q
  double* G = skR + (size_t)B.r * B.q;                               // r x r
  double* gstrip = G + (size_t)B.r * B.r;                            // q x max_len
  const int q = B.q, r = B.r, tid = threadIdx.x, nt = blockDim.x;
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
    int32_t* Kb = B.K + (size_t)b * q;
    int32_t* Lb = B.L + (size_t)b * q;
    const int32_t* I0b = B.I0s + (size_t)b * r;
    // validation (identical in every thread): block inside the input, sketch
    // sets distinct and in range, sketch initial rows distinct in [0, q)
    bool bad = r0 < 0 || c0 < 0 || nr < q || nc < q || r0 + nr > B.base.m || c0 + nc > B.base.n ||
               nr > B.max_len || nc > B.max_len;
    if (!bad && tid == 0) {
      int v = 0;
      for (int a = 0; a < q && !v; ++a) {
        if (B.kind == 0 && (Kb[a] < 0 || Kb[a] >= nr)) v = 1;
        if (Lb[a] < 0 || Lb[a] >= nc) v = 1;
        for (int c = 0; c < a && !v; ++c) v = (B.kind == 0 && Kb[c] == Kb[a]) || Lb[c] == Lb[a];
      }
      for (int a = 0; a < r && !v; ++a) {
        if (I0b[a] < 0 || I0b[a] >= q) v = 1;
        for (int c = 0; c < a && !v; ++c) v = I0b[c] == I0b[a];
      }
      s_b = v;
    }
    __syncthreads();
    if (!bad) bad = s_b != 0;
    __syncthreads();
    if (bad) {
      for (int e = tid; e < LRA_INFO_LEN; e += nt) info[e] = (e == 3) ? LRA_ERR_INVALID_ARG : 0;
      continue;
    }
    // the block as a problem of its own
    CaArgs A;
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
    A.k = q;
    A.sweeps = B.sweeps;
    A.max_swaps = B.max_swaps;
    A.h = B.h;
    A.chunk_n = (int)nc;
    A.chunk_m = (int)nr;
    A.ldm = (int)max(nr, nc);
    A.mixed = 0;
    int swaps = 0, st = LRA_OK;
    if (B.kind == 1) {
      // one C-A loop with q x q generators: rows of W[:, L], then columns of W[K, :]
      A.strip_in_smem = ca_smem_fixed(q, A.ldm) + sizeof(double) * (size_t)q * A.ldm <= B.smem_bytes;
      A.gstrip = A.strip_in_smem ? nullptr : gstrip;
      const CaSmem S = ca_smem_carve(smem, q, A.ldm, A.gstrip);
      for (int a = tid; a < q; a += nt) S.Js[a] = Lb[a];
      __syncthreads();
      unsigned long long seq = 0;
      const StepResult s1 = maxvol_step(SoloGroup{}, A, S, 1, true, S.Is, seq, true);
      __syncthreads();
      StepResult s2{LRA_OK, 0, 0.0};
      if (!(s1.status != LRA_OK && s1.status < 16)) {
        s2 = maxvol_step(SoloGroup{}, A, S, 0, true, S.Js, seq, true);
        __syncthreads();
      }
      swaps = s1.nswaps + s2.nswaps;
      st = max(s1.status, s2.status);
      if (s1.status != LRA_OK && s1.status < 16) st = s1.status;
      else if (s2.status != LRA_OK && s2.status < 16) st = s2.status;
      for (int a = tid; a < q; a += nt) { Kb[a] = S.Is[a]; Lb[a] = S.Js[a]; }
      __syncthreads();
      if (st != LRA_OK && st < 16) {
        if (tid == 0) {
          info[0] = 0; info[1] = swaps; info[2] = 0; info[3] = st;
          info[4] = 0; info[5] = 2; info[6] = r; info[7] = r;
        }
        __syncthreads();
        continue;
      }
    }
    // the q x q sketch W'[K, L], dense, in the CTA's scratch
    for (int it = tid; it < q * q; it += nt) {
      const int a = it / q, c = it - a * q;
      sk[it] = wp_entry(A.P, Kb[a], Lb[c]);
    }
    __syncthreads();
    // C-A of size r on the sketch (its nucleus is the block's: S[I', J'] = W'[I, J])
    CaArgs A2;
    std::memset(&A2, 0, sizeof(A2));
    A2.P.src = LRA_DENSE;
    A2.P.dtype = LRA_F64;
    A2.P.m = q;
    A2.P.n = q;
    A2.P.ldw = q;
    A2.P.W = sk;
    A2.P.mkind = LRA_MULT_NONE;
    A2.k = r;
    A2.sweeps = B.sweeps;
    A2.max_swaps = B.max_swaps;
    A2.h = B.h;
    A2.I0 = I0b;
    A2.I = B.I + (size_t)b * r;
    A2.J = B.J + (size_t)b * r;
    A2.C = skC;
    A2.R = skR;
    A2.G = G;
    A2.logvol = B.logvol + (size_t)b * 2 * B.sweeps;
    A2.info = info;
    A2.chunk_n = q;
    A2.chunk_m = q;
    A2.ldm = q;
    A2.strip_in_smem = 1;
    A2.gstrip = nullptr;
    A2.mixed = 0;
    {
      const CaSmem S2 = ca_smem_carve(smem, r, q, nullptr);
      ca_loop<SoloGroup, false>(SoloGroup{}, A2, S2);
    }
    __syncthreads();
    const int st2 = info[3];
    const int swaps2 = info[1], loops2 = info[2];
    __syncthreads();
    if (st2 != LRA_OK && st2 < 16) {
      if (tid == 0) {
        info[0] = 0; info[1] = swaps + swaps2; info[2] = loops2; info[3] = st2;
        info[4] = 0; info[6] = r; info[7] = r;
      }
      __syncthreads();
      continue;
    }
    const int rank = nucleus_cta(G, r, B.rank_tol, B.U + (size_t)b * r * r, smem);
    // generators in the block's indices, and the block outputs C = W'[:, J], R = W[I, :]
    int32_t* Ib = B.I + (size_t)b * r;
    int32_t* Jb = B.J + (size_t)b * r;
    for (int a = tid; a < r; a += nt) { Ib[a] = Kb[Ib[a]]; Jb[a] = Lb[Jb[a]]; }
    __syncthreads();
    double* Cb = B.C + B.offs[2 * (size_t)b];
    double* Rb = B.R + B.offs[2 * (size_t)b + 1];
    for (int64_t it = tid; it < nr * r; it += nt) {
      const int64_t i = it / r;
      const int a = (int)(it - i * r);
      Cb[it] = c_entry(A.P, i, Jb[a]);
    }
    for (int64_t it = tid; it < (int64_t)r * nc; it += nt) {
      const int a = (int)(it / nc);
      const int64_t c = it - (int64_t)a * nc;
      Rb[it] = r_entry(A.P, Ib[a], c);
    }
    if (tid == 0) {
      int s = max(st, st2);
      if (rank < r && s == LRA_OK) s = LRA_WARN_RANK_DEFICIENT;
      info[0] = rank; info[1] = swaps + swaps2; info[2] = loops2; info[3] = s;
      info[4] = 0; info[5] = (B.kind == 1 ? 2 : 0) + info[5]; info[6] = r; info[7] = r;
    }
    __syncthreads();
  }
}

// Kernel entry of one CTA shape (defined in lra_cynical_k<threads>.cu).
const void* cynical_kernel_512();
const void* cynical_kernel_256();
const void* cynical_kernel_128();
const void* cynical_kernel_64();

}  // namespace lra
