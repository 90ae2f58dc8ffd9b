// lra_mixed.cuh -- the maxvol step in FP32 with certified decisions.
//
// GB300's FP64 pipe is 1/62 of its FP32 rate.  A maxvol step (Algorithm alggos
// initialisation + Algorithm algdomin swaps) is a sequence of discrete
// decisions -- which column (cold LUP), which row (warm LU), which entry to swap
// in, when to stop -- taken on FP64 values.  Here the step runs in FP32, and every
// entry carries a rigorous bound e on its distance to the exact value of the
// same formula (real arithmetic on the FP64 inputs).  A decision is accepted
// only when the bounds certify it:
//   argmax: the winner's lower bound |v| - e exceeds every other entry's upper
//           bound |v| + e (so the exact argmax, ties included, is the same entry);
//   stop:   every upper bound is <= h;  swap: the winner's lower bound is > h;
//   zero pivot: all values and bounds are exactly 0.
// The FP64 reference differs from the exact value by its own rounding, which has
// the same first-order structure with a 2^29 times smaller unit roundoff; the
// bounds are inflated by 1 + 2^-16 to cover it.  If any decision of the step is
// not certified, or anything overflows, the step reports a fallback and the
// caller redoes it in FP64 -- so the index sets, swap counts and everything
// computed from them equal those of the FP64 path, whichever way a step ran.
//
// Bound rules (u = 2^-24, all bound arithmetic rounded upward):
//   a' = fma(-l, a_t, a_p):   e' = e_p + |l| e_t + e_l (|a_t| + e_t) + u |a'|
//   q = n * RN(1/d):          e_q = 2.0001 u |q| + ((1 + 3u)|q| e_d + e_n) / (|d| - e_d)
// Entries: FP64 input rounded to FP32 (u |v|), FP32 input (exact), sums of
// multiplier terms (u per addition), Laplace 1/|x - y| from FP32 points with a
// correctly rounded reciprocal square root.
#pragma once

#include "lra_ca_core.cuh"

namespace lra {

constexpr float kU = 5.9604644775390625e-08f;      // 2^-24
constexpr float kTiny = 1.17549435e-38f;           // FLT_MIN: covers gradual underflow
constexpr float kCert = 1.0000153f;                // 1 + 2^-16

struct V32 {
  float v, e;
};

__device__ __forceinline__ float quot_bound(float q, float en, float d, float ed) {
  const float aq = fabsf(q);
  const float den = __fsub_rd(fabsf(d), ed);
  const float num = __fmaf_ru(__fmul_ru(aq, 1.00000036f), ed, en);
  return __fadd_ru(__fadd_ru(__fmul_ru(2.0001f * kU, aq), __fdiv_ru(num, den)), kTiny);
}

__device__ __forceinline__ float elim_bound(float anew, float l, float el, float at, float et, float ep) {
  float e = __fmaf_ru(fabsf(l), et, ep);
  e = __fmaf_ru(el, __fadd_ru(fabsf(at), et), e);
  return __fmaf_ru(kU, fabsf(anew), __fadd_ru(e, kTiny));
}

__device__ __forceinline__ V32 bad32() {
  const float nan = __int_as_float(0x7fc00000);
  return V32{nan, nan};
}

// w_ij in FP32 with its bound (dense inputs and the Laplace kernel).
__device__ __forceinline__ V32 w_entry32(const DevProblem& P, int64_t i, int64_t j) {
  if (P.src == LRA_DENSE) {
    if (P.dtype == LRA_F32) return V32{__ldg(static_cast<const float*>(P.W) + i * P.ldw + j), 0.f};
    const float v = __double2float_rn(__ldg(static_cast<const double*>(P.W) + i * P.ldw + j));
    return V32{v, __fmaf_ru(kU, fabsf(v), kTiny)};
  }
  const float* x = P.X32 + 3 * i;
  const float* y = P.Y32 + 3 * j;
  float d[3], ed[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float xc = __ldg(x + c), yc = __ldg(y + c);
    d[c] = __fsub_rn(xc, yc);
    // rounding of x and y to FP32 (points are FP64) and of the subtraction
    ed[c] = __fmaf_ru(kU, __fadd_ru(__fadd_ru(fabsf(xc), fabsf(yc)), fabsf(d[c])), kTiny);
  }
  const float p1 = __fmul_rn(d[0], d[0]);
  const float p2 = __fmaf_rn(d[1], d[1], p1);
  const float r2 = __fmaf_rn(d[2], d[2], p2);
  float er = __fmul_ru(kU, __fadd_ru(__fadd_ru(p1, p2), r2));
#pragma unroll
  for (int c = 0; c < 3; ++c) er = __fmaf_ru(ed[c], __fmaf_ru(2.f, fabsf(d[c]), ed[c]), er);
  er = __fadd_ru(er, kTiny);
  if (!(er <= 0.0625f * r2)) return bad32();
  const float yv = __frsqrt_rn(r2);
  const float eps = __fdiv_ru(er, r2);
  // |y - 1/sqrt(r2)| <= u y (1+u); |1/sqrt(r2) - 1/sqrt(r2*)| <= er/2 (r2 - er)^{-3/2}
  //                                                          <= er/2 y^3 (1 + 2.5 eps) (1 + 1e-6)
  const float y3 = __fmul_ru(__fmul_ru(yv, yv), yv);
  float ey = __fmul_ru(__fmul_ru(0.5f * 1.000001f, er), __fmul_ru(y3, __fmaf_ru(2.5f, eps, 1.f)));
  ey = __fmaf_ru(1.0000002f * kU, yv, ey);
  return V32{yv, __fadd_ru(ey, kTiny)};
}

__device__ __forceinline__ V32 wp_entry32(const DevProblem& P, int64_t i, int64_t j) {
  if (P.mkind == LRA_MULT_NONE) return w_entry32(P, i, j);
  float acc = 0.f, ea = 0.f;
  if (P.mkind == LRA_MULT_ARHT) {
    const int64_t pj = __ldg(P.perm + j);
    const int64_t b = pj / P.s, t = pj - b * P.s;
    const int nt = 1 << P.depth;
    for (int a = 0; a < nt; ++a) {
      const int64_t r = (int64_t)a * P.s + t;
      const V32 w = w_entry32(P, i, r);
      const float v = (__ldg(P.sign + r) < 0) ? -w.v : w.v;
      acc = (__popc((unsigned)(a & (int)b)) & 1) ? __fsub_rn(acc, v) : __fadd_rn(acc, v);
      ea = __fmaf_ru(kU, fabsf(acc), __fadd_ru(ea, w.e));
    }
  } else {
    const int32_t* rows = P.perm + j * P.nnz;
    const int8_t* sg = P.sign + j * P.nnz;
    for (int t = 0; t < P.nnz; ++t) {
      const V32 w = w_entry32(P, i, __ldg(rows + t));
      acc = (__ldg(sg + t) < 0) ? __fsub_rn(acc, w.v) : __fadd_rn(acc, w.v);
      ea = __fmaf_ru(kU, fabsf(acc), __fadd_ru(ea, w.e));
    }
  }
  const float r = __fmul_rn(acc, P.mscale32);
  float e = __fmaf_ru(ea, P.mscale32, __fmul_ru(fabsf(acc), P.mscale_err));
  e = __fmaf_ru(kU, fabsf(r), __fadd_ru(e, kTiny));
  return V32{r, e};
}

__device__ __forceinline__ V32 strip_entry32(const DevProblem& P, int phase, const int32_t* Is, const int32_t* Js,
                                             int a, int64_t q) {
  return phase == 0 ? wp_entry32(P, Is[a], q) : wp_entry32(P, q, Js[a]);
}

// ---------------------------------------------------------------------------
// Certified argmax: best entry by FP32 magnitude (lowest column, then row, on
// ties) with its lower bound, plus the two largest upper bounds.
// ---------------------------------------------------------------------------
struct Cert {
  unsigned int key;
  int32_t i, j;
  float lo;
  float h1, h2;
  int32_t hi, hj;
  int bad;
};

static_assert(sizeof(Cert) <= 48, "certificate scratch is sized for 48-byte entries");

__device__ __forceinline__ Cert cert_none() {
  return Cert{0u, 0x7fffffff, 0x7fffffff, -INFINITY, -INFINITY, -INFINITY, -1, -1, 0};
}

__device__ __forceinline__ bool key_better(unsigned ka, int ia, int ja, unsigned kb, int ib, int jb) {
  return ka > kb || (ka == kb && (ja < jb || (ja == jb && ia < ib)));
}

__device__ __forceinline__ void cert_add(Cert& c, float v, float e, int32_t i, int32_t j) {
  const float av = fabsf(v);
  const float ae = __fmul_ru(e, kCert);
  if (!(av <= 3.0e38f) || !(ae <= 3.0e38f)) { c.bad = 1; return; }
  const unsigned key = __float_as_uint(av) + 1u;
  if (key_better(key, i, j, c.key, c.i, c.j)) { c.key = key; c.i = i; c.j = j; c.lo = __fsub_rd(av, ae); }
  const float hv = __fadd_ru(av, ae);
  if (hv > c.h1) { c.h2 = c.h1; c.h1 = hv; c.hi = i; c.hj = j; }
  else c.h2 = fmaxf(c.h2, hv);
}

__device__ __forceinline__ Cert cert_merge(const Cert& a, const Cert& b) {
  Cert r;
  if (key_better(a.key, a.i, a.j, b.key, b.i, b.j)) { r.key = a.key; r.i = a.i; r.j = a.j; r.lo = a.lo; }
  else { r.key = b.key; r.i = b.i; r.j = b.j; r.lo = b.lo; }
  if (a.h1 >= b.h1) { r.h1 = a.h1; r.hi = a.hi; r.hj = a.hj; r.h2 = fmaxf(a.h2, b.h1); }
  else { r.h1 = b.h1; r.hi = b.hi; r.hj = b.hj; r.h2 = fmaxf(b.h2, a.h1); }
  r.bad = a.bad | b.bad;
  return r;
}

__device__ __forceinline__ Cert cert_shfl(const Cert& c, int src_off) {
  Cert o;
  o.key = __shfl_xor_sync(0xffffffffu, c.key, src_off);
  o.i = __shfl_xor_sync(0xffffffffu, c.i, src_off);
  o.j = __shfl_xor_sync(0xffffffffu, c.j, src_off);
  o.lo = __shfl_xor_sync(0xffffffffu, c.lo, src_off);
  o.h1 = __shfl_xor_sync(0xffffffffu, c.h1, src_off);
  o.h2 = __shfl_xor_sync(0xffffffffu, c.h2, src_off);
  o.hi = __shfl_xor_sync(0xffffffffu, c.hi, src_off);
  o.hj = __shfl_xor_sync(0xffffffffu, c.hj, src_off);
  o.bad = __shfl_xor_sync(0xffffffffu, c.bad, src_off);
  return o;
}

__device__ __forceinline__ Cert warp_cert(Cert c) {
  for (int off = 16; off > 0; off >>= 1) c = cert_merge(c, cert_shfl(c, off));
  return c;
}

// All threads get the CTA's certificate.  red: >= 33 Certs of shared memory.
__device__ __forceinline__ Cert block_cert(Cert c, Cert* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  c = warp_cert(c);
  if (lane == 0) red[warp] = c;
  __syncthreads();
  if (warp == 0) {
    Cert d = (lane < (int)(blockDim.x >> 5)) ? red[lane] : cert_none();
    d = warp_cert(d);
    if (lane == 0) red[32] = d;
  }
  __syncthreads();
  const Cert r = red[32];
  __syncthreads();
  return r;
}

// Largest upper bound among the entries other than the winner.
__device__ __forceinline__ float cert_other_hi(const Cert& c) {
  return (c.hi == c.i && c.hj == c.j) ? c.h2 : c.h1;
}

struct MixedStep {
  int status;
  int nswaps;
  double logdet;
  int fallback;
};

// One maxvol step in FP32 with certified decisions, for a group of one CTA (the
// whole strip is this CTA's chunk).  Same contract as maxvol_step; on a
// fallback, Jsel is restored to its value on entry.
__device__ inline MixedStep maxvol_step_mixed(const CaArgs& A, const CaSmem& S, int phase, bool cold, int32_t* Jsel,
                                              bool lead) {
  const DevProblem& P = A.P;
  const int k = A.k, ldm = A.ldm, tid = threadIdx.x, nt = blockDim.x;
  const int ldl = k | 1;
  const int lane = tid & 31, warp = tid >> 5;
  const int qn = (int)(phase == 0 ? P.n : P.m);
  const Map2D mp(qn);
  float* a = reinterpret_cast<float*>(S.M);
  float* e = a + (size_t)k * ldm;
  float* B = reinterpret_cast<float*>(S.LU);       // U0 / warm LU values
  float* BE = B + (size_t)k * ldl;                 // and bounds
  float* L = reinterpret_cast<float*>(S.Lm);       // warm multipliers
  float* LE = L + (size_t)k * ldl;
  float* X = reinterpret_cast<float*>(S.x);        // exchanged column (k) and bounds
  float* XE = X + KMAX;
  float* LM = reinterpret_cast<float*>(S.lmul);    // cold multipliers and bounds
  float* LME = LM + KMAX;
  float* TQ = reinterpret_cast<float*>(S.tq);
  float* TQE = TQ + ldm;
  float* bcf = reinterpret_cast<float*>(S.bc);
  MixedStep res{LRA_OK, 0, 0.0, 0};
  LogAcc Lg{0.0, 0};

  for (int t = tid; t < k; t += nt) S.Jsave[t] = Jsel[t];
  if (tid == 0) { S.ctl[0] = 0; S.ctl[1] = 0; }
  for (int c = tid; c < qn; c += nt) S.pos[c] = 0;
  __syncthreads();
  // ---- gather the strip in FP32 with bounds
  {
    int bad = 0;
    for (int c = mp.c0; c < qn; c += mp.cstep)
      for (int r = mp.g; r < k; r += mp.G) {
        const V32 w = strip_entry32(P, phase, S.Is, S.Js, r, c);
        a[(size_t)r * ldm + c] = w.v;
        e[(size_t)r * ldm + c] = w.e;
        bad |= !(fabsf(w.v) <= 3.0e38f) || !(w.e <= 3.0e38f);
      }
    if (bad) atomicOr(&S.ctl[0], 1);
  }
  __syncthreads();
  auto fail = [&]() -> MixedStep {
    __syncthreads();
    for (int t = tid; t < k; t += nt) Jsel[t] = S.Jsave[t];
    __syncthreads();
    MixedStep f{LRA_OK, 0, 0.0, 1};
    return f;
  };
  if (S.ctl[0]) return fail();
  bool deficient = false;

  if (!cold) {
    for (int it = tid; it < k * k; it += nt) {
      const int r = it / k, t = it - r * k;
      const V32 w = strip_entry32(P, phase, S.Is, S.Js, r, Jsel[t]);
      B[r * ldl + t] = w.v;
      BE[r * ldl + t] = w.e;
    }
    __syncthreads();
    const int jj = tid & (KMAX - 1), rg = tid >> 6, NRG = nt >> 6;
    int verdict = 0;       // 0 ok, 1 exact zero pivot (cold start), 2 not certified
    for (int t = 0; t < k; ++t) {
      if (warp == 0) {
        Cert c = cert_none();
        for (int p = t + lane; p < k; p += 32) cert_add(c, B[p * ldl + t], BE[p * ldl + t], 0, p);
        c = warp_cert(c);
        const int r = c.j;
        int v = 2;
        if (!c.bad && c.key != 0u) {
          if (c.lo > cert_other_hi(c) && c.lo > 0.f) v = 0;
          else if (c.h1 == 0.f) v = 1;
        }
        if (v == 0) {
          if (lane == 0) {
            S.piv[t] = r;
            bcf[0] = __frcp_rn(B[r * ldl + t]);
            bcf[1] = B[r * ldl + t];
            bcf[2] = BE[r * ldl + t];
          }
          if (r != t)
            for (int j = t + lane; j < k; j += 32) {
              float tmp = B[t * ldl + j]; B[t * ldl + j] = B[r * ldl + j]; B[r * ldl + j] = tmp;
              tmp = BE[t * ldl + j]; BE[t * ldl + j] = BE[r * ldl + j]; BE[r * ldl + j] = tmp;
            }
        }
        if (lane == 0) S.ctl[1] = v;
      }
      __syncthreads();
      verdict = S.ctl[1];
      if (verdict != 0) break;
      const float rho = bcf[0], pv = bcf[1], epv = bcf[2];
      for (int p = t + 1 + tid; p < k; p += nt) {
        const float l = __fmul_rn(B[p * ldl + t], rho);
        L[p * ldl + t] = l;
        LE[p * ldl + t] = quot_bound(l, BE[p * ldl + t], pv, epv);
      }
      __syncthreads();
      if (jj > t && jj < k)
        for (int p = t + 1 + rg; p < k; p += NRG) {
          const float l = L[p * ldl + t], el = LE[p * ldl + t];
          const float at = B[t * ldl + jj], et = BE[t * ldl + jj];
          const float nv = __fmaf_rn(-l, at, B[p * ldl + jj]);
          BE[p * ldl + jj] = elim_bound(nv, l, el, at, et, BE[p * ldl + jj]);
          B[p * ldl + jj] = nv;
        }
      __syncthreads();
    }
    if (verdict == 2) return fail();
    if (verdict == 1) {
      cold = true;                      // the FP64 reference falls back to a cold start too
    } else {
      if (tid == 0)
        for (int t = 0; t < k; ++t) S.pos[Jsel[t]] = t + 1;
      __syncthreads();
      for (int t = 0; t < k; ++t) {
        const int r = S.piv[t];
        if (r != t)
          for (int c = tid; c < qn; c += nt) {
            float tmp = a[(size_t)t * ldm + c]; a[(size_t)t * ldm + c] = a[(size_t)r * ldm + c];
            a[(size_t)r * ldm + c] = tmp;
            tmp = e[(size_t)t * ldm + c]; e[(size_t)t * ldm + c] = e[(size_t)r * ldm + c];
            e[(size_t)r * ldm + c] = tmp;
          }
        __syncthreads();
        for (int c = mp.c0; c < qn; c += mp.cstep) {
          if (S.pos[c]) continue;
          const float at = a[(size_t)t * ldm + c], et = e[(size_t)t * ldm + c];
          for (int p = mp.first(t + 1); p < k; p += mp.G) {
            const float l = L[p * ldl + t], el = LE[p * ldl + t];
            const float nv = __fmaf_rn(-l, at, a[(size_t)p * ldm + c]);
            e[(size_t)p * ldm + c] = elim_bound(nv, l, el, at, et, e[(size_t)p * ldm + c]);
            a[(size_t)p * ldm + c] = nv;
          }
        }
        __syncthreads();
      }
      for (int t = 0; t < k; ++t) log_push(Lg, S, lead, (double)fabsf(B[t * ldl + t]));
    }
  }

  if (cold) {
    for (int c = tid; c < qn; c += nt) S.pos[c] = 0;
    __syncthreads();
    for (int t = 0; t < k; ++t) {
      Cert c = cert_none();
      for (int q = tid; q < qn; q += nt)
        if (S.pos[q] == 0) cert_add(c, a[(size_t)t * ldm + q], e[(size_t)t * ldm + q], 0, q);
      c = block_cert(c, S.cert);
      if (c.bad || c.key == 0u) return fail();
      const int w = c.j;
      if (!(c.lo > cert_other_hi(c) && c.lo > 0.f)) {
        if (c.h1 != 0.f) return fail();
        // every candidate is exactly zero: the reference meets a zero pivot
        if (tid == 0) { Jsel[t] = w; S.pos[w] = t + 1; }
        deficient = true;
        __syncthreads();
        continue;
      }
      const float pv = a[(size_t)t * ldm + w], epv = e[(size_t)t * ldm + w];
      if (tid == 0) { Jsel[t] = w; S.pos[w] = t + 1; bcf[0] = __frcp_rn(pv); }
      for (int p = tid; p <= t; p += nt) { B[p * ldl + t] = a[(size_t)p * ldm + w]; BE[p * ldl + t] = e[(size_t)p * ldm + w]; }
      __syncthreads();
      const float rho = bcf[0];
      for (int p = t + 1 + tid; p < k; p += nt) {
        const float l = __fmul_rn(a[(size_t)p * ldm + w], rho);
        LM[p] = l;
        LME[p] = quot_bound(l, e[(size_t)p * ldm + w], pv, epv);
      }
      __syncthreads();
      for (int q = mp.c0; q < qn; q += mp.cstep) {
        if (S.pos[q]) continue;
        const float at = a[(size_t)t * ldm + q], et = e[(size_t)t * ldm + q];
        for (int p = mp.first(t + 1); p < k; p += mp.G) {
          const float nv = __fmaf_rn(-LM[p], at, a[(size_t)p * ldm + q]);
          e[(size_t)p * ldm + q] = elim_bound(nv, LM[p], LME[p], at, et, e[(size_t)p * ldm + q]);
          a[(size_t)p * ldm + q] = nv;
        }
      }
      log_push(Lg, S, lead, (double)fabsf(pv));
      __syncthreads();
    }
    if (deficient) {
      res.status = LRA_WARN_RANK_DEFICIENT;
      res.logdet = -INFINITY;
      return res;
    }
  }

  // ---- back substitution C = U0^{-1} (rows of the eliminated strip), bounds carried
  float* RD = reinterpret_cast<float*>(S.rdiag);
  for (int i = tid; i < k; i += nt) RD[i] = __frcp_rn(B[i * ldl + i]);
  __syncthreads();
  for (int c = mp.c0; c < qn; c += mp.cstep)
    if (S.pos[c] == 0 && (k - 1) % mp.G == mp.g) {
      const size_t o = (size_t)(k - 1) * ldm + c;
      const float x = __fmul_rn(a[o], RD[k - 1]);
      e[o] = quot_bound(x, e[o], B[(k - 1) * ldl + k - 1], BE[(k - 1) * ldl + k - 1]);
      a[o] = x;
    }
  __syncthreads();
  for (int i = k - 1; i >= 1; --i) {
    for (int c = mp.c0; c < qn; c += mp.cstep) {
      if (S.pos[c]) continue;
      const float xi = a[(size_t)i * ldm + c], exi = e[(size_t)i * ldm + c];
      for (int p = mp.first(0); p < i; p += mp.G) {
        const size_t o = (size_t)p * ldm + c;
        const float u = B[p * ldl + i], eu = BE[p * ldl + i];
        float nv = __fmaf_rn(-u, xi, a[o]);
        float ev = elim_bound(nv, u, eu, xi, exi, e[o]);
        if (p == i - 1) {
          const float x = __fmul_rn(nv, RD[i - 1]);
          ev = quot_bound(x, ev, B[(i - 1) * ldl + i - 1], BE[(i - 1) * ldl + i - 1]);
          nv = x;
        }
        a[o] = nv;
        e[o] = ev;
      }
    }
    __syncthreads();
  }
  for (int c = mp.c0; c < qn; c += mp.cstep)
    if (S.pos[c])
      for (int r = mp.g; r < k; r += mp.G) {
        a[(size_t)r * ldm + c] = (S.pos[c] - 1 == r) ? 1.f : 0.f;
        e[(size_t)r * ldm + c] = 0.f;
      }
  __syncthreads();

  // ---- dominance swaps, every decision certified
  const float h_lo = __double2float_rd(A.h), h_hi = __double2float_ru(A.h);
  int nsw = 0;
  for (;;) {
    Cert c = cert_none();
    for (int q = mp.c0; q < qn; q += mp.cstep) {
      if (S.pos[q]) continue;
      for (int r = mp.g; r < k; r += mp.G) cert_add(c, a[(size_t)r * ldm + q], e[(size_t)r * ldm + q], r, q);
    }
    c = block_cert(c, S.cert);
    if (c.bad) return fail();
    if (c.key == 0u) break;                               // no unchosen column
    const bool arg_ok = c.lo > cert_other_hi(c);
    if (arg_ok && c.lo > h_hi) {
      // certified swap
    } else if (c.h1 <= h_lo) {
      break;                                              // certified stop: every |c| <= h
    } else {
      return fail();
    }
    if (nsw >= A.max_swaps) { res.status = LRA_WARN_NOT_CONVERGED; break; }
    const int wi = c.i, wj = c.j;
    const float cs = a[(size_t)wi * ldm + wj], ecs = e[(size_t)wi * ldm + wj];
    for (int p = tid; p < k; p += nt) { X[p] = a[(size_t)p * ldm + wj]; XE[p] = e[(size_t)p * ldm + wj]; }
    if (tid == 0) bcf[0] = __frcp_rn(cs);
    __syncthreads();
    const float rho = bcf[0];
    for (int q = tid; q < qn; q += nt) {
      const float tq = __fmul_rn(a[(size_t)wi * ldm + q], rho);
      TQ[q] = tq;
      TQE[q] = quot_bound(tq, e[(size_t)wi * ldm + q], cs, ecs);
    }
    __syncthreads();
    for (int q = mp.c0; q < qn; q += mp.cstep) {
      const float tq = TQ[q], tqe = TQE[q];
      for (int r = mp.g; r < k; r += mp.G) {
        const size_t o = (size_t)r * ldm + q;
        if (r == wi) { a[o] = tq; e[o] = tqe; }
        else {
          const float nv = __fmaf_rn(-X[r], tq, a[o]);
          e[o] = elim_bound(nv, X[r], XE[r], tq, tqe, e[o]);
          a[o] = nv;
        }
      }
    }
    __syncthreads();
    for (int p = tid; p < k; p += nt) {
      a[(size_t)p * ldm + wj] = (p == wi) ? 1.f : 0.f;
      e[(size_t)p * ldm + wj] = 0.f;
    }
    if (tid == 0) {
      S.pos[Jsel[wi]] = 0;
      S.pos[wj] = wi + 1;
      Jsel[wi] = wj;
    }
    log_push(Lg, S, lead, (double)fabsf(cs));
    ++nsw;
    __syncthreads();
  }
  log_flush(Lg, S);
  res.nswaps = nsw;
  res.logdet = Lg.sum;
  return res;
}

}  // namespace lra
