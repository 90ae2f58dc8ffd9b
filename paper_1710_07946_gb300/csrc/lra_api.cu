// lra_api.cu -- multiplier handles, problem validation and small utilities of
// the C ABI.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <vector>

#include "lra_internal.h"

namespace lra {

lra_status make_dev_problem(const lra_problem* p, lra_multiplier mult, DevProblem* out) {
  if (p == nullptr || out == nullptr) return LRA_ERR_INVALID_ARG;
  if (p->m < 1 || p->n < 1 || p->m >= (int64_t(1) << 31) || p->n >= (int64_t(1) << 31)) return LRA_ERR_INVALID_ARG;
  DevProblem d;
  std::memset(&d, 0, sizeof(d));
  d.src = p->src;
  d.dtype = p->dtype;
  d.m = p->m;
  d.n = p->n;
  d.ldw = p->ldw;
  d.W = p->W;
  d.X = p->X;
  d.Y = p->Y;
  d.ell = p->length_scale;
  if (p->src == LRA_DENSE) {
    if (p->W == nullptr || p->ldw < p->n) return LRA_ERR_INVALID_ARG;
    if (p->dtype != LRA_F64 && p->dtype != LRA_F32) return LRA_ERR_INVALID_ARG;
  } else if (p->src == LRA_KERNEL_LAPLACE || p->src == LRA_KERNEL_GAUSSIAN) {
    if (p->X == nullptr || p->Y == nullptr) return LRA_ERR_INVALID_ARG;
    if (p->src == LRA_KERNEL_GAUSSIAN && !(p->length_scale > 0.0)) return LRA_ERR_INVALID_ARG;
    // FP32 and BF16 entries are defined for the Laplace kernel only
    if (p->dtype != LRA_F64 && !((p->dtype == LRA_F32 || p->dtype == LRA_BF16) && p->src == LRA_KERNEL_LAPLACE))
      return LRA_ERR_INVALID_ARG;
  } else {
    return LRA_ERR_INVALID_ARG;
  }
  d.mkind = LRA_MULT_NONE;
  if (mult != nullptr && mult->kind != LRA_MULT_NONE) {
    const int64_t dim = (mult->side == LRA_SIDE_LEFT) ? p->m : p->n;   // M is dim x dim
    if (mult->n != dim) return LRA_ERR_INVALID_ARG;
    d.mkind = mult->kind;
    d.mside = (mult->side == LRA_SIDE_LEFT) ? 1 : 0;
    d.perm = mult->d_idx;
    d.sign = mult->d_sign;
    d.mscale = mult->scale;
    if (mult->kind == LRA_MULT_ARHT) {
      d.depth = mult->param;
      d.s = dim >> mult->param;
    } else if (mult->kind == LRA_MULT_BIDIAG) {
      d.depth = mult->param;
      d.nnz = mult->width;
      d.bval = mult->d_val;
    } else if (mult->kind == LRA_MULT_ARFT) {
      if (mult->side != LRA_SIDE_RIGHT) return LRA_ERR_INVALID_ARG;
      d.depth = mult->param;
      d.nnz = mult->width;
      d.fwt = mult->d_wt;
    } else {
      d.nnz = mult->param;
    }
    // FP32 copy of the scale; exact when it is a power of two (even depth, nnz = 1, 4, 16)
    const bool exact = (mult->kind == LRA_MULT_ARHT) ? (mult->param % 2 == 0)
                                                     : (mult->param == 1 || mult->param == 4 || mult->param == 16);
    d.mscale32 = (float)mult->scale;
    d.mscale_err = exact ? 0.0f : 1.0001f * 5.9604644775390625e-08f * d.mscale32;
  }
  *out = d;
  return LRA_OK;
}

__global__ void points_to_f32_kernel(const double* __restrict__ X, int64_t cnt, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __double2float_rn(X[i]);
}

lra_status points_to_f32(const double* X, int64_t npts, float* out, cudaStream_t stream) {
  const int64_t cnt = 3 * npts;
  const int grid = (int)std::min<int64_t>((cnt + 255) / 256, 4096);
  points_to_f32_kernel<<<grid, 256, 0, stream>>>(X, cnt, out);
  return cuda_status(cudaGetLastError());
}

lra_status current_device_info(DeviceInfo* info) {
  int dev = 0;
  LRA_CUDA_TRY(cudaGetDevice(&dev));
  int sms = 0, optin = 0;
  LRA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  LRA_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  info->device = dev;
  info->sms = sms;
  info->smem_optin = (size_t)optin;
  return LRA_OK;
}

// The columns of M = F_1 ... F_q (F_f = (I + D_f S) P_f): column j is
// F_1 (... (F_q e_j)), a list of (row, integer value) terms expanded factor by
// factor (each term a -> b = perm_f[a] with its value and b' = (b + 1) mod n
// with sign_f[b'] times it) and merged by row in a dense accumulator after
// every factor.  A column has at most min(2^q, n) nonzeros; they are stored in
// that many slots per column in ascending rows, value 0 in the unused slots.
// |values| <= 2^q (int32 for q <= 30); the scale 2^{-q/2} is applied by the
// gathers.
static lra_status make_bidiag(lra_multiplier* out, int32_t side, int64_t n, int32_t q, const int32_t* perms,
                              const int8_t* signs) {
  const int64_t w = std::min<int64_t>(int64_t(1) << q, n);
  std::vector<int32_t> rows((size_t)n * (size_t)w, 0);
  std::vector<int32_t> vals((size_t)n * (size_t)w, 0);
  std::vector<int64_t> acc((size_t)n, 0);
  std::vector<unsigned char> touched((size_t)n, 0);
  std::vector<int64_t> cur, nxt;       // rows with a nonzero value
  for (int64_t j = 0; j < n; ++j) {
    cur.assign(1, j);
    acc[(size_t)j] = 1;
    for (int f = q - 1; f >= 0; --f) {
      std::vector<std::pair<int64_t, int64_t>> terms;
      terms.reserve(cur.size());
      for (int64_t a : cur) {
        terms.push_back({a, acc[(size_t)a]});
        acc[(size_t)a] = 0;
      }
      nxt.clear();
      for (const auto& tv : terms) {
        const int64_t b = perms[(int64_t)f * n + tv.first], b1 = (b + 1) % n;
        const int64_t add[2] = {tv.second, (int64_t)signs[(int64_t)f * n + b1] * tv.second};
        const int64_t at[2] = {b, b1};
        for (int e = 0; e < 2; ++e) {
          if (!touched[(size_t)at[e]]) { touched[(size_t)at[e]] = 1; nxt.push_back(at[e]); }
          acc[(size_t)at[e]] += add[e];
        }
      }
      cur.clear();
      for (int64_t r : nxt) {
        touched[(size_t)r] = 0;
        if (acc[(size_t)r] != 0) cur.push_back(r);
      }
    }
    std::sort(cur.begin(), cur.end());
    size_t c = 0;
    for (int64_t r : cur) {
      rows[(size_t)j * w + c] = (int32_t)r;
      vals[(size_t)j * w + c] = (int32_t)acc[(size_t)r];
      acc[(size_t)r] = 0;
      ++c;
    }
  }
  lra_multiplier m = new lra_multiplier_s;
  m->kind = LRA_MULT_BIDIAG;
  m->side = side;
  m->n = n;
  m->param = q;
  m->width = (int32_t)w;
  m->scale = 1.0 / std::sqrt((double)(int64_t(1) << q));
  m->d_idx = nullptr;
  m->d_sign = nullptr;
  m->d_val = nullptr;
  m->d_dense = nullptr;
  m->d_wt = nullptr;
  bool ok = cudaMalloc(&m->d_idx, rows.size() * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc(&m->d_val, vals.size() * sizeof(int32_t)) == cudaSuccess &&
            cudaMemcpy(m->d_idx, rows.data(), rows.size() * sizeof(int32_t), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(m->d_val, vals.data(), vals.size() * sizeof(int32_t), cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok && w == n && n <= 16384) {
    // every column can be full: keep M's integers densely as well, for the
    // register-tiled product of lra_multiplier_apply
    std::vector<double> dense((size_t)n * (size_t)n, 0.0);
    for (int64_t j = 0; j < n; ++j)
      for (int64_t t = 0; t < w; ++t) {
        const int32_t v = vals[(size_t)j * w + t];
        if (v != 0) dense[(size_t)rows[(size_t)j * w + t] * n + j] = (double)v;
      }
    ok = cudaMalloc(&m->d_dense, dense.size() * sizeof(double)) == cudaSuccess &&
         cudaMemcpy(m->d_dense, dense.data(), dense.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
  }
  if (!ok) {
    cudaFree(m->d_idx);
    cudaFree(m->d_val);
    cudaFree(m->d_dense);
    delete m;
    return LRA_ERR_CUDA;
  }
  *out = m;
  return LRA_OK;
}

// Columns of the real form [Re M, Im M] of M = D Omega_{n,d} P (before the scale
// 2^{-d/2}).  A column of Omega_{n,d} is built bottom-up from the recursion
// Omega_{2q} = Phat [[Omega_q, Omega_q], [Omega_q Dhat_q, -Omega_q Dhat_q]],
// Omega_s = I_s: column c of Omega_{2q} carries column c mod q of Omega_q to the
// even rows 2r and, times +-w_{2q}^{c mod q} (minus for c >= q), to the odd rows
// 2r + 1.  Entries are kept as exponents of w_n (w_{2q} = w_n^{n / 2q}, -1 =
// w_n^{n/2}).  Column j of M is D times column perm[j]; the real form stores, in
// ascending rows, Re(D_r w_n^e) for column j and Im(D_r w_n^e) for column n + j.
void fourier_real_columns(int64_t n, int32_t d, const int32_t* perm, const double* diag,
                          std::vector<int32_t>& rows, std::vector<double>& wts) {
  const int64_t w = int64_t(1) << d, s = n >> d;
  const double kPi = 3.14159265358979323846;
  rows.assign((size_t)(2 * n * w), 0);
  wts.assign((size_t)(2 * n * w), 0.0);
  std::vector<std::pair<int64_t, int64_t>> ent((size_t)w), nxt((size_t)w);   // (row, exponent)
  std::vector<int64_t> colat((size_t)d + 1);
  for (int64_t j = 0; j < n; ++j) {
    // the column index at every level, top (size n) down to the base (size s)
    int64_t c = perm[j], size = n;
    for (int32_t lev = d; lev >= 0; --lev) {
      colat[(size_t)lev] = c;
      if (lev > 0) { size /= 2; c %= size; }
    }
    int64_t cnt = 1, q = s;
    ent[0] = {colat[0], 0};
    for (int32_t lev = 1; lev <= d; ++lev, q *= 2) {
      const int64_t cl = colat[(size_t)lev], cp = cl % q;
      const int64_t tw = (cp * (n / (2 * q)) + (cl >= q ? n / 2 : 0)) % n;
      for (int64_t t = 0; t < cnt; ++t) {
        nxt[(size_t)t] = {2 * ent[(size_t)t].first, ent[(size_t)t].second};
        nxt[(size_t)(cnt + t)] = {2 * ent[(size_t)t].first + 1, (ent[(size_t)t].second + tw) % n};
      }
      cnt *= 2;
      std::swap(ent, nxt);
    }
    std::sort(ent.begin(), ent.begin() + w);
    for (int64_t t = 0; t < w; ++t) {
      const int64_t r = ent[(size_t)t].first;
      const double phi = (2.0 * kPi * (double)ent[(size_t)t].second) / (double)n;
      const double cr = std::cos(phi), ci = std::sin(phi);
      const double dr = diag[2 * r], di = diag[2 * r + 1];
      rows[(size_t)(j * w + t)] = (int32_t)r;
      wts[(size_t)(j * w + t)] = dr * cr - di * ci;
      rows[(size_t)((n + j) * w + t)] = (int32_t)r;
      wts[(size_t)((n + j) * w + t)] = dr * ci + di * cr;
    }
  }
}

}  // namespace lra

extern "C" {

lra_status lra_precondition(lra_multiplier* out, int32_t kind, int32_t side, int64_t n, int32_t param,
                            const int32_t* idx, const int8_t* signs) {
  if (out == nullptr) return LRA_ERR_INVALID_ARG;
  *out = nullptr;
  if (side != LRA_SIDE_RIGHT && side != LRA_SIDE_LEFT) return LRA_ERR_INVALID_ARG;
  if (n < 1 || n >= (int64_t(1) << 31) || idx == nullptr || signs == nullptr) return LRA_ERR_INVALID_ARG;
  size_t cnt = 0;
  double scale = 1.0;
  if (kind == LRA_MULT_ARHT) {
    if (param < 1 || param > 10 || (n % (int64_t(1) << param)) != 0) return LRA_ERR_INVALID_ARG;
    cnt = (size_t)n;
    std::vector<unsigned char> seen((size_t)n, 0);
    for (int64_t j = 0; j < n; ++j) {
      if (idx[j] < 0 || idx[j] >= n || seen[(size_t)idx[j]]) return LRA_ERR_INVALID_ARG;
      seen[(size_t)idx[j]] = 1;
      if (signs[j] != 1 && signs[j] != -1) return LRA_ERR_INVALID_ARG;
    }
    scale = 1.0 / std::sqrt((double)(int64_t(1) << param));
  } else if (kind == LRA_MULT_SPARSE_PM1) {
    if (param < 1 || param > 16 || param > n) return LRA_ERR_INVALID_ARG;
    cnt = (size_t)n * (size_t)param;
    for (int64_t j = 0; j < n; ++j)
      for (int t = 0; t < param; ++t) {
        int32_t r = idx[j * param + t];
        if (r < 0 || r >= n) return LRA_ERR_INVALID_ARG;
        if (t > 0 && r <= idx[j * param + t - 1]) return LRA_ERR_INVALID_ARG;
        int8_t s = signs[j * param + t];
        if (s != 1 && s != -1) return LRA_ERR_INVALID_ARG;
      }
    scale = 1.0 / std::sqrt((double)param);
  } else if (kind == LRA_MULT_BIDIAG) {
    if (param < 1 || param > 30 || n < 2 || n > INT32_MAX) return LRA_ERR_INVALID_ARG;
    std::vector<unsigned char> seen((size_t)n);
    for (int f = 0; f < param; ++f) {
      std::fill(seen.begin(), seen.end(), 0);
      for (int64_t a = 0; a < n; ++a) {
        const int32_t b = idx[(int64_t)f * n + a];
        if (b < 0 || b >= n || seen[(size_t)b]) return LRA_ERR_INVALID_ARG;
        seen[(size_t)b] = 1;
        const int8_t sg = signs[(int64_t)f * n + a];
        if (sg != 1 && sg != -1) return LRA_ERR_INVALID_ARG;
      }
    }
    return lra::make_bidiag(out, side, n, param, idx, signs);
  } else {
    return LRA_ERR_INVALID_ARG;
  }
  lra_multiplier m = new lra_multiplier_s;
  m->kind = kind;
  m->side = side;
  m->n = n;
  m->param = param;
  m->scale = scale;
  m->width = 0;
  m->d_idx = nullptr;
  m->d_sign = nullptr;
  m->d_val = nullptr;
  m->d_dense = nullptr;
  m->d_wt = nullptr;
  if (cudaMalloc(&m->d_idx, cnt * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&m->d_sign, cnt * sizeof(int8_t)) != cudaSuccess ||
      cudaMemcpy(m->d_idx, idx, cnt * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_sign, signs, cnt * sizeof(int8_t), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(m->d_idx);
    cudaFree(m->d_sign);
    delete m;
    return LRA_ERR_CUDA;
  }
  *out = m;
  return LRA_OK;
}

lra_status lra_multiplier_destroy(lra_multiplier m) {
  if (m == nullptr) return LRA_OK;
  cudaError_t e1 = cudaFree(m->d_idx);
  cudaError_t e2 = cudaFree(m->d_sign);
  cudaError_t e3 = cudaFree(m->d_val);
  cudaError_t e4 = cudaFree(m->d_dense);
  cudaError_t e5 = cudaFree(m->d_wt);
  delete m;
  return (e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess && e4 == cudaSuccess && e5 == cudaSuccess)
             ? LRA_OK
             : LRA_ERR_CUDA;
}

lra_status lra_precondition_fourier(lra_multiplier* out, int64_t n, int32_t depth, const int32_t* perm,
                                    const double* diag) {
  if (out == nullptr) return LRA_ERR_INVALID_ARG;
  *out = nullptr;
  if (perm == nullptr || diag == nullptr || depth < 1 || depth > 10 || n < 2 || n >= (int64_t(1) << 30) ||
      (n % (int64_t(1) << depth)) != 0)
    return LRA_ERR_INVALID_ARG;
  std::vector<unsigned char> seen((size_t)n, 0);
  for (int64_t j = 0; j < n; ++j) {
    if (perm[j] < 0 || perm[j] >= n || seen[(size_t)perm[j]]) return LRA_ERR_INVALID_ARG;
    seen[(size_t)perm[j]] = 1;
    const double a = diag[2 * j], b = diag[2 * j + 1];
    if (!(std::fabs(a * a + b * b - 1.0) <= 1e-12)) return LRA_ERR_INVALID_ARG;
  }
  std::vector<int32_t> rows;
  std::vector<double> wts;
  lra::fourier_real_columns(n, depth, perm, diag, rows, wts);
  lra_multiplier m = new lra_multiplier_s;
  m->kind = LRA_MULT_ARFT;
  m->side = LRA_SIDE_RIGHT;
  m->n = n;
  m->param = depth;
  m->width = 1 << depth;
  m->scale = 1.0 / std::sqrt((double)(int64_t(1) << depth));
  m->d_idx = nullptr;
  m->d_sign = nullptr;
  m->d_val = nullptr;
  m->d_dense = nullptr;
  m->d_wt = nullptr;
  if (cudaMalloc(&m->d_idx, rows.size() * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&m->d_wt, wts.size() * sizeof(double)) != cudaSuccess ||
      cudaMemcpy(m->d_idx, rows.data(), rows.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_wt, wts.data(), wts.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(m->d_idx);
    cudaFree(m->d_wt);
    delete m;
    return LRA_ERR_CUDA;
  }
  *out = m;
  return LRA_OK;
}

const char* lra_version(void) { return "lra-gb300 0.1 (sm_103a)"; }

}  // extern "C"
