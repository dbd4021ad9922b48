// Set-up, right-hand side, stand-alone operator apply and gradient kernels.
#include <algorithm>
#include <cmath>

#include "pcg_kernels.cuh"

namespace sylv {

namespace {
constexpr int SETUP_BLOCK = 256;

inline int blocks_for(int64_t n, int block) { return (int)((n + block - 1) / block); }
}  // namespace

// flags bits
constexpr unsigned FLAG_ROWPTR = 1u, FLAG_COL = 2u, FLAG_NNZ = 4u, FLAG_VALUE = 8u,
                   FLAG_DEGREE = 16u;

// Validates the CSR structure; records the largest number of off-diagonal entries per row.
__global__ void k_csr_check(int64_t n, const int32_t* __restrict__ rowptr,
                            const int32_t* __restrict__ col, int64_t nnz,
                            unsigned int* flags, unsigned int* maxdeg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    if (rowptr[0] != 0 || (int64_t)rowptr[n] != nnz) atomicOr(flags, FLAG_NNZ);
  }
  if (i >= n) return;
  const int64_t lo = rowptr[i], hi = rowptr[i + 1];
  if (lo < 0 || hi < lo || hi > nnz) {
    atomicOr(flags, FLAG_ROWPTR);
    return;
  }
  unsigned deg = 0;
  for (int64_t e = lo; e < hi; ++e) {
    const int32_t c = col[e];
    if (c < 0 || (int64_t)c >= n) {
      atomicOr(flags, FLAG_COL);
      return;
    }
    if ((int64_t)c != i) ++deg;
  }
  if (deg > (unsigned)EMAX) atomicOr(flags, FLAG_DEGREE);
  atomicMax(maxdeg, deg);
}

// Sliced ELL: slot e of row i at e * ld + i; diagonal entries (summed) go to diag.
__global__ void k_ell_build(int64_t n, int64_t ld, const int32_t* __restrict__ rowptr,
                            const int32_t* __restrict__ col, const double* __restrict__ val,
                            int E, int32_t* ell_col, float* ell_val32, double* ell_val64,
                            float* diag32, double* diag64) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double dg = 0.0;
  int e = 0;
  for (int64_t t = rowptr[i]; t < rowptr[i + 1]; ++t) {
    const int32_t c = col[t];
    const double v = val[t];
    if ((int64_t)c == i) {
      dg += v;
    } else if (e < E) {
      ell_col[e * ld + i] = c;
      ell_val32[e * ld + i] = (float)v;
      ell_val64[e * ld + i] = v;
      ++e;
    }
  }
  for (; e < E; ++e) {
    ell_col[e * ld + i] = (int32_t)i;
    ell_val32[e * ld + i] = 0.0f;
    ell_val64[e * ld + i] = 0.0;
  }
  diag32[i] = (float)dg;
  diag64[i] = dg;
}

// Row i of L L for a symmetric L held as diagonal + sliced ELL (padding slots point at the row
// itself): the prior shape L^T L = L^2 of the intrinsic GMRF (App. C).  Row i collects
// L_ii row_i(L) + sum_e L_{i c_e} row_{c_e}(L); the off-diagonal entries are merged by column
// and sorted ascending, the diagonal is returned apart.  Returns the number of off-diagonals.
constexpr int SQ_MAX = 1 + EMAX + EMAX * EMAX;

__device__ int square_row(int64_t ld, int E, const int32_t* __restrict__ ell_col,
                          const double* __restrict__ ell_val, const double* __restrict__ diag,
                          int64_t i, int32_t* cols, double* vals, double* dg_out) {
  int cnt = 0;
  auto add = [&](int32_t c, double v) {
    for (int t = 0; t < cnt; ++t)
      if (cols[t] == c) {
        vals[t] += v;
        return;
      }
    cols[cnt] = c;
    vals[cnt] = v;
    ++cnt;
  };
  const double di = diag[i];
  double dg = di * di;
  for (int e = 0; e < E; ++e) {
    const int32_t c = ell_col[e * ld + i];
    if ((int64_t)c == i) continue;
    const double v = ell_val[e * ld + i];
    add(c, di * v);                       // L_ii L_ic
    add(c, v * diag[c]);                  // L_ic L_cc
    for (int f = 0; f < E; ++f) {         // L_ic L_{c c2}
      const int32_t c2 = ell_col[f * ld + c];
      if (c2 == c) continue;
      const double v2 = ell_val[f * ld + c];
      if ((int64_t)c2 == i) dg += v * v2;
      else add(c2, v * v2);
    }
  }
  // insertion sort by column: a fixed order for the sums that use the row
  for (int a = 1; a < cnt; ++a) {
    const int32_t c = cols[a];
    const double v = vals[a];
    int b = a - 1;
    while (b >= 0 && cols[b] > c) {
      cols[b + 1] = cols[b];
      vals[b + 1] = vals[b];
      --b;
    }
    cols[b + 1] = c;
    vals[b + 1] = v;
  }
  *dg_out = dg;
  return cnt;
}

__global__ void k_square_count(int64_t n, int64_t ld, int E, const int32_t* __restrict__ ell_col,
                               const double* __restrict__ ell_val,
                               const double* __restrict__ diag, unsigned int* width) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t cols[SQ_MAX];
  double vals[SQ_MAX], dg;
  const int cnt = square_row(ld, E, ell_col, ell_val, diag, i, cols, vals, &dg);
  atomicMax(width, (unsigned int)cnt);
}

__global__ void k_square_fill(int64_t n, int64_t ld, int E, const int32_t* __restrict__ ell_col,
                              const double* __restrict__ ell_val, const double* __restrict__ diag,
                              int E2, int32_t* sq_col, float* sq_val32, double* sq_val64,
                              float* sq_diag32, double* sq_diag64) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t cols[SQ_MAX];
  double vals[SQ_MAX], dg;
  const int cnt = square_row(ld, E, ell_col, ell_val, diag, i, cols, vals, &dg);
  for (int e = 0; e < E2; ++e) {
    const bool real = e < cnt;
    sq_col[e * ld + i] = real ? cols[e] : (int32_t)i;
    sq_val64[e * ld + i] = real ? vals[e] : 0.0;
    sq_val32[e * ld + i] = real ? (float)vals[e] : 0.0f;
  }
  sq_diag64[i] = dg;
  sq_diag32[i] = (float)dg;
}

// Probe estimator of the posterior variances: num += z o x and den += z o z over R probes z
// (caller layout, pitch ldu) and their solves x = G^{-1} z; then var = num / den.
__global__ void k_var_accum(int64_t n, int k, int64_t ldu, int64_t ld, const double* __restrict__ Z,
                            const double* __restrict__ X, int R, double* num, double* den) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)k * n) return;
  const int64_t j = t / n, i = t - j * n;
  double a = num[j * ld + i], b = den[j * ld + i];
  for (int r = 0; r < R; ++r) {
    const double z = Z[((int64_t)r * k + j) * ldu + i];
    a += z * X[((int64_t)r * k + j) * ldu + i];
    b += z * z;
  }
  num[j * ld + i] = a;
  den[j * ld + i] = b;
}

// Probes s = 0..R-1 of a colouring: probe p0 + s is colour q = (p0 + s) / k in source
// j = (p0 + s) % k, i.e. Z[s][j'][i] = 1 where j' = j and colour[i] = q, else 0.  Colours
// outside [0, ncol) are flagged.
__global__ void k_probe_fill(int64_t n, int k, int64_t ldu, const int32_t* __restrict__ colour,
                             int ncol, int p0, int R, double* __restrict__ Z,
                             unsigned int* flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = colour[i];
  if (c < 0 || c >= ncol) atomicOr(flag, 1u);
  for (int s = 0; s < R; ++s) {
    const int q = (p0 + s) / k, j0 = (p0 + s) % k;
    for (int j = 0; j < k; ++j) Z[((int64_t)s * k + j) * ldu + i] = (j == j0 && c == q) ? 1.0 : 0.0;
  }
}

__global__ void k_var_finish(int64_t n, int k, int64_t ldu, int64_t ld,
                             const double* __restrict__ num, const double* __restrict__ den,
                             double* var) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)k * n) return;
  const int64_t j = t / n, i = t - j * n;
  const double b = den[j * ld + i];
  var[j * ldu + i] = b > 0.0 ? num[j * ld + i] / b : 0.0;
}

// Copies rows x n values (pitch ld) into FP32 and FP64 buffers and checks them (>= 0, or > 0
// if positive, and finite).
__global__ void k_convert_check(const double* __restrict__ src, int64_t rows, int64_t n,
                                int64_t ld_src, int64_t ld_dst, float* dst32, double* dst64,
                                int positive, unsigned int* flags) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * n) return;
  const int64_t r = t / n, i = t - r * n;
  const double v = src[r * ld_src + i];
  if (!isfinite(v) || v < 0.0 || (positive && !(v > 0.0))) atomicOr(flags, FLAG_VALUE);
  dst32[r * ld_dst + i] = (float)v;
  dst64[r * ld_dst + i] = v;
}

// b = B^T C y (eq. mu*): B[r][j][i] = sum_c a_cj d_ci y[r][c][i]
__global__ void k_rhs(OpData op, const double* __restrict__ Y, double* __restrict__ B, int R,
                      int64_t i0, int64_t i1) {
  const int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= i1) return;
  const int64_t ld = op.ld, ldu = op.ldu;
  for (int r = 0; r < R; ++r) {
    double acc[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) acc[j] = 0.0;
    for (int c = 0; c < op.m; ++c) {
      const double dy = op.D64[c * ld + i] * Y[((int64_t)r * op.m + c) * ldu + i];
#pragma unroll
      for (int j = 0; j < KMAX; ++j)
        if (j < op.k) acc[j] += op.A64[c * op.k + j] * dy;
    }
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < op.k) B[((int64_t)r * op.k + j) * ldu + i] = acc[j];
  }
}

// FP32 pairs of an FP64 array (the double-float residual's operator copies): hi = fl32(v),
// lo = fl32(v - hi), so v = hi + lo to 2^-48 |v|.  Flags entries outside what the double-float
// residual takes (nonzero with |v| outside [2^-40, 2^40], or not finite).
__global__ void __launch_bounds__(256) k_split_hl(const double* __restrict__ src, int64_t total,
                                                  int64_t rows_ld, float* __restrict__ dst,
                                                  unsigned int* flag) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const double v = src[t];
  const float h = (float)v;
  const float l = (float)(v - (double)h);
  dst[t] = h;
  dst[rows_ld + t] = l;
  const double a = fabs(v);
  if (!isfinite(v) || (v != 0.0 && (a < 0x1p-40 || a > 0x1p40))) atomicOr(flag, 1u);
}

// Pixel blocks P_i (FP64) and their scaled Cholesky factors, once per handle.
template <int K>
__global__ void __launch_bounds__(256) k_block_setup(OpData op, double* __restrict__ blk,
                                                     double* __restrict__ fac,
                                                     float* __restrict__ fs32,
                                                     __half2* __restrict__ fl16) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= op.n) return;
  const int64_t ld = op.ld;
  double P[K * (K + 1) / 2];
#pragma unroll
  for (int a = 0; a < K * (K + 1) / 2; ++a) P[a] = 0.0;
  for (int c = 0; c < op.m; ++c) {
    const double d = op.D64[c * ld + i];
#pragma unroll
    for (int a = 0; a < K; ++a) {
      const double da = d * op.A64[c * K + a];
#pragma unroll
      for (int b = 0; b <= a; ++b) P[a * (a + 1) / 2 + b] += da * op.A64[c * K + b];
    }
  }
  const double wi = op.has_w ? op.w64[i] : 1.0;
  const double dg = op.diag64[i];
#pragma unroll
  for (int a = 0; a < K; ++a) P[a * (a + 1) / 2 + a] += op.tk2_64[a] * wi + op.tau64[a] * dg;
#pragma unroll
  for (int a = 0; a < K * (K + 1) / 2; ++a) blk[(size_t)a * ld + i] = P[a];
  BlockChol<K, double> f;
  block_chol_factor<K, double>(P, f);
#pragma unroll
  for (int a = 0; a < K; ++a) {
    fac[(size_t)a * ld + i] = f.s[a];
    fs32[(size_t)a * ld + i] = (float)f.s[a];
  }
#pragma unroll
  for (int a = 0; a < K * (K + 1) / 2; ++a) fac[(size_t)(K + a) * ld + i] = f.l[a];
#pragma unroll
  for (int a = 0; a < K * (K + 1) / 2; a += 2) {
    const double hi = a + 1 < K * (K + 1) / 2 ? f.l[a + 1] : 0.0;
    fl16[(size_t)(a / 2) * ld + i] = __halves2half2(__double2half(f.l[a]), __double2half(hi));
  }
}

// Stand-alone operator apply Y = G X (eq. block-vector-mapping-matvec with Algorithm 1);
// grid-stride over pixels.
template <int K, int M, int E, typename T>
__global__ void __launch_bounds__(256, 4) k_apply(OpData op, const T* __restrict__ X,
                                               T* __restrict__ Y, int R) {
  __shared__ CtaShared<T, 1> sh;
  stage_operator<T, 1>(op, K, sh);
  __syncthreads();
  const int64_t ldu = op.ldu;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < op.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int r = 0; r < R; ++r) {
      const T* x = X + (size_t)r * K * ldu;
      T* y = Y + (size_t)r * K * ldu;
      T xi[K], acc[K];
#pragma unroll
      for (int j = 0; j < K; ++j) xi[j] = x[j * ldu + i];
      apply_pixel<K, M, E, T, T, 1>(op, sh, x, ldu, i, xi, acc);
#pragma unroll
      for (int j = 0; j < K; ++j) y[j * ldu + i] = acc[j];
    }
  }
}

// Per-block partial gradients (see sylv_backward); out layout [tau(k), kappa(k), beta(k)].
template <int K>
__global__ void __launch_bounds__(256) k_grad(OpData op, const double* __restrict__ X,
                                              const double* __restrict__ lam,
                                              const double* __restrict__ Y, int R,
                                              int want_beta, double* partial) {
  __shared__ double red[32 * 3 * K];
  const int64_t ld = op.ld, ldu = op.ldu;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < op.n;
  double g[3 * K];
#pragma unroll
  for (int t = 0; t < 3 * K; ++t) g[t] = 0.0;
  if (valid) {
    const double dg = op.diag64[i];
    const double wi = op.has_w ? op.w64[i] : 1.0;
    for (int r = 0; r < R; ++r) {
      const double* x = X + (size_t)r * K * ldu;
      const double* l = lam + (size_t)r * K * ldu;
      double xi[K], li[K], Lx[K];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        xi[j] = x[j * ldu + i];
        li[j] = l[j * ldu + i];
        Lx[j] = dg * xi[j];
      }
      for (int e = 0; e < op.E; ++e) {
        const int64_t c = op.ell_col[e * ld + i];
        const double v = op.ell_val64[e * ld + i];
#pragma unroll
        for (int j = 0; j < K; ++j) Lx[j] += v * x[j * ldu + c];
      }
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const double kap2 = op.kappa64[j] * op.kappa64[j];
        g[j] -= li[j] * (kap2 * wi * xi[j] + Lx[j]);
        g[K + j] -= 2.0 * op.tau64[j] * op.kappa64[j] * li[j] * wi * xi[j];
      }
      if (want_beta) {
        const double* y = Y + (size_t)r * op.m * ldu;
        for (int c = 0; c < op.m; ++c) {
          double t = 0.0, u = 0.0;
#pragma unroll
          for (int j = 0; j < K; ++j) {
            t += op.A64[c * K + j] * xi[j];
            u += op.A64[c * K + j] * li[j];
          }
          const double dc = op.D64[c * ld + i];
          const double yc = y[c * ldu + i];
#pragma unroll
          for (int j = 0; j < K; ++j)
            g[2 * K + j] += op.logf64[c] * op.A64[c * K + j] * dc *
                            (li[j] * yc - u * xi[j] - li[j] * t);
        }
      }
    }
  }
  block_sum<3 * K>(g, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int t = 0; t < 3 * K; ++t) partial[(size_t)blockIdx.x * 3 * K + t] = g[t];
  }
}

__global__ void k_grad_final(const double* __restrict__ partial, int ntiles, int nv,
                             double* out) {
  // one block; fixed-order sums
  __shared__ double red[32];
  for (int t = 0; t < nv; ++t) {
    double v[1] = {0.0};
    for (int b = threadIdx.x; b < ntiles; b += blockDim.x) v[0] += partial[(size_t)b * nv + t];
    block_sum<1>(v, red);
    if (threadIdx.x == 0) out[t] = v[0];
  }
}

__global__ void k_init_states(int ncols, const int* __restrict__ col_sys,
                              const int* __restrict__ col_rhs, const SysDesc* __restrict__ d,
                              Control* ctl) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    ctl->n_active = 0u;
    ctl->n_unfinished = (unsigned)ncols;
    ctl->error = 0u;
  }
  if (t >= ncols) return;
  ColState& cs = d[col_sys[t]].st[col_rhs[t]];
  cs.bnorm2 = 0.0;
  cs.rr64 = 0.0;
  cs.gamma = 0.0;
  cs.alpha = 0.0;
  cs.beta = 0.0;
  cs.rr_in0 = 0.0;
  cs.rr_in = 0.0;
  cs.thr_in = 0.0;
  cs.relres = 0.0;
  cs.phase = PH_START;
  cs.it = 0;
  cs.outer = 0;
  cs.status = SYLV_OK;
  cs.first = 1;
  cs.stop_after = 0;
  cs.dpend = 0;
  if (col_rhs[t] == 0) *d[col_sys[t]].counter = 0u;
}

// ------------------------------------------------------------------------------------------
cudaError_t launch_csr_check(const OpData& op, const int32_t* rowptr, const int32_t* col,
                             int64_t nnz, unsigned int* flags, unsigned int* maxdeg,
                             cudaStream_t s) {
  k_csr_check<<<blocks_for(op.n, SETUP_BLOCK), SETUP_BLOCK, 0, s>>>(op.n, rowptr, col, nnz,
                                                                    flags, maxdeg);
  return cudaGetLastError();
}

cudaError_t launch_ell_build(const OpData& op, const int32_t* rowptr, const int32_t* col,
                             const double* val, int32_t* ell_col, float* ell_val32,
                             double* ell_val64, float* diag32, double* diag64, int E,
                             cudaStream_t s) {
  k_ell_build<<<blocks_for(op.n, SETUP_BLOCK), SETUP_BLOCK, 0, s>>>(
      op.n, op.ld, rowptr, col, val, E, ell_col, ell_val32, ell_val64, diag32, diag64);
  return cudaGetLastError();
}

cudaError_t launch_square_count(const OpData& op, unsigned int* width, cudaStream_t s) {
  k_square_count<<<blocks_for(op.n, SETUP_BLOCK), SETUP_BLOCK, 0, s>>>(
      op.n, op.ld, op.E, op.ell_col, op.ell_val64, op.diag64, width);
  return cudaGetLastError();
}

cudaError_t launch_square_fill(const OpData& op, int E2, int32_t* sq_col, float* sq_val32,
                               double* sq_val64, float* sq_diag32, double* sq_diag64,
                               cudaStream_t s) {
  k_square_fill<<<blocks_for(op.n, SETUP_BLOCK), SETUP_BLOCK, 0, s>>>(
      op.n, op.ld, op.E, op.ell_col, op.ell_val64, op.diag64, E2, sq_col, sq_val32, sq_val64,
      sq_diag32, sq_diag64);
  return cudaGetLastError();
}

cudaError_t launch_var_accum(const OpData& op, const double* Z, const double* X, int R,
                             double* num, double* den, cudaStream_t s) {
  const int64_t tot = (int64_t)op.k * op.n;
  k_var_accum<<<blocks_for(tot, SETUP_BLOCK), SETUP_BLOCK, 0, s>>>(op.n, op.k, op.ldu, op.ld, Z, X,
                                                                   R, num, den);
  return cudaGetLastError();
}

cudaError_t launch_probe_fill(const OpData& op, const int32_t* colour, int ncol, int p0, int R,
                              double* Z, unsigned int* flag, cudaStream_t s) {
  k_probe_fill<<<blocks_for(op.n, SETUP_BLOCK), SETUP_BLOCK, 0, s>>>(op.n, op.k, op.ldu, colour,
                                                                     ncol, p0, R, Z, flag);
  return cudaGetLastError();
}

cudaError_t launch_var_finish(const OpData& op, const double* num, const double* den,
                              double* var, cudaStream_t s) {
  const int64_t tot = (int64_t)op.k * op.n;
  k_var_finish<<<blocks_for(tot, SETUP_BLOCK), SETUP_BLOCK, 0, s>>>(op.n, op.k, op.ldu, op.ld, num,
                                                                    den, var);
  return cudaGetLastError();
}

cudaError_t launch_convert_check(const double* src, int64_t rows, int64_t n, int64_t ld_src,
                                 int64_t ld_dst, float* dst32, double* dst64, int positive,
                                 unsigned int* flags, cudaStream_t s) {
  const int64_t tot = rows * n;
  if (tot == 0) return cudaSuccess;
  k_convert_check<<<blocks_for(tot, SETUP_BLOCK), SETUP_BLOCK, 0, s>>>(
      src, rows, n, ld_src, ld_dst, dst32, dst64, positive, flags);
  return cudaGetLastError();
}

cudaError_t launch_block_setup(const OpData& op, double* blk64, double* fac64, float* fs32,
                               __half2* fl16, cudaStream_t s) {
  const int nb = blocks_for(op.n, 256);
#define CALL(K) k_block_setup<K><<<nb, 256, 0, s>>>(op, blk64, fac64, fs32, fl16)
  SYLV_DISPATCH_K(op.k, CALL)
#undef CALL
  return cudaGetLastError();
}

cudaError_t launch_split_hl(const double* src, int64_t rows, int64_t ld, float* dst,
                            unsigned int* flag, cudaStream_t s) {
  const int64_t total = rows * ld;
  if (total == 0) return cudaSuccess;
  k_split_hl<<<blocks_for(total, SETUP_BLOCK), SETUP_BLOCK, 0, s>>>(src, total, total, dst,
                                                                    flag);
  return cudaGetLastError();
}

cudaError_t launch_rhs(const OpData& op, const double* Y, double* B, int R, cudaStream_t s) {
  return launch_rhs_range(op, Y, B, R, 0, op.n, s);
}

cudaError_t launch_rhs_range(const OpData& op, const double* Y, double* B, int R, int64_t i0,
                             int64_t i1, cudaStream_t s) {
  if (i1 <= i0) return cudaSuccess;
  k_rhs<<<blocks_for(i1 - i0, SETUP_BLOCK), SETUP_BLOCK, 0, s>>>(op, Y, B, R, i0, i1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply(const OpData& op, const T* X, T* Y, int R, cudaStream_t s) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  const int nb = (int)std::min<int64_t>(blocks_for(op.n, 256), (int64_t)nsm * 8);
  const int k = op.k, m = op.m, e = op.E;
#define CALL(K, M, E) k_apply<K, M, E, T><<<nb, 256, 0, s>>>(op, X, Y, R)
  SYLV_DISPATCH_SHAPE(k, m, e)
#undef CALL
  return cudaGetLastError();
}
template cudaError_t launch_apply<float>(const OpData&, const float*, float*, int,
                                         cudaStream_t);
template cudaError_t launch_apply<double>(const OpData&, const double*, double*, int,
                                          cudaStream_t);

cudaError_t launch_grad(const OpData& op, const double* X, const double* lam, const double* Y,
                        int R, int want_beta, double* partial, int ntiles, double* out,
                        cudaStream_t s) {
#define CALL(K) k_grad<K><<<ntiles, 256, 0, s>>>(op, X, lam, Y, R, want_beta, partial)
  SYLV_DISPATCH_K(op.k, CALL)
#undef CALL
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_grad_final<<<1, 256, 0, s>>>(partial, ntiles, 3 * op.k, out);
  return cudaGetLastError();
}

cudaError_t launch_init_states(int ncols, const int* col_sys, const int* col_rhs,
                               const SysDesc* d, Control* c, cudaStream_t s) {
  k_init_states<<<blocks_for(ncols, 128), 128, 0, s>>>(ncols, col_sys, col_rhs, d, c);
  return cudaGetLastError();
}

}  // namespace sylv
