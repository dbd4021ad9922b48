// Kernels of the preconditioned CG iteration and of the FP64 refinement loop.
//
// Per inner iteration two kernels run over every active system:
//
//   inner_apply:  d += alpha_prev p_old (the previous iteration's step),  p = z + beta p_old,
//                 q = G z + beta q   (= G p, since G p = G z + beta G p_old),
//                 partial sums of p . q; the last CTA of a system sets alpha = gamma / (p . q).
//   inner_update: r -= alpha q,  z = P^{-1} r (pixel-block Jacobi),
//                 partial sums of r . z and r . r; the last CTA sets beta, gamma and the
//                 stopping state.
//
// This is Algorithm 2 with a preconditioner, reordered so that the operator is applied to the
// freshly written z (no halo of the still-to-be-updated p is needed), the direction update
// p = z + beta p is folded into the operator kernel, and so is the solution step d += alpha p
// of the iteration before (both need the old p, which is then read once per iteration instead
// of twice).  When the inner solve ends on an update, that update's alpha p is added by
// update_x (ColState::dpend).  The operator application is the block
// mapping of eq. block-vector-mapping-matvec fused with the neighbour stencil of Algorithm 1:
//   (G X)_{j,i} = tau_j (kappa_j^2 w_i x_{j,i} + L_ii x_{j,i} + sum_e L_{i,col_e} x_{j,col_e})
//               + sum_c a_cj d_ci (a_c . x_i).
//
// The FP64 refinement loop adds two kernels: update_x (X += d [+ alpha p]) and residual (r = B - G X in
// FP64, r_in = r rounded to the inner type, d = 0, z = P^{-1} r_in), whose last CTA decides
// convergence of each column on the true FP64 residual.
//
// Work split: each system owns `nslots` CTAs (all resident at once); CTA `slot` handles tiles
// slot, slot + nslots, ... of blockDim.x consecutive pixels, keeps per-warp partial sums in
// shared memory, writes one partial per column at the end, and the last of the system's CTAs
// to finish (atomic counter, no waiting) reduces the nslots partials in a fixed order.  The
// staged FP32 pair with one or two columns instead lets every CTA of the next kernel form the
// sums (pcg_tma.cuh); the state changes are the same functions in both cases.
#pragma once

#include <cmath>
#include <cstdint>

#include "sylv_internal.cuh"

namespace sylv {

template <typename T> struct OpT;
template <> struct OpT<float> {
  static __device__ __forceinline__ const float* val(const OpData& o) { return o.ell_val32; }
  static __device__ __forceinline__ const float* diag(const OpData& o) { return o.diag32; }
  static __device__ __forceinline__ const float* D(const OpData& o) { return o.D32; }
  static __device__ __forceinline__ const float* w(const OpData& o) { return o.w32; }
  static __device__ __forceinline__ float A(const OpData& o, int i) { return o.A32[i]; }
  static __device__ __forceinline__ float tau(const OpData& o, int j) { return o.tau32[j]; }
  static __device__ __forceinline__ float tk2(const OpData& o, int j) { return o.tk2_32[j]; }
};
template <> struct OpT<double> {
  static __device__ __forceinline__ const double* val(const OpData& o) { return o.ell_val64; }
  static __device__ __forceinline__ const double* diag(const OpData& o) { return o.diag64; }
  static __device__ __forceinline__ const double* D(const OpData& o) { return o.D64; }
  static __device__ __forceinline__ const double* w(const OpData& o) { return o.w64; }
  static __device__ __forceinline__ double A(const OpData& o, int i) { return o.A64[i]; }
  static __device__ __forceinline__ double tau(const OpData& o, int j) { return o.tau64[j]; }
  static __device__ __forceinline__ double tk2(const OpData& o, int j) { return o.tk2_64[j]; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// Sums NV values over the CTA; the result is valid in thread 0.  smem: 32 * NV doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int t = 0; t < NV; ++t) v[t] = warp_sum(v[t]);
  if (lane == 0) {
#pragma unroll
    for (int t = 0; t < NV; ++t) smem[warp * NV + t] = v[t];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      double x = lane < nw ? smem[lane * NV + t] : 0.0;
      v[t] = warp_sum(x);
    }
  }
  __syncthreads();
}

// Mixing rows, prior scalars and per-column state of one system, staged in shared memory.
// Rows of A are padded to 8 entries so a row is read with one or two 16-byte loads.
template <typename T, int NV>
struct CtaShared {
  alignas(16) T A[MMAX][8];
  alignas(16) T tau[8];
  alignas(16) T tk2[8];
  T sc[RMAX];        // per-column scalar (beta or alpha)
  T sc2[RMAX];       // second per-column scalar (the operator kernels: the last alpha)
  int act[RMAX];     // column takes part in this kernel
  int aux[RMAX];     // per-column flag (first iteration)
  double wacc[RMAX][MAX_WARPS][NV];  // per-warp partial sums
  double red[32 * NV];
  int flag;
};

template <typename T, int NV>
__device__ __forceinline__ void stage_operator(const OpData& op, int K, CtaShared<T, NV>& sh) {
  for (int t = threadIdx.x; t < MMAX * 8; t += blockDim.x) {
    const int c = t >> 3, j = t & 7;
    sh.A[c][j] = (c < op.m && j < K) ? OpT<T>::A(op, c * K + j) : T(0);
  }
  if (threadIdx.x < 8) {
    const int j = threadIdx.x;
    sh.tau[j] = j < K ? OpT<T>::tau(op, j) : T(0);
    sh.tk2[j] = j < K ? OpT<T>::tk2(op, j) : T(0);
  }
}

template <typename T, int NV>
__device__ __forceinline__ void zero_wacc(CtaShared<T, NV>& sh, int R) {
  const int nw = blockDim.x >> 5;
  for (int t = threadIdx.x; t < R * nw * NV; t += blockDim.x) {
    const int r = t / (nw * NV), rem = t - r * nw * NV;
    sh.wacc[r][rem / NV][rem % NV] = 0.0;
  }
}

// Reads K entries of a padded row with 16-byte shared-memory loads.
template <int K, typename T>
__device__ __forceinline__ void load_row(const T* row, T (&a)[K]) {
  constexpr int V = 16 / sizeof(T);
#pragma unroll
  for (int q = 0; q < (K + V - 1) / V; ++q) {
    if constexpr (sizeof(T) == 4) {
      const float4 v = *reinterpret_cast<const float4*>(row + 4 * q);
      const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (4 * q + t < K) a[4 * q + t] = vv[t];
    } else {
      const double2 v = *reinterpret_cast<const double2*>(row + 2 * q);
      const double vv[2] = {v.x, v.y};
#pragma unroll
      for (int t = 0; t < 2; ++t)
        if (2 * q + t < K) a[2 * q + t] = vv[t];
    }
  }
}

// acc = (G x)_i for one column: x points at the column's k x ldx block, xi holds x at pixel i.
// M and E are the number of channels and the ELL width when known at compile time (0: read
// from op, loaded in batches of 4 at clamped, always valid addresses so that a batch of loads
// is issued together).
template <int K, int M, int E, typename T, typename TX, int NV>
__device__ __forceinline__ void apply_pixel(const OpData& op, const CtaShared<T, NV>& sh,
                                            const TX* __restrict__ x, int64_t ldx, int64_t i,
                                            const T (&xi)[K], T (&acc)[K]) {
  const int64_t ld = op.ld;
  constexpr int EC = E > 0 ? E : 4;
  constexpr int MC = M > 0 ? M : 4;
  const int Er = E > 0 ? E : op.E;
  const int Mr = M > 0 ? M : op.m;
  const T dg = __ldg(OpT<T>::diag(op) + i);
  const T wi = op.has_w ? __ldg(OpT<T>::w(op) + i) : T(1);
  T lap[K];
#pragma unroll
  for (int j = 0; j < K; ++j) lap[j] = dg * xi[j];
  for (int e0 = 0; e0 < Er; e0 += EC) {
    int64_t col[EC];
    T val[EC];
#pragma unroll
    for (int t = 0; t < EC; ++t) {
      const int e = E > 0 ? t : min(e0 + t, Er - 1);
      col[t] = __ldg(op.ell_col + e * ld + i);
      val[t] = __ldg(OpT<T>::val(op) + e * ld + i);
      if (E == 0 && e0 + t >= Er) val[t] = T(0);
    }
#pragma unroll
    for (int t = 0; t < EC; ++t)
#pragma unroll
      for (int j = 0; j < K; ++j) lap[j] += val[t] * T(x[j * ldx + col[t]]);
  }
#pragma unroll
  for (int j = 0; j < K; ++j) acc[j] = sh.tk2[j] * wi * xi[j] + sh.tau[j] * lap[j];
  for (int c0 = 0; c0 < Mr; c0 += MC) {
    T dv[MC];
#pragma unroll
    for (int t = 0; t < MC; ++t) {
      const int c = M > 0 ? t : min(c0 + t, Mr - 1);
      dv[t] = __ldg(OpT<T>::D(op) + c * ld + i);
      if (M == 0 && c0 + t >= Mr) dv[t] = T(0);
    }
#pragma unroll
    for (int t = 0; t < MC; ++t) {
      T a[K];
      load_row<K, T>(sh.A[c0 + t], a);   // rows past m are zero
      T u = T(0);
#pragma unroll
      for (int j = 0; j < K; ++j) u += a[j] * xi[j];
      u *= dv[t];
#pragma unroll
      for (int j = 0; j < K; ++j) acc[j] += a[j] * u;
    }
  }
}

// Pixel-block Jacobi preconditioner: P = diag_j(tau_j (kappa_j^2 w + L_ii)) + sum_c d_c a_c a_c^T
// (the exact k x k diagonal block of G at the pixel).  It is factored as P = S C C^T S with
// S = diag(P_jj)^{-1/2} (symmetric scaling first, so that badly scaled mixing columns do not
// cost precision) and C lower triangular; pivots are kept positive, so the preconditioner is
// SPD even where rounding makes the scaled block look singular.  The factor is computed once
// per handle in FP64 (k_block_setup); the FP64 iteration uses it as is, the FP32 iteration
// uses the scaling in FP32 and C in FP16 (off-diagonal entries of C lie in [-1, 1], its
// stored inverted diagonal in [1, 1e3]).  Applying the rounded factor is applying the exact
// inverse of another SPD matrix close to P, so PCG stays a valid PCG.
template <int K, typename T>
struct BlockChol {
  T s[K];                // scaling
  T l[K * (K + 1) / 2];  // packed lower factor, row-major; diagonal entries stored inverted
};

// Factors a packed SPD block P (row-major lower triangle) into f; P is overwritten.  The
// reciprocal square roots use the device rsqrt (a preconditioner needs no correctly rounded
// division or square root; both sides of PCG use the same factor).
template <int K, typename T>
__device__ __forceinline__ void block_chol_factor(T (&P)[K * (K + 1) / 2], BlockChol<K, T>& f) {
#pragma unroll
  for (int u = 0; u < K; ++u) {
    const T pu = P[u * (u + 1) / 2 + u];
    f.s[u] = pu > T(0) ? rsqrt(pu) : T(1);
  }
#pragma unroll
  for (int u = 0; u < K; ++u)
#pragma unroll
    for (int v = 0; v <= u; ++v) P[u * (u + 1) / 2 + v] *= f.s[u] * f.s[v];
  const T floor_piv = sizeof(T) == 4 ? T(1e-6) : T(1e-14);
#pragma unroll
  for (int u = 0; u < K; ++u) {
#pragma unroll
    for (int v = 0; v <= u; ++v) {
      T x = P[u * (u + 1) / 2 + v];
#pragma unroll
      for (int c = 0; c < v; ++c) x -= f.l[u * (u + 1) / 2 + c] * f.l[v * (v + 1) / 2 + c];
      if (u == v) {
        x = x > floor_piv ? x : floor_piv;
        f.l[u * (u + 1) / 2 + u] = rsqrt(x);
      } else {
        f.l[u * (u + 1) / 2 + v] = x * f.l[v * (v + 1) / 2 + v];
      }
    }
  }
}

template <int K, typename T>
__device__ __forceinline__ void block_solve(const BlockChol<K, T>& f, const T (&r)[K],
                                            T (&z)[K]) {
  T y[K];
#pragma unroll
  for (int a = 0; a < K; ++a) {
    T v = r[a] * f.s[a];
#pragma unroll
    for (int c = 0; c < a; ++c) v -= f.l[a * (a + 1) / 2 + c] * y[c];
    y[a] = v * f.l[a * (a + 1) / 2 + a];
  }
#pragma unroll
  for (int a = K - 1; a >= 0; --a) {
    T v = y[a];
#pragma unroll
    for (int c = a + 1; c < K; ++c) v -= f.l[c * (c + 1) / 2 + a] * z[c];
    z[a] = v * f.l[a * (a + 1) / 2 + a];
  }
#pragma unroll
  for (int a = 0; a < K; ++a) z[a] *= f.s[a];
}

// FP64 operator from the precomputed pixel blocks: acc = P_i x_i + sum_j tau_j (L_off x_j)_i,
// i.e. the same G x as apply_pixel with the pixel-local terms gathered into one k x k block
// (k(k+1) FMAs instead of m(2k+1) + 2k; FP64 is the scarce unit on this GPU).
template <int K, int E, typename TX, int NV>
__device__ __forceinline__ void apply_pixel_blk64(const OpData& op,
                                                  const CtaShared<double, NV>& sh,
                                                  const TX* __restrict__ x, int64_t ldx,
                                                  int64_t i, const double (&xi)[K],
                                                  double (&acc)[K]) {
  const int64_t ld = op.ld;
  constexpr int EC = E > 0 ? E : 4;
  const int Er = E > 0 ? E : op.E;
#pragma unroll
  for (int a = 0; a < K; ++a) acc[a] = 0.0;
#pragma unroll
  for (int a = 0; a < K; ++a) {
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      const double pab = __ldg(op.blk64 + (size_t)(a * (a + 1) / 2 + b) * ld + i);
      acc[a] += pab * xi[b];
      if (b != a) acc[b] += pab * xi[a];
    }
  }
  double lap[K];
#pragma unroll
  for (int j = 0; j < K; ++j) lap[j] = 0.0;
  for (int e0 = 0; e0 < Er; e0 += EC) {
    int64_t col[EC];
    double val[EC];
#pragma unroll
    for (int t = 0; t < EC; ++t) {
      const int e = E > 0 ? t : min(e0 + t, Er - 1);
      col[t] = __ldg(op.ell_col + e * ld + i);
      val[t] = __ldg(op.ell_val64 + e * ld + i);
      if (E == 0 && e0 + t >= Er) val[t] = 0.0;
    }
#pragma unroll
    for (int t = 0; t < EC; ++t)
#pragma unroll
      for (int j = 0; j < K; ++j) lap[j] += val[t] * double(x[j * ldx + col[t]]);
  }
#pragma unroll
  for (int j = 0; j < K; ++j) acc[j] += sh.tau[j] * lap[j];
}

// Loads the precomputed FP64 factor of the pixel block (see block_chol).
template <int K>
__device__ __forceinline__ void load_factor64(const OpData& op, int64_t i,
                                              BlockChol<K, double>& f) {
  const int64_t ld = op.ld;
#pragma unroll
  for (int a = 0; a < K; ++a) f.s[a] = __ldg(op.fac64 + (size_t)a * ld + i);
#pragma unroll
  for (int a = 0; a < K * (K + 1) / 2; ++a) f.l[a] = __ldg(op.fac64 + (size_t)(K + a) * ld + i);
}

// Loads the stored FP32 preconditioner of the pixel: FP32 scaling and FP16 factor.
template <int K>
__device__ __forceinline__ void load_factor32(const OpData& op, int64_t i,
                                              BlockChol<K, float>& f) {
  const int64_t ld = op.ld;
#pragma unroll
  for (int a = 0; a < K; ++a) f.s[a] = __ldg(op.fs32 + (size_t)a * ld + i);
#pragma unroll
  for (int a = 0; a < K * (K + 1) / 2; a += 2) {
    const float2 v = __half22float2(op.fl16[(size_t)(a / 2) * ld + i]);
    f.l[a] = v.x;
    if (a + 1 < K * (K + 1) / 2) f.l[a + 1] = v.y;
  }
}

// Adds this warp's share of NV sums of column r into the CTA's per-warp accumulators.
template <typename T, int NV>
__device__ __forceinline__ void warp_accumulate(CtaShared<T, NV>& sh, int r,
                                                const double (&v)[NV]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    const double s = warp_sum(v[t]);
    if (lane == 0) sh.wacc[r][warp][t] += s;
  }
}

__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// The same as warp_accumulate for FP32 values: the 32 lanes are summed in FP32 (a fixed tree)
// and lane 0 adds the warp's sum to the FP64 accumulator, so the FP64 unit (1/64 of the FP32
// rate on this GPU) sees one conversion and one addition per warp instead of a tree per lane.
template <typename T, int NV>
__device__ __forceinline__ void warp_accumulate_f32(CtaShared<T, NV>& sh, int r,
                                                    const float (&v)[NV]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    const float s = warp_sum_f32(v[t]);
    if (lane == 0) sh.wacc[r][warp][t] += double(s);
  }
}

// Column state after an inner operator kernel with total p . q: alpha, or the end of the inner
// solve (exact solution reached, or breakdown).  `count` keeps the active/unfinished counters.
__device__ __forceinline__ void after_apply(ColState& cs, double pq, Control* ctl, bool count) {
  if (pq > 0.0 && isfinite(pq)) {
    cs.alpha = cs.gamma / pq;
    cs.first = 0;
  } else if (cs.rr_in == 0.0) {
    cs.phase = PH_INNER_DONE;  // exact solution: nothing left to do
    if (count) atomicSub(&ctl->n_active, 1u);
  } else {
    cs.phase = PH_FAILED;
    cs.status = SYLV_E_BREAKDOWN;
    if (count) {
      atomicSub(&ctl->n_active, 1u);
      atomicSub(&ctl->n_unfinished, 1u);
    }
  }
}

// Column state after an inner update with totals r . z and r . r: beta and gamma, or the end of
// the inner solve (target reached, iteration cap, breakdown).
__device__ __forceinline__ void after_update(ColState& cs, double rz, double rr, Control* ctl,
                                             bool count) {
  cs.it += 1;
  cs.rr_in = rr;
  if (!isfinite(rz) || !isfinite(rr)) {
    cs.phase = PH_FAILED;
    cs.status = SYLV_E_BREAKDOWN;
    if (count) {
      atomicSub(&ctl->n_active, 1u);
      atomicSub(&ctl->n_unfinished, 1u);
    }
  } else if (rr <= cs.thr_in || rr == 0.0) {
    cs.phase = PH_INNER_DONE;
    cs.dpend = 1;
    if (count) atomicSub(&ctl->n_active, 1u);
  } else if (!(rz > 0.0)) {
    cs.phase = PH_FAILED;
    cs.status = SYLV_E_BREAKDOWN;
    if (count) {
      atomicSub(&ctl->n_active, 1u);
      atomicSub(&ctl->n_unfinished, 1u);
    }
  } else if (cs.it >= ctl->maxit) {
    cs.phase = PH_INNER_DONE;
    cs.dpend = 1;
    cs.stop_after = 1;
    if (count) atomicSub(&ctl->n_active, 1u);
  } else {
    cs.beta = rz / cs.gamma;
    cs.gamma = rz;
  }
}

// Column state after an FP64 residual with totals ||r64||^2, ||B||^2, r.z, r.r (inner type):
// converged, capped, failed, or the start of an inner solve with its target.
__device__ __forceinline__ void after_residual(ColState& cs, const double (&t)[4], Control* ctl) {
  const double rr64 = t[0], rz = t[2], rr = t[3];
  if (cs.phase == PH_START) cs.bnorm2 = t[1];
  cs.rr64 = rr64;
  const double den = cs.bnorm2 > 0.0 ? cs.bnorm2 : 1.0;
  const double rel2 = rr64 / den;
  cs.relres = sqrt(rel2);
  const bool capped = cs.stop_after || cs.it >= ctl->maxit || cs.outer >= ctl->max_outer;
  if (!isfinite(rr64)) {
    cs.phase = PH_FAILED;
    cs.status = SYLV_E_BREAKDOWN;
    atomicSub(&ctl->n_unfinished, 1u);
  } else if (rel2 <= ctl->tol2) {
    cs.phase = PH_CONVERGED;
    cs.status = SYLV_OK;
    atomicSub(&ctl->n_unfinished, 1u);
  } else if (capped) {
    cs.phase = PH_FAILED;
    cs.status = SYLV_E_NOT_CONVERGED;
    atomicSub(&ctl->n_unfinished, 1u);
  } else if (!(rz > 0.0) || !isfinite(rz)) {
    cs.phase = PH_FAILED;
    cs.status = SYLV_E_BREAKDOWN;
    atomicSub(&ctl->n_unfinished, 1u);
  } else {
    // inner target: the reduction still needed (with a safety margin), but no finer than the
    // inner precision can deliver in one refinement step
    const double need = ctl->tol2 * ctl->safety2 * den / rr64;
    const double fac = need > ctl->tol_in2 ? need : ctl->tol_in2;
    cs.phase = PH_INNER;
    cs.first = 1;
    cs.dpend = 0;
    cs.gamma = rz;
    cs.rr_in0 = rr;
    cs.rr_in = rr;
    cs.thr_in = fac * rr;
    cs.outer += 1;
    atomicAdd(&ctl->n_active, 1u);
  }
}

// This CTA's per-column partials (sum of the per-warp sums), no arrival.
template <typename T, int NV>
__device__ __forceinline__ void write_cta_partials(double* dst, int slot, CtaShared<T, NV>& sh,
                                                   int R) {
  const int nw = blockDim.x >> 5;
  __syncthreads();
  for (int t = threadIdx.x; t < R * NV; t += blockDim.x) {
    const int r = t / NV, v = t - r * NV;
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh.wacc[r][w][v];
    dst[((size_t)slot * R + r) * NPART + v] = s;
  }
}

// Writes this CTA's partials, then returns true in the last CTA of the system to arrive, which
// then holds the fixed-order totals of every active column in sh.red[r * NV + t] (thread 0).
template <typename T, int NV>
__device__ __forceinline__ bool finish_partials(const SysDesc& sd, int slot, int nslots,
                                                CtaShared<T, NV>& sh, int R,
                                                double (&tot)[RMAX][NV]) {
  const int nw = blockDim.x >> 5;
  __syncthreads();
  for (int t = threadIdx.x; t < R * NV; t += blockDim.x) {
    const int r = t / NV, v = t - r * NV;
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh.wacc[r][w][v];
    sd.partial[((size_t)slot * R + r) * NPART + v] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(sd.counter, 1u);
    sh.flag = (prev == (unsigned)nslots - 1u) ? 1 : 0;
  }
  __syncthreads();
  if (!sh.flag) return false;
  __threadfence();
  for (int r = 0; r < R; ++r) {
    if (!sh.act[r]) continue;
    double acc[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) acc[t] = 0.0;
    for (int sl = threadIdx.x; sl < nslots; sl += blockDim.x) {
      const double* p = sd.partial + ((size_t)sl * R + r) * NPART;
#pragma unroll
      for (int t = 0; t < NV; ++t) acc[t] += __ldcg(p + t);
    }
    block_sum<NV>(acc, sh.red);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int t = 0; t < NV; ++t) tot[r][t] = acc[t];
    }
  }
  return true;
}

// ---------------------------------------------------------------------------------------------
// inner_apply: d += alpha p (the previous iteration's step, deferred to here so that p is read
// once per iteration), p = z + beta p, q = G z + beta q, partial p . q
// ---------------------------------------------------------------------------------------------
// FP32 instances are held to 64 registers (4 CTAs of 256 per SM); FP64 ones, whose
// preconditioner factor alone needs ~60 registers, to 128.
template <int K, int M, int E, typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2)
k_inner_apply(const SysDesc* __restrict__ descs, const CtaRef* __restrict__ ctas, Control* ctl) {
  __shared__ CtaShared<T, 1> sh;
  const CtaRef cr = ctas[blockIdx.x];
  if (cr.sys < 0) return;  // idle CTA of a reassigned launch
  const SysDesc& sd = descs[cr.sys];
  const OpData& op = sd.op;
  const int R = sd.R;
  int act = 0;
  if (threadIdx.x < RMAX) {
    const int r = threadIdx.x;
    if (r < R) {
      const ColState& cs = sd.st[r];
      act = cs.phase == PH_INNER;
      sh.sc[r] = T(cs.beta);
      sh.sc2[r] = T(cs.alpha);
      sh.aux[r] = cs.first;
    }
    sh.act[r] = act;
  }
  stage_operator<T, 1>(op, K, sh);
  zero_wacc<T, 1>(sh, R);
  if (!__syncthreads_or(act)) return;

  const int64_t ld = op.ld, n = op.n;
  for (int tile = cr.slot; tile < sd.ntiles; tile += sd.nslots[0]) {
    const int64_t i0 = (int64_t)tile * blockDim.x + threadIdx.x;
    const bool valid = i0 < n;
    const int64_t i = valid ? i0 : 0;
    for (int r = 0; r < R; ++r) {
      if (!sh.act[r]) continue;
      const size_t off = (size_t)r * K * ld;
      const T* z = (const T*)sd.vz + off;
      T* p = (T*)sd.vp + off;
      T* q = (T*)sd.vq + off;
      T* d = (T*)sd.vd + off;
      T zi[K], w[K];
#pragma unroll
      for (int j = 0; j < K; ++j) zi[j] = z[j * ld + i];
      if constexpr (sizeof(T) == 8) {
        apply_pixel_blk64<K, E, T, 1>(op, sh, z, ld, i, zi, w);
      } else {
        apply_pixel<K, M, E, T, T, 1>(op, sh, z, ld, i, zi, w);
      }
      T pq = T(0);
      if (valid) {
        const T beta = sh.sc[r], alpha = sh.sc2[r];
        const bool first = sh.aux[r] != 0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
          T pj = zi[j], qj = w[j];
          if (!first) {
            const T po = p[j * ld + i];
            d[j * ld + i] += alpha * po;   // the previous iteration's d += alpha p
            pj += beta * po;
            qj += beta * q[j * ld + i];
          }
          p[j * ld + i] = pj;
          q[j * ld + i] = qj;
          pq += pj * qj;
        }
      }
      if constexpr (sizeof(T) == 4) {
        const float v[1] = {float(pq)};
        warp_accumulate_f32<T, 1>(sh, r, v);
      } else {
        const double v[1] = {double(pq)};
        warp_accumulate<T, 1>(sh, r, v);
      }
    }
  }
  double tot[RMAX][1];
  if (!finish_partials<T, 1>(sd, cr.slot, sd.nslots[0], sh, R, tot)) return;
  if (threadIdx.x == 0) {
    for (int r = 0; r < R; ++r)
      if (sh.act[r]) after_apply(sd.st[r], tot[r][0], ctl, true);
    *sd.counter = 0u;
  }
}

// ---------------------------------------------------------------------------------------------
// inner_update: r -= alpha q, z = P^{-1} r, partial r . z and r . r (d += alpha p is left to
// the next operator kernel, or to k_update_x when the inner solve ends here)
// ---------------------------------------------------------------------------------------------
template <int K, int M, int E, typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2)
k_inner_update(const SysDesc* __restrict__ descs, const CtaRef* __restrict__ ctas,
               Control* ctl) {
  __shared__ CtaShared<T, 2> sh;
  const CtaRef cr = ctas[blockIdx.x];
  if (cr.sys < 0) return;  // idle CTA of a reassigned launch
  const SysDesc& sd = descs[cr.sys];
  const OpData& op = sd.op;
  const int R = sd.R;
  int act = 0;
  if (threadIdx.x < RMAX) {
    const int r = threadIdx.x;
    if (r < R) {
      const ColState& cs = sd.st[r];
      act = cs.phase == PH_INNER;
      sh.sc[r] = T(cs.alpha);
    }
    sh.act[r] = act;
  }
  stage_operator<T, 2>(op, K, sh);
  zero_wacc<T, 2>(sh, R);
  if (!__syncthreads_or(act)) return;

  const int64_t ld = op.ld, n = op.n;
  const bool prec = ctl->precond == SYLV_PRECOND_BLOCK_JACOBI;
  for (int tile = cr.slot; tile < sd.ntiles; tile += sd.nslots[1]) {
    const int64_t i0 = (int64_t)tile * blockDim.x + threadIdx.x;
    const bool valid = i0 < n;
    const int64_t i = valid ? i0 : 0;
    BlockChol<K, T> f;
    if (prec) {
      if constexpr (sizeof(T) == 8) {
        load_factor64<K>(op, i, f);
      } else {
        load_factor32<K>(op, i, f);
      }
    }
    for (int r = 0; r < R; ++r) {
      if (!sh.act[r]) continue;
      const size_t off = (size_t)r * K * ld;
      T* rv = (T*)sd.vr + off;
      T* z = (T*)sd.vz + off;
      const T* q = (const T*)sd.vq + off;
      const T alpha = sh.sc[r];
      T rz = T(0), rr = T(0);
      if (valid) {
        T ri[K], zi[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
          ri[j] = rv[j * ld + i] - alpha * q[j * ld + i];
          rv[j * ld + i] = ri[j];
        }
        if (prec) {
          block_solve<K, T>(f, ri, zi);
        } else {
#pragma unroll
          for (int j = 0; j < K; ++j) zi[j] = ri[j];
        }
#pragma unroll
        for (int j = 0; j < K; ++j) {
          z[j * ld + i] = zi[j];
          rz += ri[j] * zi[j];
          rr += ri[j] * ri[j];
        }
      }
      if constexpr (sizeof(T) == 4) {
        const float v[2] = {float(rz), float(rr)};
        warp_accumulate_f32<T, 2>(sh, r, v);
      } else {
        const double v[2] = {double(rz), double(rr)};
        warp_accumulate<T, 2>(sh, r, v);
      }
    }
  }
  double tot[RMAX][2];
  if (!finish_partials<T, 2>(sd, cr.slot, sd.nslots[1], sh, R, tot)) return;
  if (threadIdx.x == 0) {
    for (int r = 0; r < R; ++r)
      if (sh.act[r]) after_update(sd.st[r], tot[r][0], tot[r][1], ctl, true);
    *sd.counter = 0u;
  }
}

// ---------------------------------------------------------------------------------------------
// update_x: X += d for columns whose inner solve finished (with the last iteration's alpha p,
// in the inner type as the operator kernel would have added it, when the solve ended on an
// update)
// ---------------------------------------------------------------------------------------------
template <int K, typename T>
__global__ void __launch_bounds__(256)
k_update_x(const SysDesc* __restrict__ descs, const CtaRef* __restrict__ ctas) {
  const CtaRef cr = ctas[blockIdx.x];
  if (cr.sys < 0) return;  // idle CTA of a reassigned launch
  const SysDesc& sd = descs[cr.sys];
  const int64_t ld = sd.op.ld, ldu = sd.op.ldu, n = sd.op.n;
  for (int r = 0; r < sd.R; ++r) {
    const ColState& cs = sd.st[r];
    if (cs.phase != PH_INNER_DONE) continue;
    const bool pend = cs.dpend != 0;
    const T alpha = T(cs.alpha);
    const T* d = (const T*)sd.vd + (size_t)r * K * ld;
    const T* p = (const T*)sd.vp + (size_t)r * K * ld;
    double* X = sd.X + (size_t)r * K * ldu;
    for (int tile = cr.slot; tile < sd.ntiles; tile += sd.nslots[2]) {
      const int64_t i = (int64_t)tile * blockDim.x + threadIdx.x;
      if (i >= n) continue;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        T dj = d[j * ld + i];
        if (pend) dj += alpha * p[j * ld + i];
        X[j * ldu + i] += double(dj);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// residual: r64 = B - G X (FP64), r_in = r64 rounded, d = 0, z = P^{-1} r_in; decisions
// ---------------------------------------------------------------------------------------------
template <int K, int M, int E, typename T>
__global__ void __launch_bounds__(256)
k_residual(const SysDesc* __restrict__ descs, const CtaRef* __restrict__ ctas, Control* ctl) {
  __shared__ CtaShared<double, 4> sh;     // FP64 operator
  const CtaRef cr = ctas[blockIdx.x];
  if (cr.sys < 0) return;  // idle CTA of a reassigned launch
  const SysDesc& sd = descs[cr.sys];
  const OpData& op = sd.op;
  const int R = sd.R;
  int act = 0;
  if (threadIdx.x < RMAX) {
    const int r = threadIdx.x;
    int ph = PH_CONVERGED;
    if (r < R) {
      ph = sd.st[r].phase;
      act = (ph == PH_START || ph == PH_INNER_DONE);
    }
    sh.act[r] = act;
    sh.aux[r] = ph;
  }
  stage_operator<double, 4>(op, K, sh);
  zero_wacc<double, 4>(sh, R);
  if (!__syncthreads_or(act)) return;

  const int64_t ld = op.ld, n = op.n;
  const bool prec = ctl->precond == SYLV_PRECOND_BLOCK_JACOBI;
  const bool x0_zero = ctl->x0_zero != 0;
  for (int tile = cr.slot; tile < sd.ntiles; tile += sd.nslots[2]) {
    const int64_t i0 = (int64_t)tile * blockDim.x + threadIdx.x;
    const bool valid = i0 < n;
    const int64_t i = valid ? i0 : 0;
    BlockChol<K, T> f;
    if (prec) {
      if constexpr (sizeof(T) == 8) {
        load_factor64<K>(op, i, f);
      } else {
        load_factor32<K>(op, i, f);
      }
    }
    for (int r = 0; r < R; ++r) {
      if (!sh.act[r]) continue;
      const size_t off = (size_t)r * K * ld;
      const size_t offu = (size_t)r * K * op.ldu;
      const int64_t ldu = op.ldu;
      const double* X = sd.X + offu;
      const double* B = sd.B + offu;
      T* d = (T*)sd.vd + off;
      T* rv = (T*)sd.vr + off;
      T* z = (T*)sd.vz + off;
      double xi[K], gx[K];
      if (x0_zero && sh.aux[r] == PH_START) {
        // X = 0: the residual is B itself (no operator application needed)
#pragma unroll
        for (int j = 0; j < K; ++j) gx[j] = 0.0;
      } else {
#pragma unroll
        for (int j = 0; j < K; ++j) xi[j] = X[j * ldu + i];
        apply_pixel_blk64<K, E, double, 4>(op, sh, X, ldu, i, xi, gx);
      }
      double rr64 = 0.0, bb = 0.0, rz = 0.0, rr = 0.0;
      if (valid) {
        T ri[K], zi[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const double bj = B[j * ldu + i];
          const double r64 = bj - gx[j];
          rr64 += r64 * r64;
          bb += bj * bj;
          ri[j] = T(r64);
          rv[j * ld + i] = ri[j];
          d[j * ld + i] = T(0);
        }
        if (prec) {
          block_solve<K, T>(f, ri, zi);
        } else {
#pragma unroll
          for (int j = 0; j < K; ++j) zi[j] = ri[j];
        }
        T rzt = T(0), rrt = T(0);   // products in the inner type, like the inner kernels
#pragma unroll
        for (int j = 0; j < K; ++j) {
          z[j * ld + i] = zi[j];
          rzt += ri[j] * zi[j];
          rrt += ri[j] * ri[j];
        }
        rz = double(rzt);
        rr = double(rrt);
      }
      const double v[4] = {rr64, bb, rz, rr};
      warp_accumulate<double, 4>(sh, r, v);
    }
  }
  double tot[RMAX][4];
  if (!finish_partials<double, 4>(sd, cr.slot, sd.nslots[2], sh, R, tot)) return;
  if (threadIdx.x == 0) {
    for (int r = 0; r < R; ++r)
      if (sh.act[r]) after_residual(sd.st[r], tot[r], ctl);
    *sd.counter = 0u;
  }
}

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------
// Shapes with compile-time (k, m, E) kernels; every other shape uses the (k, 0, 0) kernels.
#define SYLV_SPECIAL_SHAPES(X) \
  X(3, 5, 4) X(4, 6, 4) X(4, 7, 4) X(5, 7, 4) X(6, 8, 4) X(6, 9, 4) X(4, 9, 12)

#define SYLV_IS_SPECIAL_(K_, M_, E_) || (k == K_ && m == M_ && e == E_)
inline bool special_shape(int k, int m, int e) {
  return false SYLV_SPECIAL_SHAPES(SYLV_IS_SPECIAL_);
}

// Calls CALL(K, M, E) for the kernel instance that serves shape (k, m, e).
#define SYLV_TRY_SPECIAL_(K_, M_, E_) \
  if (!done && k == K_ && m == M_ && e == E_) { CALL(K_, M_, E_); done = true; }
#define SYLV_DISPATCH_SHAPE(k, m, e)                     \
  bool done = false;                                     \
  SYLV_SPECIAL_SHAPES(SYLV_TRY_SPECIAL_)                 \
  if (!done) {                                           \
    switch (k) {                                         \
      case 1: CALL(1, 0, 0); break;                      \
      case 2: CALL(2, 0, 0); break;                      \
      case 3: CALL(3, 0, 0); break;                      \
      case 4: CALL(4, 0, 0); break;                      \
      case 5: CALL(5, 0, 0); break;                      \
      case 6: CALL(6, 0, 0); break;                      \
      case 7: CALL(7, 0, 0); break;                      \
      case 8: CALL(8, 0, 0); break;                      \
      default: return cudaErrorInvalidValue;             \
    }                                                    \
  }

#define SYLV_DISPATCH_K(k, CALL)           \
  switch (k) {                             \
    case 1: CALL(1); break;                \
    case 2: CALL(2); break;                \
    case 3: CALL(3); break;                \
    case 4: CALL(4); break;                \
    case 5: CALL(5); break;                \
    case 6: CALL(6); break;                \
    case 7: CALL(7); break;                \
    case 8: CALL(8); break;                \
    default: return cudaErrorInvalidValue; \
  }

template <typename T>
cudaError_t launch_inner_apply_impl(int k, int m, int e, int ncta, int block,
                                    const SysDesc* d, const CtaRef* c, Control* ctl,
                                    cudaStream_t s) {
  if (ncta <= 0) return cudaSuccess;
#define CALL(K, M, E) k_inner_apply<K, M, E, T><<<ncta, block, 0, s>>>(d, c, ctl)
  SYLV_DISPATCH_SHAPE(k, m, e)
#undef CALL
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_inner_update_impl(int k, int m, int e, int ncta, int block,
                                     const SysDesc* d, const CtaRef* c, Control* ctl,
                                     cudaStream_t s) {
  if (ncta <= 0) return cudaSuccess;
#define CALL(K, M, E) k_inner_update<K, M, E, T><<<ncta, block, 0, s>>>(d, c, ctl)
  SYLV_DISPATCH_SHAPE(k, m, e)
#undef CALL
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual_impl(int k, int m, int e, int ncta, int block, const SysDesc* d,
                                 const CtaRef* c, Control* ctl, cudaStream_t s) {
  if (ncta <= 0) return cudaSuccess;
#define CALL(K, M, E) k_residual<K, M, E, T><<<ncta, block, 0, s>>>(d, c, ctl)
  SYLV_DISPATCH_SHAPE(k, m, e)
#undef CALL
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update_x_impl(int k, int ncta, int block, const SysDesc* d, const CtaRef* c,
                                 cudaStream_t s) {
  if (ncta <= 0) return cudaSuccess;
#define CALL(K) k_update_x<K, T><<<ncta, block, 0, s>>>(d, c)
  SYLV_DISPATCH_K(k, CALL)
#undef CALL
  return cudaGetLastError();
}

// Resident CTAs per SM of the plain kernel `kind` (0 apply, 1 update, 2 residual).
template <typename T>
int occupancy_impl(int kind, int k, int m, int e, int block) {
  int nb = 0;
  auto take = [&](const void* fn) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, 0) != cudaSuccess) nb = 1;
  };
  auto body = [&]() -> cudaError_t {
#define CALL(K, M, E)                                                     \
  do {                                                                    \
    if (kind == 0) take((const void*)k_inner_apply<K, M, E, T>);          \
    else if (kind == 1) take((const void*)k_inner_update<K, M, E, T>);    \
    else take((const void*)k_residual<K, M, E, T>);                       \
  } while (0)
    SYLV_DISPATCH_SHAPE(k, m, e)
#undef CALL
    return cudaSuccess;
  };
  body();
  return nb < 1 ? 1 : nb;
}

}  // namespace sylv
