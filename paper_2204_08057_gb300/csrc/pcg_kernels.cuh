// Kernels of the preconditioned CG iteration and of the FP64 refinement loop.
//
// Per inner iteration two kernels run over every tile of every active system:
//
//   inner_apply:  p = z + beta p,  q = G z + beta q   (= G p, since G p = G z + beta G p_old),
//                 partial sums of p . q; the last CTA of a system sets alpha = gamma / (p . q).
//   inner_update: d += alpha p,  r -= alpha q,  z = P^{-1} r (pixel-block Jacobi),
//                 partial sums of r . z and r . r; the last CTA sets beta, gamma and the
//                 stopping state.
//
// This is Algorithm 2 with a preconditioner, reordered so that the operator is applied to the
// freshly written z (no halo of the still-to-be-updated p is needed) and the direction update
// p = z + beta p is folded into the operator kernel.  The operator application is the block
// mapping of eq. block-vector-mapping-matvec fused with the neighbour stencil of Algorithm 1:
//   (G X)_{j,i} = tau_j (kappa_j^2 w_i x_{j,i} + L_ii x_{j,i} + sum_e L_{i,col_e} x_{j,col_e})
//               + sum_c a_cj d_ci (a_c . x_i).
//
// The FP64 refinement loop adds two kernels: update_x (X += d) and residual (r = B - G X in
// FP64, r_in = r rounded to the inner type, d = 0, z = P^{-1} r_in), whose last CTA decides
// convergence of each column on the true FP64 residual.
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

// Called by all threads after thread 0 wrote this CTA's partials.  True in the last CTA of
// the system to arrive; that CTA then owns the partials and resets the counter.
__device__ __forceinline__ bool arrive_last(unsigned int* counter, unsigned int total,
                                            int* s_flag) {
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    *s_flag = (prev == total - 1u) ? 1 : 0;
  }
  __syncthreads();
  const bool last = *s_flag != 0;
  if (last) __threadfence();
  return last;
}

// Fixed-order sum of partial value v of column r over the system's tiles (valid in thread 0).
template <int NV>
__device__ __forceinline__ void reduce_partials(const SysDesc& sd, int r, const int (&vidx)[NV],
                                                double (&out)[NV], double* smem) {
  double acc[NV];
#pragma unroll
  for (int t = 0; t < NV; ++t) acc[t] = 0.0;
  for (int tl = threadIdx.x; tl < sd.ntiles; tl += blockDim.x) {
    const double* p = sd.partial + ((size_t)tl * sd.R + r) * NPART;
#pragma unroll
    for (int t = 0; t < NV; ++t) acc[t] += __ldcg(p + vidx[t]);
  }
  block_sum<NV>(acc, smem);
#pragma unroll
  for (int t = 0; t < NV; ++t) out[t] = acc[t];
}

// Per-pixel operator data held in registers for the duration of a CTA.
template <typename T>
struct PixelOp {
  int col[EMAX];
  T val[EMAX];
  T dg;    // L_ii
  T wi;    // mass diagonal
  T dv[MMAX];
};

template <typename T>
__device__ __forceinline__ void load_pixel_op(const OpData& op, int64_t i, bool valid,
                                              bool need_lap, PixelOp<T>& po) {
  const int64_t ld = op.ld;
  if (need_lap) {
#pragma unroll
    for (int e = 0; e < EMAX; ++e) {
      if (e < op.E) {
        po.col[e] = valid ? __ldg(op.ell_col + e * ld + i) : 0;
        po.val[e] = valid ? __ldg(OpT<T>::val(op) + e * ld + i) : T(0);
      }
    }
  }
  po.dg = valid ? __ldg(OpT<T>::diag(op) + i) : T(0);
  po.wi = (op.has_w && valid) ? __ldg(OpT<T>::w(op) + i) : T(1);
#pragma unroll
  for (int c = 0; c < MMAX; ++c)
    if (c < op.m) po.dv[c] = valid ? __ldg(OpT<T>::D(op) + c * ld + i) : T(0);
}

// acc = G x at pixel i for one column: x points at the column's k x ld block.
template <int K, typename T, typename TX>
__device__ __forceinline__ void apply_pixel(const OpData& op, const PixelOp<T>& po,
                                            const T* s_A, const T* s_tau, const T* s_tk2,
                                            const TX* __restrict__ x, int64_t i,
                                            const T (&xi)[K], T (&acc)[K]) {
  const int64_t ld = op.ld;
  T lap[K];
#pragma unroll
  for (int j = 0; j < K; ++j) lap[j] = po.dg * xi[j];
#pragma unroll
  for (int e = 0; e < EMAX; ++e) {
    if (e < op.E) {
      const int64_t cidx = po.col[e];
      const T v = po.val[e];
#pragma unroll
      for (int j = 0; j < K; ++j) lap[j] += v * T(x[j * ld + cidx]);
    }
  }
#pragma unroll
  for (int j = 0; j < K; ++j) acc[j] = s_tk2[j] * po.wi * xi[j] + s_tau[j] * lap[j];
#pragma unroll
  for (int c = 0; c < MMAX; ++c) {
    if (c < op.m) {
      T t = T(0);
#pragma unroll
      for (int j = 0; j < K; ++j) t += s_A[c * K + j] * xi[j];
      t *= po.dv[c];
#pragma unroll
      for (int j = 0; j < K; ++j) acc[j] += s_A[c * K + j] * t;
    }
  }
}

// Pixel-block Jacobi preconditioner: P = diag_j(tau_j (kappa_j^2 w + L_ii)) + sum_c d_c a_c a_c^T
// (the exact k x k diagonal block of G at the pixel).  It is factored as P = S C C^T S with
// S = diag(P_jj)^{-1/2} (symmetric scaling first, so that badly scaled mixing columns do not
// cost precision) and C lower triangular; pivots are kept positive, so the preconditioner is
// SPD even where rounding makes the scaled block look singular.
template <int K, typename T>
struct BlockChol {
  T s[K];               // scaling
  T l[K * (K + 1) / 2]; // packed lower factor, row-major; diagonal entries stored inverted
};

template <int K, typename T>
__device__ __forceinline__ void block_chol(const OpData& op, const PixelOp<T>& po, const T* s_A,
                                           const T* s_tau, const T* s_tk2, BlockChol<K, T>& f) {
  T P[K * (K + 1) / 2];
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) P[a * (a + 1) / 2 + b] = T(0);
#pragma unroll
  for (int c = 0; c < MMAX; ++c) {
    if (c < op.m) {
      const T d = po.dv[c];
#pragma unroll
      for (int a = 0; a < K; ++a) {
        const T da = d * s_A[c * K + a];
#pragma unroll
        for (int b = 0; b <= a; ++b) P[a * (a + 1) / 2 + b] += da * s_A[c * K + b];
      }
    }
  }
#pragma unroll
  for (int a = 0; a < K; ++a) P[a * (a + 1) / 2 + a] += s_tk2[a] * po.wi + s_tau[a] * po.dg;
#pragma unroll
  for (int a = 0; a < K; ++a) {
    const T pa = P[a * (a + 1) / 2 + a];
    f.s[a] = pa > T(0) ? T(1) / sqrt(pa) : T(1);
  }
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) P[a * (a + 1) / 2 + b] *= f.s[a] * f.s[b];
  const T floor_piv = sizeof(T) == 4 ? T(1e-6) : T(1e-14);
#pragma unroll
  for (int a = 0; a < K; ++a) {
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      T v = P[a * (a + 1) / 2 + b];
#pragma unroll
      for (int c = 0; c < b; ++c) v -= f.l[a * (a + 1) / 2 + c] * f.l[b * (b + 1) / 2 + c];
      if (a == b) {
        v = v > floor_piv ? v : floor_piv;
        f.l[a * (a + 1) / 2 + a] = T(1) / sqrt(v);
      } else {
        f.l[a * (a + 1) / 2 + b] = v * f.l[b * (b + 1) / 2 + b];
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

// Shared per-CTA prologue: system, tile, per-column flags and scalars, mixing in shared memory.
template <int K, typename T>
struct CtaCommon {
  T A[MMAX * K];
  T tau[K];
  T tk2[K];
  T sc[RMAX];       // per-column scalar (beta or alpha)
  int act[RMAX];
  int aux[RMAX];    // per-column flag (first, or phase)
  double red[32 * 4];
  int flag;
};

template <int K, typename T>
__device__ __forceinline__ void load_mixing(const OpData& op, CtaCommon<K, T>& cc) {
  for (int t = threadIdx.x; t < op.m * K; t += blockDim.x) cc.A[t] = OpT<T>::A(op, t);
  if (threadIdx.x < K) {
    cc.tau[threadIdx.x] = OpT<T>::tau(op, threadIdx.x);
    cc.tk2[threadIdx.x] = OpT<T>::tk2(op, threadIdx.x);
  }
}

// ---------------------------------------------------------------------------------------------
// inner_apply: p = z + beta p, q = G z + beta q, partial p . q
// ---------------------------------------------------------------------------------------------
template <int K, typename T>
__global__ void __launch_bounds__(MAX_BLOCK)
k_inner_apply(const SysDesc* __restrict__ descs, const TileRef* __restrict__ tiles, Control* ctl) {
  __shared__ CtaCommon<K, T> cc;
  const TileRef tr = tiles[blockIdx.x];
  const SysDesc& sd = descs[tr.sys];
  const OpData& op = sd.op;
  const int R = sd.R;
  int act = 0;
  if (threadIdx.x < RMAX) {
    const int r = threadIdx.x;
    if (r < R) {
      const ColState& cs = sd.st[r];
      act = cs.phase == PH_INNER;
      cc.sc[r] = T(cs.beta);
      cc.aux[r] = cs.first;
    }
    cc.act[r] = act;
  }
  load_mixing<K, T>(op, cc);
  if (!__syncthreads_or(act)) return;

  const int64_t ld = op.ld;
  const int64_t i = (int64_t)tr.tile * sd.tile_px + threadIdx.x;
  const bool valid = threadIdx.x < sd.tile_px && i < op.n;
  PixelOp<T> po;
  load_pixel_op<T>(op, i, valid, true, po);

  for (int r = 0; r < R; ++r) {
    if (!cc.act[r]) continue;
    const size_t off = (size_t)r * K * ld;
    const T* z = (const T*)sd.vz + off;
    T* p = (T*)sd.vp + off;
    T* q = (T*)sd.vq + off;
    T zi[K], w[K];
#pragma unroll
    for (int j = 0; j < K; ++j) zi[j] = valid ? z[j * ld + i] : T(0);
    apply_pixel<K, T, T>(op, po, cc.A, cc.tau, cc.tk2, z, i, zi, w);
    T pq = T(0);
    if (valid) {
      const T beta = cc.sc[r];
      const bool first = cc.aux[r] != 0;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        T pj = zi[j], qj = w[j];
        if (!first) {
          pj += beta * p[j * ld + i];
          qj += beta * q[j * ld + i];
        }
        p[j * ld + i] = pj;
        q[j * ld + i] = qj;
        pq += pj * qj;
      }
    }
    double v[1] = {double(pq)};
    block_sum<1>(v, cc.red);
    if (threadIdx.x == 0) sd.partial[((size_t)tr.tile * R + r) * NPART + 0] = v[0];
  }
  __syncthreads();
  if (!arrive_last(sd.counter, (unsigned)sd.ntiles, &cc.flag)) return;
  for (int r = 0; r < R; ++r) {
    if (!cc.act[r]) continue;
    const int idx[1] = {0};
    double tot[1];
    reduce_partials<1>(sd, r, idx, tot, cc.red);
    if (threadIdx.x == 0) {
      ColState& cs = sd.st[r];
      const double pq = tot[0];
      if (pq > 0.0 && isfinite(pq)) {
        cs.alpha = cs.gamma / pq;
        cs.first = 0;
      } else if (cs.rr_in == 0.0) {
        cs.phase = PH_INNER_DONE;  // exact solution: nothing left to do
        atomicSub(&ctl->n_active, 1u);
      } else {
        cs.phase = PH_FAILED;
        cs.status = SYLV_E_BREAKDOWN;
        atomicSub(&ctl->n_active, 1u);
        atomicSub(&ctl->n_unfinished, 1u);
      }
    }
  }
  if (threadIdx.x == 0) *sd.counter = 0u;
}

// ---------------------------------------------------------------------------------------------
// inner_update: d += alpha p, r -= alpha q, z = P^{-1} r, partial r . z and r . r
// ---------------------------------------------------------------------------------------------
template <int K, typename T>
__global__ void __launch_bounds__(MAX_BLOCK)
k_inner_update(const SysDesc* __restrict__ descs, const TileRef* __restrict__ tiles,
               Control* ctl) {
  __shared__ CtaCommon<K, T> cc;
  const TileRef tr = tiles[blockIdx.x];
  const SysDesc& sd = descs[tr.sys];
  const OpData& op = sd.op;
  const int R = sd.R;
  int act = 0;
  if (threadIdx.x < RMAX) {
    const int r = threadIdx.x;
    if (r < R) {
      const ColState& cs = sd.st[r];
      act = cs.phase == PH_INNER;
      cc.sc[r] = T(cs.alpha);
    }
    cc.act[r] = act;
  }
  load_mixing<K, T>(op, cc);
  if (!__syncthreads_or(act)) return;

  const int64_t ld = op.ld;
  const int64_t i = (int64_t)tr.tile * sd.tile_px + threadIdx.x;
  const bool valid = threadIdx.x < sd.tile_px && i < op.n;
  const bool prec = ctl->precond == SYLV_PRECOND_BLOCK_JACOBI;
  BlockChol<K, T> f;
  if (prec) {
    PixelOp<T> po;
    load_pixel_op<T>(op, i, valid, false, po);
    block_chol<K, T>(op, po, cc.A, cc.tau, cc.tk2, f);
  }
  for (int r = 0; r < R; ++r) {
    if (!cc.act[r]) continue;
    const size_t off = (size_t)r * K * ld;
    T* d = (T*)sd.vd + off;
    T* rv = (T*)sd.vr + off;
    T* z = (T*)sd.vz + off;
    const T* p = (const T*)sd.vp + off;
    const T* q = (const T*)sd.vq + off;
    const T alpha = cc.sc[r];
    T rz = T(0), rr = T(0);
    if (valid) {
      T ri[K], zi[K];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        d[j * ld + i] += alpha * p[j * ld + i];
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
    double v[2] = {double(rz), double(rr)};
    block_sum<2>(v, cc.red);
    if (threadIdx.x == 0) {
      double* pp = sd.partial + ((size_t)tr.tile * R + r) * NPART;
      pp[0] = v[0];
      pp[1] = v[1];
    }
  }
  __syncthreads();
  if (!arrive_last(sd.counter, (unsigned)sd.ntiles, &cc.flag)) return;
  for (int r = 0; r < R; ++r) {
    if (!cc.act[r]) continue;
    const int idx[2] = {0, 1};
    double tot[2];
    reduce_partials<2>(sd, r, idx, tot, cc.red);
    if (threadIdx.x == 0) {
      ColState& cs = sd.st[r];
      const double rz = tot[0], rr = tot[1];
      cs.it += 1;
      cs.rr_in = rr;
      if (!isfinite(rz) || !isfinite(rr)) {
        cs.phase = PH_FAILED;
        cs.status = SYLV_E_BREAKDOWN;
        atomicSub(&ctl->n_active, 1u);
        atomicSub(&ctl->n_unfinished, 1u);
      } else if (rr <= cs.thr_in || rr == 0.0) {
        cs.phase = PH_INNER_DONE;
        atomicSub(&ctl->n_active, 1u);
      } else if (!(rz > 0.0)) {
        cs.phase = PH_FAILED;
        cs.status = SYLV_E_BREAKDOWN;
        atomicSub(&ctl->n_active, 1u);
        atomicSub(&ctl->n_unfinished, 1u);
      } else if (cs.it >= ctl->maxit) {
        cs.phase = PH_INNER_DONE;
        cs.stop_after = 1;
        atomicSub(&ctl->n_active, 1u);
      } else {
        cs.beta = rz / cs.gamma;
        cs.gamma = rz;
      }
    }
  }
  if (threadIdx.x == 0) *sd.counter = 0u;
}

// ---------------------------------------------------------------------------------------------
// update_x: X += d for columns whose inner solve finished
// ---------------------------------------------------------------------------------------------
template <int K, typename T>
__global__ void __launch_bounds__(MAX_BLOCK)
k_update_x(const SysDesc* __restrict__ descs, const TileRef* __restrict__ tiles) {
  const TileRef tr = tiles[blockIdx.x];
  const SysDesc& sd = descs[tr.sys];
  const int64_t ld = sd.op.ld;
  const int64_t i = (int64_t)tr.tile * sd.tile_px + threadIdx.x;
  if (threadIdx.x >= sd.tile_px || i >= sd.op.n) return;
  for (int r = 0; r < sd.R; ++r) {
    if (sd.st[r].phase != PH_INNER_DONE) continue;
    const size_t off = (size_t)r * K * ld;
    const T* d = (const T*)sd.vd + off;
    double* X = sd.X + off;
#pragma unroll
    for (int j = 0; j < K; ++j) X[j * ld + i] += double(d[j * ld + i]);
  }
}

// ---------------------------------------------------------------------------------------------
// residual: r64 = B - G X (FP64), r_in = r64 rounded, d = 0, z = P^{-1} r_in; decisions
// ---------------------------------------------------------------------------------------------
template <int K, typename T>
__global__ void __launch_bounds__(MAX_BLOCK)
k_residual(const SysDesc* __restrict__ descs, const TileRef* __restrict__ tiles, Control* ctl) {
  __shared__ CtaCommon<K, double> cd;   // FP64 operator
  __shared__ T sA[MMAX * K];            // inner-type preconditioner data
  __shared__ T stau[K], stk2[K];
  const TileRef tr = tiles[blockIdx.x];
  const SysDesc& sd = descs[tr.sys];
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
    cd.act[r] = act;
    cd.aux[r] = ph;
  }
  load_mixing<K, double>(op, cd);
  for (int t = threadIdx.x; t < op.m * K; t += blockDim.x) sA[t] = OpT<T>::A(op, t);
  if (threadIdx.x < K) {
    stau[threadIdx.x] = OpT<T>::tau(op, threadIdx.x);
    stk2[threadIdx.x] = OpT<T>::tk2(op, threadIdx.x);
  }
  if (!__syncthreads_or(act)) return;

  const int64_t ld = op.ld;
  const int64_t i = (int64_t)tr.tile * sd.tile_px + threadIdx.x;
  const bool valid = threadIdx.x < sd.tile_px && i < op.n;
  PixelOp<double> po;
  load_pixel_op<double>(op, i, valid, true, po);
  const bool prec = ctl->precond == SYLV_PRECOND_BLOCK_JACOBI;
  BlockChol<K, T> f;
  if (prec) {
    PixelOp<T> pt;
    load_pixel_op<T>(op, i, valid, false, pt);
    block_chol<K, T>(op, pt, sA, stau, stk2, f);
  }
  for (int r = 0; r < R; ++r) {
    if (!cd.act[r]) continue;
    const size_t off = (size_t)r * K * ld;
    const double* X = sd.X + off;
    const double* B = sd.B + off;
    T* d = (T*)sd.vd + off;
    T* rv = (T*)sd.vr + off;
    T* z = (T*)sd.vz + off;
    double rr64 = 0.0, bb = 0.0, rz = 0.0, rr = 0.0;
    if (valid) {
      double xi[K], gx[K];
#pragma unroll
      for (int j = 0; j < K; ++j) xi[j] = X[j * ld + i];
      apply_pixel<K, double, double>(op, po, cd.A, cd.tau, cd.tk2, X, i, xi, gx);
      T ri[K], zi[K];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const double bj = B[j * ld + i];
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
#pragma unroll
      for (int j = 0; j < K; ++j) {
        z[j * ld + i] = zi[j];
        rz += double(ri[j]) * double(zi[j]);
        rr += double(ri[j]) * double(ri[j]);
      }
    }
    double v[4] = {rr64, bb, rz, rr};
    block_sum<4>(v, cd.red);
    if (threadIdx.x == 0) {
      double* pp = sd.partial + ((size_t)tr.tile * R + r) * NPART;
      pp[0] = v[0];
      pp[1] = v[1];
      pp[2] = v[2];
      pp[3] = v[3];
    }
  }
  __syncthreads();
  if (!arrive_last(sd.counter, (unsigned)sd.ntiles, &cd.flag)) return;
  for (int r = 0; r < R; ++r) {
    if (!cd.act[r]) continue;
    const int idx[4] = {0, 1, 2, 3};
    double tot[4];
    reduce_partials<4>(sd, r, idx, tot, cd.red);
    if (threadIdx.x == 0) {
      ColState& cs = sd.st[r];
      const double rr64 = tot[0], rz = tot[2], rr = tot[3];
      if (cs.phase == PH_START) cs.bnorm2 = tot[1];
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
        // inner target: the reduction still needed (with a safety margin), but no finer
        // than the inner precision can deliver in one refinement step
        const double need = ctl->tol2 * ctl->safety2 * den / rr64;
        const double fac = need > ctl->tol_in2 ? need : ctl->tol_in2;
        cs.phase = PH_INNER;
        cs.first = 1;
        cs.gamma = rz;
        cs.rr_in0 = rr;
        cs.rr_in = rr;
        cs.thr_in = fac * rr;
        cs.outer += 1;
        atomicAdd(&ctl->n_active, 1u);
      }
    }
  }
  if (threadIdx.x == 0) *sd.counter = 0u;
}

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------
#define SYLV_DISPATCH_K(k, CALL) \
  switch (k) {                   \
    case 1: CALL(1); break;      \
    case 2: CALL(2); break;      \
    case 3: CALL(3); break;      \
    case 4: CALL(4); break;      \
    case 5: CALL(5); break;      \
    case 6: CALL(6); break;      \
    case 7: CALL(7); break;      \
    case 8: CALL(8); break;      \
    default: return cudaErrorInvalidValue; \
  }

template <typename T>
cudaError_t launch_inner_apply_impl(int k, int ntiles, int block, const SysDesc* d,
                                    const TileRef* t, Control* c, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
#define CALL(K) k_inner_apply<K, T><<<ntiles, block, 0, s>>>(d, t, c)
  SYLV_DISPATCH_K(k, CALL)
#undef CALL
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_inner_update_impl(int k, int ntiles, int block, const SysDesc* d,
                                     const TileRef* t, Control* c, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
#define CALL(K) k_inner_update<K, T><<<ntiles, block, 0, s>>>(d, t, c)
  SYLV_DISPATCH_K(k, CALL)
#undef CALL
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual_impl(int k, int ntiles, int block, const SysDesc* d,
                                 const TileRef* t, Control* c, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
#define CALL(K) k_residual<K, T><<<ntiles, block, 0, s>>>(d, t, c)
  SYLV_DISPATCH_K(k, CALL)
#undef CALL
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update_x_impl(int k, int ntiles, int block, const SysDesc* d,
                                 const TileRef* t, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
#define CALL(K) k_update_x<K, T><<<ntiles, block, 0, s>>>(d, t)
  SYLV_DISPATCH_K(k, CALL)
#undef CALL
  return cudaGetLastError();
}

}  // namespace sylv
