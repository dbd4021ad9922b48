// Block-Lanczos solver of the Sylvester form of the posterior-mean system (Sec. 3.3,
// Algorithms 4 and 5).
//
// Separable case: noise precision d_ci = t_c nu_i (C = T kron N) and one prior shape
// Q_j = phi_j Q_0 (all kappa_j equal, Q_0 = kappa_0^2 W + L, phi_j = tau_j).  Then
// G vec(M) = vec(B) is eq. Axb-Sylv,
//
//     N^{-1} Q_0 M + M Lhat = Yhat,   Lhat = A^T T A P^{-1},   Yhat = N^{-1} B P^{-1},
//
// and the block Krylov space of the large operator N^{-1} Q_0 (symmetric in (x, y)_N, the
// Lemma of Sec. 3.3) built from Yhat carries the solution of all k shifted systems
// (N^{-1} Q_0 + rho_l) m_l = Yhat u_l at once (Lhat = U diag(rho) U^{-1}).
//
// GPU design (one inner run = Algorithm 5's first pass):
//   * The basis is kept in HBM as raw blocks Vt_s = V_s B_s (B_s upper triangular, the Cholesky
//     factor of the block's N-Gram matrix; the passes form V_s = Vt_s B_s^{-1} per pixel by
//     forward substitution), so a block is written once and read back by the next two passes
//     and by the final assembly M = sum_s V_s G_s (eq. soln-darstellung).  The paper regenerates the blocks in a second
//     Lanczos pass instead; on GB300 the basis fits in memory, and the second pass diverges
//     when B_0 is ill conditioned (as it is for power-law mixing over the Planck channels).
//   * Per Lanczos step two kernels: pass A (W = N^{-1} Q_0 V_s - V_{s-1} B_s^T with the
//     stencil of Algorithm 1 on Vt_s, partial sums of H_s = V_s^T N W), pass B
//     (Vt_{s+1} = W - V_s H_s, partial sums of its N-Gram matrix S).  B_{s+1} = chol(S) is the
//     N-orthonormal QR of Algorithm 4 as a Cholesky QR.  In the plain kernels the last CTA of
//     a pass (atomic counter, fixed-order sums, no waiting) forms the totals, the factor and
//     the records.  The staged kernels elect no last CTA: every CTA of the next pass sums the
//     partials and factors S itself while its producer warp fills the stage ring (pass A of
//     step s + 1 forms B_{s+1}, pass B forms H_s), and a one-CTA kernel closes each chunk.
//   * The residual estimate of Algorithm 5 is evaluated on the host at every poll from the
//     recorded blocks, by one block-LDL^T step per shift and step: the last block z_l of
//     (T_s + rho_l I)^{-1} E_1 B_0 u_l gives gamma = sum_l ||B_{s+1} z_l||^2, the same number
//     as the paper's eigendecomposition formula without a (s k)^3 eigensolve per step.  The
//     run ends at the first step whose gamma meets the target (steps the GPU ran past it
//     between two polls are not used).
//   * The start block is rotated into the eigenbasis of Lhat and its columns scaled to unit
//     N-norm before its Cholesky QR (Yhat U Sigma^{-1}; same span, so the same Krylov space),
//     which keeps the Gram matrix well conditioned when Lhat is.
//   * After the run the host solves the k shifted block-tridiagonal systems for Z (eq.
//     soln-constr, Z = Zhat U^{-1}), and one kernel adds M = sum_s Vt_s (B_s^{-1} G_s) to X.
//   * Mixed precision: the basis, the operator, the partial sums within a CTA and the k x k
//     Cholesky in FP32, the sums across CTAs in two-float arithmetic, the residual estimate,
//     the coefficients and X in FP64; an outer loop forms the true
//     residual B - G X in FP64 (the FP64 pixel-block operator) and restarts the Lanczos run on
//     it until ||B - G X|| / ||B|| <= tol.  In FP64 mode the same loop runs with an FP64 basis.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "pcg_tma.cuh"

namespace sylv {
namespace lz {

constexpr int NT = 256;                        // threads per CTA = pixels per tile
constexpr int NSMAX = KMAX * (KMAX + 1) / 2;   // packed symmetric k x k
constexpr int NVMAX = NSMAX + 2;               // partial sums per CTA (start kernel: + 2)
constexpr int GCHUNK = 32;                     // assembly coefficient blocks staged at a time

enum Done : int { RUNNING = 0, BREAKDOWN = 2, CAPPED = 3 };

struct Ctl {
  int step;           // Lanczos steps completed in the current inner run
  int done;           // Done (the device sets BREAKDOWN and CAPPED, the host stops on gamma)
  int cap;            // steps allowed in this run (basis capacity and iteration budget)
  unsigned counter;   // last-CTA detection, zero between kernels
  unsigned err;       // nonzero: a bounded wait of a staged kernel expired (SYLV_E_TIMEOUT)
  int sa;             // staged passes: the last step whose pass B ran (pass A runs sa + 1)
  int sb;             // staged passes: the step whose pass A ran last (pass B runs it)
  int pad;
};

// Small k x k quantities shared by the passes (row-major, KMAX x KMAX storage).
struct Coef {
  double Rc[KMAX * KMAX];         // B_s, upper triangular: raw block Vt_s = V_s B_s; step s also
                                  // subtracts V_{s-1} B_s^T
  double Rp[KMAX * KMAX];         // B_{s-1}
  double rci[KMAX];               // 1 / diagonal of B_s
  double rpi[KMAX];               // 1 / diagonal of B_{s-1}
  double H[KMAX * KMAX];          // H_s
  double R2[2][KMAX * KMAX];      // staged passes: B_s in slot s & 1 (slot 1 starts as B_1)
  double ri2[2][KMAX];            // and the reciprocals of its diagonal
  double tot[NVMAX];              // start kernel: Gram matrix of the start block, ||r||^2, ||B||^2
};

struct Args {
  OpData op;
  const double* nu64;      // ld: nu_i = d_0i
  const double* nuinv64;
  const float* nu32;
  const float* nuinv32;
  void* basis;             // cap x k x ld raw blocks of the inner type
  int64_t bstride;         // elements per block
  void* wbuf;              // k x ld
  double* partial;         // gridDim.x x NVMAX
  float* partA;            // staged pass A partial sums, value-major, stride gpA
  float* partB;            // staged pass B partial sums, value-major, stride gpB
  int gpA, gpB;            // the producing grid rounded up to 32 (padding stays zero)
  Ctl* ctl;
  Coef* co;
  double* histH;           // cap x k*k: H_s
  double* histB;           // cap x k*k: B_{s+1}
  const double* G;         // nsteps x k*k: assembly coefficients N_s G_s
  const double* B;         // caller right-hand side, k x ldu
  double* X;               // caller solution, k x ldu
  int64_t ldu;
  double kap2;             // kappa_0^2
  double phinv[KMAX];      // 1 / phi_j
  double U[KMAX * KMAX];   // eigenvectors of Lhat (columns), row-major
  int x0_zero;             // start kernel: X = 0, the residual is B
  int nsteps;              // assembly: blocks to add
};

template <typename T> struct NuT;
template <> struct NuT<float> {
  static __device__ __forceinline__ float nu(const Args& a, int64_t i) { return __ldg(a.nu32 + i); }
  static __device__ __forceinline__ float inv(const Args& a, int64_t i) { return __ldg(a.nuinv32 + i); }
};
template <> struct NuT<double> {
  static __device__ __forceinline__ double nu(const Args& a, int64_t i) { return __ldg(a.nu64 + i); }
  static __device__ __forceinline__ double inv(const Args& a, int64_t i) { return __ldg(a.nuinv64 + i); }
};

template <typename T, int NW = NT / 32>
struct Smem {
  T Rc[KMAX][KMAX];   // B_s
  T Rp[KMAX][KMAX];   // B_{s-1}
  T rci[KMAX];
  T rpi[KMAX];
  double red[NW * NVMAX];
  double tot[NVMAX];
  int flag;
};

// v B = x for upper triangular B given with the reciprocals of its diagonal: the basis vector
// of a raw block row, v = x B^{-1}, by forward substitution (no explicit inverse).
template <int K, typename T>
__device__ __forceinline__ void solve_right(const T (&x)[K], const T (&R)[KMAX][KMAX],
                                            const T (&ri)[KMAX], T (&v)[K]) {
#pragma unroll
  for (int l = 0; l < K; ++l) {
    T y = x[l];
#pragma unroll
    for (int p = 0; p < l; ++p) y -= v[p] * R[p][l];
    v[l] = y * ri[l];
  }
}

template <int K, typename T, typename SM>
__device__ __forceinline__ void load_factors(const Coef* co, SM& sh, bool prev) {
  for (int t = threadIdx.x; t < K * K; t += blockDim.x) {
    const int p = t / K, q = t % K;
    sh.Rc[p][q] = T(co->Rc[p * KMAX + q]);
    if (prev) sh.Rp[p][q] = T(co->Rp[p * KMAX + q]);
  }
  if (threadIdx.x < K) {
    sh.rci[threadIdx.x] = T(co->rci[threadIdx.x]);
    if (prev) sh.rpi[threadIdx.x] = T(co->rpi[threadIdx.x]);
  }
}

// ---- reductions -----------------------------------------------------------------------------
// GB300 executes FP64 at 1/64 of the FP32 rate, so a CTA-wide tree of FP64 shuffles at the end
// of every CTA costs more than the CTA's streaming work.  The FP32 passes therefore keep their
// per-thread sums, warp trees and per-CTA sums in FP32, and only the sum over CTAs is carried in
// two-float (hi + lo) arithmetic, by error-free transformations (Knuth's TwoSum), to about
// 2^-48 relative; the FP64 kernels reduce in FP64.  Partial sums are stored value-major,
// partial[t * gridDim.x + blockIdx.x], so that the last CTA to arrive (atomic counter, no
// waiting) reads them with coalesced loads; it forms the totals in a fixed order that depends
// only on the grid size, so they are reproducible.
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

struct FF {   // unevaluated sum hi + lo of two floats
  float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, float b) {
  const float s = a.hi + b;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b - bb);
  return FF{s, a.lo + e};
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  FF r = ff_add(a, b.hi);
  r.lo += b.lo;
  const float s = r.hi + r.lo;   // renormalise
  r.lo = r.lo - (s - r.hi);
  r.hi = s;
  return r;
}

__device__ __forceinline__ FF warp_sum_ff(FF v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    FF o;
    o.hi = __shfl_down_sync(0xffffffffu, v.hi, off);
    o.lo = __shfl_down_sync(0xffffffffu, v.lo, off);
    v = ff_add(v, o);
  }
  return v;
}

// Arrival at the per-grid counter after this CTA's partials are written; true in the last CTA.
template <typename S>
__device__ __forceinline__ bool arrive_last(S& sh, unsigned* counter) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(counter, 1u);
    sh.flag = prev == gridDim.x - 1u ? 1 : 0;
  }
  __syncthreads();
  if (!sh.flag) return false;
  __threadfence();
  return true;
}

// FP32 per-thread values; totals (as double) in sh.tot of the last CTA.
template <int NV, typename S>
__device__ __forceinline__ bool reduce_last(const float (&v)[NV], S& sh, double* partial,
                                            unsigned* counter) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (int)(blockDim.x >> 5);
  float* redf = reinterpret_cast<float*>(sh.red);
  float* pf = reinterpret_cast<float*>(partial);
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    const float s = warp_sum_f(v[t]);
    if (lane == 0) redf[warp * NV + t] = s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    float s = 0.f;
    for (int w = 0; w < nw; ++w) s += redf[w * NV + threadIdx.x];
    pf[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
  if (!arrive_last(sh, counter)) return false;
  // thread x takes the partials of CTAs x, x + blockDim.x, ... (all their loads independent, so
  // they are in flight together), then two-float trees over the warp and over the warps
  FF acc[NV];
#pragma unroll
  for (int t = 0; t < NV; ++t) acc[t] = FF{0.f, 0.f};
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    float x[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) x[t] = __ldcg(pf + (size_t)t * gridDim.x + b);
#pragma unroll
    for (int t = 0; t < NV; ++t) acc[t] = ff_add(acc[t], x[t]);
  }
  __syncthreads();   // redf is reused
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    const FF w = warp_sum_ff(acc[t]);
    if (lane == 0) {
      redf[(warp * NV + t) * 2] = w.hi;
      redf[(warp * NV + t) * 2 + 1] = w.lo;
    }
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    FF tot{0.f, 0.f};
    for (int w = 0; w < nw; ++w)
      tot = ff_add(tot, FF{redf[(w * NV + threadIdx.x) * 2], redf[(w * NV + threadIdx.x) * 2 + 1]});
    sh.tot[threadIdx.x] = double(tot.hi) + double(tot.lo);
  }
  __syncthreads();
  return true;
}

// Staged passes elect no last CTA.  At its end every CTA writes its FP32 partial sums
// (value-major with stride gp, the producing grid rounded up to 32 and zero padded), and every
// CTA of the next pass forms the totals itself at its start while its producer warp is already
// filling the stage ring.  All CTAs add in the same order, so they hold identical totals (and
// identical k x k factors); no CTA of a pass waits for the others at its end.
//
// Per-CTA sums, with the free stage ring as scratch (blockDim.x * NV floats): the per-thread
// values are transposed through shared memory, SEG threads per value add blockDim.x / SEG rows
// each and SEG-lane shuffles finish.
template <int NV>
__device__ __forceinline__ void write_partials_t(const float (&v)[NV], float* pf, int gp,
                                                 float* scratch) {
  constexpr int SEG = 8;
  // blockDim.x is a multiple of SEG and at least SEG * NV
  const int nt = (int)blockDim.x, rows = nt / SEG;
  const int x = threadIdx.x, val = x / SEG, part = x % SEG;
#pragma unroll
  for (int t = 0; t < NV; ++t) scratch[t * nt + x] = v[t];
  __syncthreads();
  if (x < ((SEG * NV + 31) / 32) * 32) {   // whole warps, so the shuffles are full-warp
    float s = 0.f;
    if (val < NV)
      for (int r = part * rows; r < (part + 1) * rows; ++r) s += scratch[val * nt + r];
#pragma unroll
    for (int off = SEG / 2; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off, SEG);
    if (val < NV && part == 0) pf[(size_t)val * gp + blockIdx.x] = s;
  }
}

// Named barrier of the NCS consumer threads (the producer warp is not part of it).
template <int NCS>
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(NCS) : "memory");
}

// Totals of NV values over the partials of one grid (stride gp, a multiple of 32, zero
// padded), as doubles in tot[0 .. NV); run by threads 0 .. NCS - 1, which meet at the named
// barrier afterwards.  SEG lanes per value; lane p adds the 4-vectors p, p + SEG, ... in
// two-float arithmetic (one accumulator per vector component), then SEG-lane shuffles.
template <int NV, int NCS>
__device__ __forceinline__ void sum_partials(const float* pf, int gp, double* tot) {
  constexpr int SEG = 8, NGRP = NCS / SEG, BATCH = 8;
  const int x = threadIdx.x, grp = x / SEG, part = x % SEG;
  const int nq = gp / 4;
#pragma unroll 1
  for (int v0 = 0; v0 < NV; v0 += NGRP) {
    const int v = v0 + grp;
    FF acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (v < NV) {
      const float4* p4 = reinterpret_cast<const float4*>(pf + (size_t)v * gp);
#pragma unroll 1
      for (int q0 = part; q0 < nq; q0 += SEG * BATCH) {
        float4 y[BATCH];
#pragma unroll
        for (int b = 0; b < BATCH; ++b) {   // every load of the batch before any add
          const int q = q0 + b * SEG;
          y[b] = q < nq ? __ldcg(p4 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int b = 0; b < BATCH; ++b) {
          acc[0] = ff_add(acc[0], y[b].x);
          acc[1] = ff_add(acc[1], y[b].y);
          acc[2] = ff_add(acc[2], y[b].z);
          acc[3] = ff_add(acc[3], y[b].w);
        }
      }
    }
    FF t = ff_add(ff_add(acc[0], acc[1]), ff_add(acc[2], acc[3]));
#pragma unroll
    for (int off = SEG / 2; off > 0; off >>= 1) {
      FF o;
      o.hi = __shfl_down_sync(0xffffffffu, t.hi, off, SEG);
      o.lo = __shfl_down_sync(0xffffffffu, t.lo, off, SEG);
      t = ff_add(t, o);
    }
    if (v < NV && part == 0) tot[v] = double(t.hi) + double(t.lo);
  }
  consumers_sync<NCS>();
}

// FP64 per-thread values (FP64 kernels and the start kernel).
template <int NV, typename S>
__device__ __forceinline__ bool reduce_last(const double (&v)[NV], S& sh, double* partial,
                                            unsigned* counter) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (int)(blockDim.x >> 5);
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    const double s = warp_sum(v[t]);
    if (lane == 0) sh.red[warp * NV + t] = s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh.red[w * NV + threadIdx.x];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
  if (!arrive_last(sh, counter)) return false;
  double acc[NV];
#pragma unroll
  for (int t = 0; t < NV; ++t) acc[t] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    double x[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) x[t] = __ldcg(partial + (size_t)t * gridDim.x + b);
#pragma unroll
    for (int t = 0; t < NV; ++t) acc[t] += x[t];
  }
  __syncthreads();   // sh.red is reused
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    const double w = warp_sum(acc[t]);
    if (lane == 0) sh.red[warp * NV + t] = w;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double tot = 0.0;
    for (int w = 0; w < nw; ++w) tot += sh.red[w * NV + threadIdx.x];
    sh.tot[threadIdx.x] = tot;
  }
  __syncthreads();
  return true;
}

// Last CTA of pass B, warp 0: B_{s+1} = chol(S) (S = B^T B, the N-orthonormal QR of the new
// block), the reciprocals of its diagonal, and its history.  Right-looking Cholesky with the
// columns in the lanes' registers: per column one reciprocal square root of the pivot and a
// rank-one update of the trailing block; no explicit inverse (the passes apply B^{-1} by
// forward substitution).  Dependent FP64 operations take 100-200 cycles each on GB300 and S is
// an FP32-accurate sum on the FP32 path, so that path factors in FP32; the FP64 path in FP64.
// False when a pivot falls to the rounding level of the inner type (the block Krylov space is
// numerically exhausted).
template <typename R> struct Arith;
template <> struct Arith<double> {
  using V = double;
  static __device__ __forceinline__ V of(double d) { return d; }
  static __device__ __forceinline__ double dbl(V x) { return x; }
  static __device__ __forceinline__ V add(V a, V b) { return a + b; }
  static __device__ __forceinline__ V mul(V a, V b) { return a * b; }
  static __device__ __forceinline__ V neg(V a) { return -a; }
  static __device__ __forceinline__ V rsq(V a) { return rsqrt(a); }
  static __device__ __forceinline__ float lead(V a) { return float(a); }
};
template <> struct Arith<float> {
  using V = float;
  static __device__ __forceinline__ V of(double d) { return float(d); }
  static __device__ __forceinline__ double dbl(V x) { return double(x); }
  static __device__ __forceinline__ V add(V a, V b) { return a + b; }
  static __device__ __forceinline__ V mul(V a, V b) { return a * b; }
  static __device__ __forceinline__ V neg(V a) { return -a; }
  static __device__ __forceinline__ V rsq(V a) {   // one Newton step on the approximate rsqrt
    const float r = rsqrtf(a);
    return r * (1.5f - 0.5f * a * r * r);
  }
  static __device__ __forceinline__ float lead(V a) { return a; }
};

template <typename V>
__device__ __forceinline__ V shfl_v(V x, int src) { return __shfl_sync(0xffffffffu, x, src); }
template <>
__device__ __forceinline__ FF shfl_v<FF>(FF x, int src) {
  return FF{__shfl_sync(0xffffffffu, x.hi, src), __shfl_sync(0xffffffffu, x.lo, src)};
}

// Lane l of warp 0 holds column l of S, R and R^{-1} in registers; rows move between lanes by
// shuffles.  Called by all 32 lanes of warp 0 (lanes >= K carry zero columns).
template <int K, typename T>
__device__ __forceinline__ bool chol_lanes(const double* tot, typename Arith<T>::V (&Rc)[K],
                                           typename Arith<T>::V (&rinv)[K]) {
  using AR = Arith<T>;
  using V = typename AR::V;
  const int lane = threadIdx.x & 31;
  float tr = 0.f;
#pragma unroll
  for (int p = 0; p < K; ++p) tr += float(tot[p * K - p * (p - 1) / 2]);
  V col[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    // packed upper triangle, row by row: entry (p, q), q >= p, at p K - p (p - 1) / 2 + q - p
    const int p0 = i < lane ? i : lane, q0 = i < lane ? lane : i;
    col[i] = lane < K ? AR::of(tot[p0 * K - p0 * (p0 - 1) / 2 + (q0 - p0)]) : AR::of(0.0);
    Rc[i] = AR::of(0.0);
  }
  const float thr = (sizeof(T) == 4 ? 1e-12f : 1e-26f) * tr;
  bool bad = false;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    V d = shfl_v(col[j], j);                       // trailing pivot, held by lane j
    if (!(AR::lead(d) > thr) || !isfinite(AR::lead(d))) {
      bad = true;
      d = AR::of(1.0);
    }
    const V r = AR::rsq(d);
    rinv[j] = r;
    Rc[j] = lane > j ? AR::mul(col[j], r) : (lane == j ? AR::mul(d, r) : AR::of(0.0));
#pragma unroll
    for (int i = j + 1; i < K; ++i) {              // col[i] -= R[j][i] R[j][lane]
      const V rji = shfl_v(Rc[j], i);
      col[i] = AR::add(col[i], AR::neg(AR::mul(rji, Rc[j])));
    }
  }
  return !bad;
}

template <int K, typename T, typename SM>
__device__ __noinline__ bool qr_coefficients(const Args& a, int s, SM& sh) {
  using AR = Arith<T>;
  using V = typename AR::V;
  const int lane = threadIdx.x & 31;
  V Rc[K], rinv[K];
  if (!chol_lanes<K, T>(sh.tot, Rc, rinv)) return false;
  if (lane < K) {
    double* hb = a.histB + (size_t)(s - 1) * K * K;
    Coef* co = a.co;
    // the factor this kernel used (staged in shared memory at its start) becomes the previous
    double prev[K];
#pragma unroll
    for (int i = 0; i < K; ++i) prev[i] = double(sh.Rc[i][lane]);
    const double prevri = double(sh.rci[lane]);
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const double rb = AR::dbl(Rc[i]);
      hb[i * K + lane] = rb;
      co->Rp[i * KMAX + lane] = prev[i];
      co->Rc[i * KMAX + lane] = rb;
    }
    co->rpi[lane] = prevri;
    // rinv[j] is uniform over the lanes: lane j publishes its own
    double own = 0.0;
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j == lane) own = AR::dbl(rinv[j]);
    co->rci[lane] = own;
  }
  return true;
}

// Staged passes, warp 0: B = chol(S) of this CTA's totals into shared memory (FP32 Rc, rci).
// With `rec` (one CTA) also its record: histB row `hrow` and, for slot >= 0, coefficient slot
// `slot` for the passes that follow.
template <int K, typename SM>
__device__ __noinline__ bool factor_staged(const Args& a, SM& sh, bool rec, int hrow, int slot) {
  const int lane = threadIdx.x & 31;
  float Rc[K], rinv[K];
  const bool ok = chol_lanes<K, float>(sh.tot, Rc, rinv);
  if (ok && lane < K) {
    float own = 0.f;   // rinv[j] is uniform over the lanes: lane j keeps its own
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j == lane) own = rinv[j];
#pragma unroll
    for (int i = 0; i < K; ++i) sh.Rc[i][lane] = Rc[i];
    sh.rci[lane] = own;
    if (rec) {
      double* hb = a.histB + (size_t)hrow * K * K;
#pragma unroll
      for (int i = 0; i < K; ++i) {
        hb[i * K + lane] = double(Rc[i]);
        if (slot >= 0) a.co->R2[slot][i * KMAX + lane] = double(Rc[i]);
      }
      if (slot >= 0) a.co->ri2[slot][lane] = double(own);
    }
  }
  return ok;
}

template <int K>
__device__ __forceinline__ void load_slot(const Coef* co, int slot, float (&R)[KMAX][KMAX],
                                          float (&ri)[KMAX]) {
  for (int t = threadIdx.x; t < K * K; t += blockDim.x)
    R[t / K][t % K] = float(co->R2[slot][(t / K) * KMAX + t % K]);
  if (threadIdx.x < K) ri[threadIdx.x] = float(co->ri2[slot][threadIdx.x]);
}

// ---- start: r = B - G X (FP64), rotated and weighted start block, its N-Gram matrix ----------
template <int K, int E, typename T>
__global__ void __launch_bounds__(NT, 2) k_lz_start(const Args a) {
  __shared__ CtaShared<double, 1> op_sh;
  __shared__ Smem<T> sh;
  constexpr int NS = K * (K + 1) / 2;
  const OpData& op = a.op;
  stage_operator<double, 1>(op, K, op_sh);
  __syncthreads();
  const int64_t ld = op.ld, n = op.n, ldu = a.ldu;
  T* raw = (T*)a.basis;
  double acc[NS + 2];
#pragma unroll
  for (int t = 0; t < NS + 2; ++t) acc[t] = 0.0;
  const int64_t ntiles = (n + NT - 1) / NT;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i = tile * NT + threadIdx.x;
    if (i >= n) continue;
    double r[K];
    if (a.x0_zero) {
#pragma unroll
      for (int j = 0; j < K; ++j) r[j] = a.B[j * ldu + i];
    } else {
      double xi[K], gx[K];
#pragma unroll
      for (int j = 0; j < K; ++j) xi[j] = a.X[j * ldu + i];
      apply_pixel_blk64<K, E, double, 1>(op, op_sh, a.X, ldu, i, xi, gx);
#pragma unroll
      for (int j = 0; j < K; ++j) r[j] = a.B[j * ldu + i] - gx[j];
    }
    const double ninv = __ldg(a.nuinv64 + i), nu = __ldg(a.nu64 + i);
    double yh[K], C[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const double bj = a.B[j * ldu + i];
      acc[NS] += r[j] * r[j];
      acc[NS + 1] += bj * bj;
      yh[j] = r[j] * ninv * a.phinv[j];
    }
#pragma unroll
    for (int l = 0; l < K; ++l) {
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < K; ++j) v += yh[j] * a.U[j * KMAX + l];
      C[l] = v;
      raw[l * ld + i] = T(v);
    }
    int t = 0;
#pragma unroll
    for (int p = 0; p < K; ++p)
#pragma unroll
      for (int q = p; q < K; ++q) acc[t++] += nu * C[p] * C[q];
  }
  if (!reduce_last<NS + 2>(acc, sh, a.partial, &a.ctl->counter)) return;
  if (threadIdx.x < NS + 2) a.co->tot[threadIdx.x] = sh.tot[threadIdx.x];
  if (threadIdx.x == 0) a.ctl->counter = 0u;
}

// ---- pass A: W = N^{-1} Q_0 V_s - V_{s-1} B_s^T, partial sums of H_s = V_s^T N W -------------
template <int K, int E, typename T>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 3 : 2) k_lz_a(const Args a) {
  __shared__ Smem<T> sh;
  constexpr int NS = K * (K + 1) / 2;
  if (a.ctl->done != RUNNING) return;
  const int s = a.ctl->step + 1;
  load_factors<K, T>(a.co, sh, s > 1);
  __syncthreads();
  const OpData& op = a.op;
  const int64_t ld = op.ld, n = op.n;
  const T* cur = (const T*)a.basis + (size_t)(s - 1) * a.bstride;
  const T* prev = s > 1 ? (const T*)a.basis + (size_t)(s - 2) * a.bstride : cur;
  T* W = (T*)a.wbuf;
  const T* val = OpT<T>::val(op);
  const T* dgp = OpT<T>::diag(op);
  const T* wp = OpT<T>::w(op);
  const T kap2 = T(a.kap2);
  const int Er = E > 0 ? E : op.E;
  T acc[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) acc[t] = T(0);
  const int64_t ntiles = (n + NT - 1) / NT;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i = tile * NT + threadIdx.x;
    if (i >= n) continue;
    T u[K], lap[K];
    const T dg = __ldg(dgp + i) + kap2 * (op.has_w ? __ldg(wp + i) : T(1));
#pragma unroll
    for (int j = 0; j < K; ++j) {
      u[j] = __ldg(cur + j * ld + i);
      lap[j] = dg * u[j];
    }
    constexpr int EC = E > 0 ? E : 4;
    for (int e0 = 0; e0 < Er; e0 += EC) {
      int64_t col[EC];
      T v[EC];
#pragma unroll
      for (int t = 0; t < EC; ++t) {
        const int e = E > 0 ? t : min(e0 + t, Er - 1);
        col[t] = __ldg(op.ell_col + e * ld + i);
        v[t] = __ldg(val + e * ld + i);
        if (E == 0 && e0 + t >= Er) v[t] = T(0);
      }
#pragma unroll
      for (int t = 0; t < EC; ++t)
#pragma unroll
        for (int j = 0; j < K; ++j) lap[j] += v[t] * __ldg(cur + j * ld + col[t]);
    }
    T vv[K], qv[K], w[K];
    const T ninv = NuT<T>::inv(a, i), nu = NuT<T>::nu(a, i);
    solve_right<K, T>(u, sh.Rc, sh.rci, vv);
    solve_right<K, T>(lap, sh.Rc, sh.rci, qv);
#pragma unroll
    for (int l = 0; l < K; ++l) w[l] = qv[l] * ninv;
    if (s > 1) {
      T uo[K], vo[K];
#pragma unroll
      for (int j = 0; j < K; ++j) uo[j] = __ldg(prev + j * ld + i);
      solve_right<K, T>(uo, sh.Rp, sh.rpi, vo);
#pragma unroll
      for (int l = 0; l < K; ++l) {
        T x = T(0);
#pragma unroll
        for (int p = l; p < K; ++p) x += vo[p] * sh.Rc[l][p];
        w[l] -= x;
      }
    }
    T nw[K];
#pragma unroll
    for (int l = 0; l < K; ++l) {
      W[l * ld + i] = w[l];
      nw[l] = nu * w[l];
    }
    int t = 0;
#pragma unroll
    for (int p = 0; p < K; ++p)
#pragma unroll
      for (int q = p; q < K; ++q) acc[t++] += vv[p] * nw[q] + vv[q] * nw[p];
  }
  if (!reduce_last<NS>(acc, sh, a.partial, &a.ctl->counter)) return;
  if (threadIdx.x == 0) {
    int t = 0;
    double* hh = a.histH + (size_t)(s - 1) * K * K;
    for (int p = 0; p < K; ++p)
      for (int q = p; q < K; ++q, ++t) {
        const double h = 0.5 * sh.tot[t];
        a.co->H[p * KMAX + q] = h;
        a.co->H[q * KMAX + p] = h;
        hh[p * K + q] = h;
        hh[q * K + p] = h;
      }
    a.ctl->counter = 0u;
  }
}

// ---- pass B: Vt_{s+1} = W - V_s H_s, partial sums of S = Vt_{s+1}^T N Vt_{s+1}; last CTA: QR
// coefficient B_{s+1} = chol(S), normalizer, residual estimate, stopping -------------------------
template <int K, typename T>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 3 : 2) k_lz_b(const Args a) {
  __shared__ Smem<T> sh;
  __shared__ T Hs[KMAX][KMAX];
  constexpr int NS = K * (K + 1) / 2;
  if (a.ctl->done != RUNNING) return;
  const int s = a.ctl->step + 1;
  load_factors<K, T>(a.co, sh, false);
  for (int t = threadIdx.x; t < K * K; t += NT) Hs[t / K][t % K] = T(a.co->H[(t / K) * KMAX + t % K]);
  __syncthreads();
  const int64_t ld = a.op.ld, n = a.op.n;
  const T* cur = (const T*)a.basis + (size_t)(s - 1) * a.bstride;
  T* next = (T*)a.basis + (size_t)s * a.bstride;
  const T* W = (const T*)a.wbuf;
  T acc[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) acc[t] = T(0);
  const int64_t ntiles = (n + NT - 1) / NT;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i = tile * NT + threadIdx.x;
    if (i >= n) continue;
    T u[K], ww[K], vv[K], un[K];
    // every load of the pixel before any store (W and the next block are distinct buffers,
    // which the compiler cannot know)
#pragma unroll
    for (int j = 0; j < K; ++j) {
      u[j] = __ldg(cur + j * ld + i);
      ww[j] = __ldg(W + j * ld + i);
    }
    solve_right<K, T>(u, sh.Rc, sh.rci, vv);
#pragma unroll
    for (int l = 0; l < K; ++l) {
      T x = ww[l];
#pragma unroll
      for (int p = 0; p < K; ++p) x -= vv[p] * Hs[p][l];
      un[l] = x;
    }
#pragma unroll
    for (int l = 0; l < K; ++l) next[l * ld + i] = un[l];
    const T nu = NuT<T>::nu(a, i);
    int t = 0;
#pragma unroll
    for (int p = 0; p < K; ++p) {
      const T np = nu * un[p];
#pragma unroll
      for (int q = p; q < K; ++q) acc[t++] += np * un[q];
    }
  }
  if (!reduce_last<NS>(acc, sh, a.partial, &a.ctl->counter)) return;
  // ---- last CTA: QR coefficients and the stopping state ------------------------------------
  if (threadIdx.x < 32) {
    const bool ok = qr_coefficients<K, T>(a, s, sh);
    if (threadIdx.x == 0) {
      Ctl* ctl = a.ctl;
      ctl->step = s;
      if (!ok) ctl->done = BREAKDOWN;
      else if (s >= ctl->cap) ctl->done = CAPPED;
      ctl->counter = 0u;
    }
  }
}

// ---- staged FP32 passes ----------------------------------------------------------------------
// The same two passes with every contiguous row a tile needs (the raw blocks, W, the ELL rows,
// the Laplacian diagonal, nu and 1/nu; TILE_PX values each) brought into shared memory by
// cp.async.bulk copies: one producer warp fills a ring of stages on "full" mbarriers, eight
// consumer warps (one pixel per thread) compute from it and release each stage on an "empty"
// mbarrier.  Stencil neighbours inside the tile are read from the staged block, the others
// (one image row away) from global memory.  Every wait is bounded; on expiry the CTA sets
// Ctl::err, waits (bounded) for its copies in flight and leaves without its partial sums.
using tma::NCONS;
using tma::WS_THREADS;
constexpr int NST_A = 3;   // stages of the pass-A ring (3 x 23 KB for k = 6, E = 4)
constexpr int NST_B = 4;   // stages of the pass-B ring (4 x 13 KB for k = 6)

template <int NST>
struct Pipe {
  uint64_t full[NST];
  uint64_t empty[NST];
  int bad;
  int issued;
};

template <int NST>
__device__ __forceinline__ void pipe_init(Pipe<NST>& ps) {
  for (int q = 0; q < NST; ++q) {
    tma::mbar_init(&ps.full[q], 1);
    tma::mbar_init(&ps.empty[q], NCONS);
  }
  ps.bad = 0;
  ps.issued = 0;
  tma::fence_mbar_init();
}

// Producer warp, units u0 .. u1 - 1: waits until the consumers released stage u % NST (from
// the second round of the ring on), then issues unit u.
template <int NST, typename Issue>
__device__ __forceinline__ void producer_range(Pipe<NST>& ps, int u0, int u1, Issue&& issue) {
  const int lane = threadIdx.x & 31;
  for (int u = u0; u < u1; ++u) {
    const int st = u % NST;
    if (u >= NST) {
      bool ok = true;
      if (lane == 0) ok = tma::mbar_wait_bounded(&ps.empty[st], ((u / NST) - 1) & 1);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok || ps.bad) {
        if (lane == 0) ps.bad = 1;
        break;
      }
    }
    issue(u, st);
    if (lane == 0) ps.issued = u + 1;
  }
}

template <int K, int E>
struct LayoutA {
  static constexpr int NST = E > 8 ? 2 : NST_A;   // wide stencils: two stages of ~35 KB
  static constexpr int CUR = 0, PREV = K, VAL = 2 * K, COL = 2 * K + E, DIAG = 2 * K + 2 * E,
                       NU = DIAG + 1, NUINV = DIAG + 2;
  static constexpr int ROWS = 2 * K + 2 * E + 3;
  static constexpr int STAGE_BYTES = ROWS * TILE_PX * 4;
};

template <int K>
struct LayoutB {
  static constexpr int W = 0, CUR = K, NU = 2 * K;
  static constexpr int ROWS = 2 * K + 1;
  static constexpr int STAGE_BYTES = ROWS * TILE_PX * 4;
};

template <int NST>
__device__ __forceinline__ bool staged_failed(Pipe<NST>& ps, int consumed, Ctl* ctl) {
  __syncthreads();
  if (!ps.bad) return false;
  if (threadIdx.x == 0) {
    atomicOr(&ctl->err, 1u);
    for (int u = consumed; u < ps.issued; ++u)
      tma::mbar_wait_bounded(&ps.full[u % NST], (u / NST) & 1);
  }
  __syncthreads();
  return true;
}

// Copies issued before a run ends at the start of a pass: wait (bounded) until they landed.
template <int NST>
__device__ __forceinline__ void drain_issued(Pipe<NST>& ps) {
  for (int u = 0; u < ps.issued; ++u) tma::mbar_wait_bounded(&ps.full[u % NST], (u / NST) & 1);
}

// Pass A, step s = Ctl::sa + 1.  The producer warp issues the first ring of stages at once;
// meanwhile the consumers sum pass B's partials (the N-Gram matrix of Vt_s) and warp 0 factors
// it, B_s = chol(S) (CTA 0 records it).  A breakdown, or a run that reached its cap, ends here.
template <int K, int E>
__global__ void __launch_bounds__(WS_THREADS, 3) k_lz_a_tma(const Args a) {
  using L = LayoutA<K, E>;
  constexpr int NS = K * (K + 1) / 2;
  static_assert(8 * NS <= WS_THREADS && (size_t)WS_THREADS * NS * 4 <= (size_t)L::NST * L::STAGE_BYTES,
                "per-CTA sums need 8 threads per value and the stage ring as scratch");
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ Smem<float, WS_THREADS / 32> sh;
  __shared__ __align__(8) Pipe<L::NST> ps;
  if (a.ctl->done != RUNNING) return;
  const int s = a.ctl->sa + 1;
  // B_{s-1} from its slot (s = 1: B_1 from the host, into the current factor)
  if (s > 1) load_slot<K>(a.co, (s - 1) & 1, sh.Rp, sh.rpi);
  else load_slot<K>(a.co, 1, sh.Rc, sh.rci);
  if (threadIdx.x == 0) pipe_init(ps);
  __syncthreads();
  const OpData& op = a.op;
  const int64_t ld = op.ld, n = op.n;
  const float* cur = (const float*)a.basis + (size_t)(s - 1) * a.bstride;
  const float* prev = s > 1 ? (const float*)a.basis + (size_t)(s - 2) * a.bstride : cur;
  float* W = (float*)a.wbuf;
  const float kap2 = float(a.kap2);
  const int ntiles = (int)((n + TILE_PX - 1) / TILE_PX);
  const int nunits = (int)blockIdx.x < ntiles ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  const int head = nunits < L::NST ? nunits : L::NST;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto issue = [&](int u, int st) {
    const int64_t base = ((int64_t)blockIdx.x + (int64_t)u * gridDim.x) * TILE_PX;
    float* stage = reinterpret_cast<float*>(dsm + (size_t)st * L::STAGE_BYTES);
    const uint32_t rowb = TILE_PX * 4;
    const int nrows = s > 1 ? L::ROWS : L::ROWS - K;
    if (lane == 0) {
      tma::fence_proxy_async();
      tma::mbar_expect_tx(&ps.full[st], (uint32_t)nrows * rowb);
    }
    __syncwarp();
    for (int q = lane; q < L::ROWS; q += 32) {
      const void* src = nullptr;
      if (q < K) src = cur + (size_t)q * ld + base;
      else if (q < 2 * K) src = s > 1 ? prev + (size_t)(q - K) * ld + base : nullptr;
      else if (q < L::COL) src = op.ell_val32 + (size_t)(q - L::VAL) * ld + base;
      else if (q < L::DIAG) src = op.ell_col + (size_t)(q - L::COL) * ld + base;
      else if (q == L::DIAG) src = op.diag32 + base;
      else if (q == L::NU) src = a.nu32 + base;
      else src = a.nuinv32 + base;
      if (src) tma::bulk_load(stage + (size_t)q * TILE_PX, src, rowb, &ps.full[st]);
    }
  };
  if (warp == NCONS) {
    producer_range(ps, 0, head, issue);
  } else if (s > 1) {
    sum_partials<NS, TILE_PX>(a.partB, a.gpB, sh.tot);
    if (warp == 0) {
      const bool rec = blockIdx.x == 0;
      const bool ok = factor_staged<K>(a, sh, rec, s - 2, s & 1);
      if (lane == 0) {
        const int stop = !ok ? BREAKDOWN : (s - 1 >= a.ctl->cap ? CAPPED : RUNNING);
        sh.flag = stop;
        if (rec) {
          a.ctl->step = s - 1;
          if (stop != RUNNING) a.ctl->done = stop;
          else a.ctl->sb = s;
        }
      }
    }
  } else if (threadIdx.x == 0) {
    sh.flag = RUNNING;
    if (blockIdx.x == 0) a.ctl->sb = 1;
  }
  __syncthreads();
  if (sh.flag != RUNNING) {
    if (threadIdx.x == 0) drain_issued(ps);
    return;
  }
  int consumed = 0;
  float acc[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) acc[t] = 0.f;
  if (warp == NCONS) {
    producer_range(ps, head, nunits, issue);
  } else {
    const int t = threadIdx.x;
    for (int u = 0; u < nunits; ++u) {
      const int st = u % L::NST;
      if (!tma::mbar_wait_bounded(&ps.full[st], (u / L::NST) & 1) || ps.bad) {
        ps.bad = 1;
        break;
      }
      const int64_t base = ((int64_t)blockIdx.x + (int64_t)u * gridDim.x) * TILE_PX;
      const int64_t i = base + t;
      const float* stage = reinterpret_cast<const float*>(dsm + (size_t)st * L::STAGE_BYTES);
      const int32_t* scol = reinterpret_cast<const int32_t*>(stage + (size_t)L::COL * TILE_PX);
      float uu[K], lap[K];
      const float dg = stage[L::DIAG * TILE_PX + t] + kap2;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        uu[j] = stage[(L::CUR + j) * TILE_PX + t];
        lap[j] = dg * uu[j];
      }
      const float* src[E];
      int64_t stride[E];
      float v[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int64_t c = scol[e * TILE_PX + t];
        v[e] = stage[(L::VAL + e) * TILE_PX + t];
        const uint32_t loc = (uint32_t)(c - base);
        const bool in_tile = loc < (uint32_t)TILE_PX;
        src[e] = in_tile ? stage + (size_t)L::CUR * TILE_PX + loc : cur + c;
        stride[e] = in_tile ? (int64_t)TILE_PX : ld;
      }
      float nb[E][K];
#pragma unroll
      for (int e = 0; e < E; ++e)
#pragma unroll
        for (int j = 0; j < K; ++j) nb[e][j] = src[e][j * stride[e]];
      if constexpr (K % 2 == 0) {   // pairs of columns with the packed FP32 FMA (fma.rn.f32x2)
        float2 l2[K / 2];
#pragma unroll
        for (int q = 0; q < K / 2; ++q) l2[q] = make_float2(lap[2 * q], lap[2 * q + 1]);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const float2 ve = make_float2(v[e], v[e]);
#pragma unroll
          for (int q = 0; q < K / 2; ++q)
            l2[q] = __ffma2_rn(ve, make_float2(nb[e][2 * q], nb[e][2 * q + 1]), l2[q]);
        }
#pragma unroll
        for (int q = 0; q < K / 2; ++q) {
          lap[2 * q] = l2[q].x;
          lap[2 * q + 1] = l2[q].y;
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e)
#pragma unroll
          for (int j = 0; j < K; ++j) lap[j] += v[e] * nb[e][j];
      }
      const float ninv = stage[L::NUINV * TILE_PX + t], nu = stage[L::NU * TILE_PX + t];
      float vv[K], qv[K], w[K];
      solve_right<K, float>(uu, sh.Rc, sh.rci, vv);
      solve_right<K, float>(lap, sh.Rc, sh.rci, qv);
#pragma unroll
      for (int l = 0; l < K; ++l) w[l] = qv[l] * ninv;
      if (s > 1) {
        float uo[K], vo[K];
#pragma unroll
        for (int p = 0; p < K; ++p) uo[p] = stage[(L::PREV + p) * TILE_PX + t];
        solve_right<K, float>(uo, sh.Rp, sh.rpi, vo);
#pragma unroll
        for (int l = 0; l < K; ++l) {
          float x = 0.f;
#pragma unroll
          for (int p = l; p < K; ++p) x += vo[p] * sh.Rc[l][p];
          w[l] -= x;
        }
      }
      __syncwarp();
      if (lane == 0) tma::mbar_arrive(&ps.empty[st]);
      consumed = u + 1;
      if (i < n) {
        float nw[K];
#pragma unroll
        for (int l = 0; l < K; ++l) {
          W[l * ld + i] = w[l];
          nw[l] = nu * w[l];
        }
        int x = 0;
#pragma unroll
        for (int p = 0; p < K; ++p)
#pragma unroll
          for (int q = p; q < K; ++q) acc[x++] += vv[p] * nw[q] + vv[q] * nw[p];
      }
    }
  }
  if (staged_failed(ps, consumed, a.ctl)) return;
  write_partials_t<NS>(acc, a.partA, a.gpA, reinterpret_cast<float*>(dsm));
}

// Pass B, step s = Ctl::sb: the consumers first sum pass A's partials into H_s (CTA 0 records
// it) while the producer fills the ring.
template <int K>
__global__ void __launch_bounds__(WS_THREADS, 3) k_lz_b_tma(const Args a) {
  using L = LayoutB<K>;
  constexpr int NS = K * (K + 1) / 2;
  static_assert(8 * NS <= WS_THREADS && (size_t)WS_THREADS * NS * 4 <= (size_t)NST_B * L::STAGE_BYTES,
                "per-CTA sums need 8 threads per value and the stage ring as scratch");
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ Smem<float, WS_THREADS / 32> sh;
  __shared__ float Hs[KMAX][KMAX];
  __shared__ __align__(8) Pipe<NST_B> ps;
  if (a.ctl->done != RUNNING) return;
  const int s = a.ctl->sb;
  load_slot<K>(a.co, s & 1, sh.Rc, sh.rci);
  if (threadIdx.x == 0) pipe_init(ps);
  __syncthreads();
  const int64_t ld = a.op.ld, n = a.op.n;
  const float* cur = (const float*)a.basis + (size_t)(s - 1) * a.bstride;
  float* next = (float*)a.basis + (size_t)s * a.bstride;
  const float* W = (const float*)a.wbuf;
  const int ntiles = (int)((n + TILE_PX - 1) / TILE_PX);
  const int nunits = (int)blockIdx.x < ntiles ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  const int head = nunits < NST_B ? nunits : NST_B;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto issue = [&](int u, int st) {
    const int64_t base = ((int64_t)blockIdx.x + (int64_t)u * gridDim.x) * TILE_PX;
    float* stage = reinterpret_cast<float*>(dsm + (size_t)st * L::STAGE_BYTES);
    const uint32_t rowb = TILE_PX * 4;
    if (lane == 0) {
      tma::fence_proxy_async();
      tma::mbar_expect_tx(&ps.full[st], (uint32_t)L::ROWS * rowb);
    }
    __syncwarp();
    for (int q = lane; q < L::ROWS; q += 32) {
      const void* src;
      if (q < K) src = W + (size_t)q * ld + base;
      else if (q < 2 * K) src = cur + (size_t)(q - K) * ld + base;
      else src = a.nu32 + base;
      tma::bulk_load(stage + (size_t)q * TILE_PX, src, rowb, &ps.full[st]);
    }
  };
  if (warp == NCONS) {
    producer_range(ps, 0, head, issue);
  } else {
    sum_partials<NS, TILE_PX>(a.partA, a.gpA, sh.tot);
    for (int t = threadIdx.x; t < K * K; t += TILE_PX) {
      const int p = t / K, q = t % K, lo = p < q ? p : q, hi = p < q ? q : p;
      const double h = 0.5 * sh.tot[lo * K - lo * (lo - 1) / 2 + (hi - lo)];
      Hs[p][q] = float(h);
      if (blockIdx.x == 0) a.histH[(size_t)(s - 1) * K * K + t] = h;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->sa = s;
  }
  __syncthreads();
  int consumed = 0;
  float acc[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) acc[t] = 0.f;
  if (warp == NCONS) {
    producer_range(ps, head, nunits, issue);
  } else {
    const int t = threadIdx.x;
    for (int u = 0; u < nunits; ++u) {
      const int st = u % NST_B;
      if (!tma::mbar_wait_bounded(&ps.full[st], (u / NST_B) & 1) || ps.bad) {
        ps.bad = 1;
        break;
      }
      const int64_t i = ((int64_t)blockIdx.x + (int64_t)u * gridDim.x) * TILE_PX + t;
      const float* stage = reinterpret_cast<const float*>(dsm + (size_t)st * L::STAGE_BYTES);
      float uu[K], ww[K], vv[K], un[K];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        uu[j] = stage[(L::CUR + j) * TILE_PX + t];
        ww[j] = stage[(L::W + j) * TILE_PX + t];
      }
      const float nu = stage[L::NU * TILE_PX + t];
      __syncwarp();
      if (lane == 0) tma::mbar_arrive(&ps.empty[st]);
      consumed = u + 1;
      solve_right<K, float>(uu, sh.Rc, sh.rci, vv);
#pragma unroll
      for (int l = 0; l < K; ++l) {
        float x = ww[l];
#pragma unroll
        for (int p = 0; p < K; ++p) x -= vv[p] * Hs[p][l];
        un[l] = x;
      }
      if (i < n) {
#pragma unroll
        for (int l = 0; l < K; ++l) next[l * ld + i] = un[l];
        int x = 0;
#pragma unroll
        for (int p = 0; p < K; ++p) {
          const float np = nu * un[p];
#pragma unroll
          for (int q = p; q < K; ++q) acc[x++] += np * un[q];
        }
      }
    }
  }
  if (staged_failed(ps, consumed, a.ctl)) return;
  write_partials_t<NS>(acc, a.partB, a.gpB, reinterpret_cast<float*>(dsm));
}

// End of a chunk of staged steps (one CTA of TILE_PX threads): B_{s+1} of the last step s from
// pass B's sums, recorded so that the host sees it at the poll, and the stopping state; the next
// pass A forms the same factor again.
template <int K>
__global__ void __launch_bounds__(TILE_PX, 1) k_lz_fin(const Args a) {
  constexpr int NS = K * (K + 1) / 2;
  __shared__ Smem<float, TILE_PX / 32> sh;
  if (a.ctl->done != RUNNING) return;
  const int s = a.ctl->sa;
  if (s < 1) return;
  sum_partials<NS, TILE_PX>(a.partB, a.gpB, sh.tot);
  if (threadIdx.x < 32) {
    const bool ok = factor_staged<K>(a, sh, true, s - 1, -1);
    if (threadIdx.x == 0) {
      a.ctl->step = s;
      if (!ok) a.ctl->done = BREAKDOWN;
      else if (s >= a.ctl->cap) a.ctl->done = CAPPED;
    }
  }
}

// ---- assembly: X += sum_s Vt_s G'_s with G'_s = N_s G_s --------------------------------------
template <int K, typename T>
__global__ void __launch_bounds__(NT, 2) k_lz_assemble(const Args a) {
  __shared__ T g[GCHUNK][K * K];
  const int64_t ld = a.op.ld, n = a.op.n, ldu = a.ldu;
  const int64_t ntiles = (n + NT - 1) / NT;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i = tile * NT + threadIdx.x;
    const bool valid = i < n;
    T acc[K];
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] = T(0);
    for (int s0 = 0; s0 < a.nsteps; s0 += GCHUNK) {
      const int ns = min(GCHUNK, a.nsteps - s0);
      __syncthreads();
      for (int t = threadIdx.x; t < ns * K * K; t += NT)
        g[t / (K * K)][t % (K * K)] = T(a.G[(size_t)s0 * K * K + t]);
      __syncthreads();
      if (!valid) continue;
      // AB blocks at a time: every load of the batch is issued before its products, so that
      // AB K loads per thread are in flight (the sums keep the step order)
      constexpr int AB = 4;
      int q = 0;
      for (; q + AB <= ns; q += AB) {
        T u[AB][K];
#pragma unroll
        for (int b = 0; b < AB; ++b) {
          const T* blk = (const T*)a.basis + (size_t)(s0 + q + b) * a.bstride;
#pragma unroll
          for (int p = 0; p < K; ++p) u[b][p] = __ldg(blk + p * ld + i);
        }
#pragma unroll
        for (int b = 0; b < AB; ++b)
#pragma unroll
          for (int j = 0; j < K; ++j) {
            T x = acc[j];
#pragma unroll
            for (int p = 0; p < K; ++p) x += u[b][p] * g[q + b][p * K + j];
            acc[j] = x;
          }
      }
      for (; q < ns; ++q) {
        const T* blk = (const T*)a.basis + (size_t)(s0 + q) * a.bstride;
        T u[K];
#pragma unroll
        for (int p = 0; p < K; ++p) u[p] = __ldg(blk + p * ld + i);
#pragma unroll
        for (int j = 0; j < K; ++j) {
          T x = acc[j];
#pragma unroll
          for (int p = 0; p < K; ++p) x += u[p] * g[q][p * K + j];
          acc[j] = x;
        }
      }
    }
    if (valid) {
#pragma unroll
      for (int j = 0; j < K; ++j) a.X[j * ldu + i] += double(acc[j]);
    }
  }
}

// ---- separability: nu_i = d_0i, deviation of d_ci / d_0i from t_c ---------------------------
__global__ void k_sep(const OpData op, const double* __restrict__ t, double* nu64,
                      double* nuinv64, float* nu32, float* nuinv32, double* dev) {
  __shared__ double red[MMAX][NT / 32];
  double mx[MMAX];
  for (int c = 0; c < MMAX; ++c) mx[c] = 0.0;
  const int64_t ld = op.ld;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < ld; i += (int64_t)gridDim.x * NT) {
    if (i >= op.n) {
      nu64[i] = 1.0;
      nuinv64[i] = 1.0;
      nu32[i] = 1.0f;
      nuinv32[i] = 1.0f;
      continue;
    }
    const double d0 = op.D64[i];
    nu64[i] = d0;
    nuinv64[i] = 1.0 / d0;
    nu32[i] = float(d0);
    nuinv32[i] = float(1.0 / d0);
    for (int c = 1; c < op.m; ++c) {
      const double r = op.D64[c * ld + i] - t[c] * d0;
      const double e = d0 > 0.0 ? fabs(r) / (fabs(t[c]) * d0 + 1e-300) : INFINITY;
      mx[c] = fmax(mx[c], e != e ? INFINITY : e);
    }
    if (!(d0 > 0.0)) mx[0] = INFINITY;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = 0; c < MMAX; ++c) {
    double v = mx[c];
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
    if (lane == 0) red[c][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < MMAX) {
    double v = 0.0;
    for (int w = 0; w < NT / 32; ++w) v = fmax(v, red[threadIdx.x][w]);
    dev[(size_t)blockIdx.x * MMAX + threadIdx.x] = v;
  }
}

#define LZ_DISPATCH_K(k, CALL)             \
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
cudaError_t launch_start(const Args& a, int ncta, cudaStream_t s) {
  const int k = a.op.k;
  if (a.op.E == 4) {
#define CALL(K) k_lz_start<K, 4, T><<<ncta, NT, 0, s>>>(a)
    LZ_DISPATCH_K(k, CALL)
#undef CALL
  } else {
#define CALL(K) k_lz_start<K, 0, T><<<ncta, NT, 0, s>>>(a)
    LZ_DISPATCH_K(k, CALL)
#undef CALL
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_a(const Args& a, int ncta, cudaStream_t s) {
  const int k = a.op.k;
  if (a.op.E == 4) {
#define CALL(K) k_lz_a<K, 4, T><<<ncta, NT, 0, s>>>(a)
    LZ_DISPATCH_K(k, CALL)
#undef CALL
  } else {
#define CALL(K) k_lz_a<K, 0, T><<<ncta, NT, 0, s>>>(a)
    LZ_DISPATCH_K(k, CALL)
#undef CALL
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_b(const Args& a, int ncta, cudaStream_t s) {
#define CALL(K) k_lz_b<K, T><<<ncta, NT, 0, s>>>(a)
  LZ_DISPATCH_K(a.op.k, CALL)
#undef CALL
  return cudaGetLastError();
}

// Staged FP32 passes: compiled for E = 4 (lattices and latitude-longitude spheres), no mass
// diagonal; other problems use the plain kernels.
bool staged_available(const OpData& op) {
  return (op.E == 4 || op.E == 12) && !op.has_w && op.ld % TILE_PX == 0;
}

template <int K, int E>
cudaError_t set_smem_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_lz_a_tma<K, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       LayoutA<K, E>::NST * LayoutA<K, E>::STAGE_BYTES);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_lz_b_tma<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              NST_B * LayoutB<K>::STAGE_BYTES);
}

cudaError_t launch_a_tma(const Args& a, int ncta, cudaStream_t s) {
#define CALL_E(K, E)                                                                         \
  do {                                                                                       \
    static const cudaError_t attr = set_smem_attrs<K, E>();                                  \
    if (attr != cudaSuccess) return attr;                                                    \
    k_lz_a_tma<K, E><<<ncta, WS_THREADS, LayoutA<K, E>::NST * LayoutA<K, E>::STAGE_BYTES, s>>>(a); \
  } while (0)
  if (a.op.E == 12) {
#define CALL(K) CALL_E(K, 12)
    LZ_DISPATCH_K(a.op.k, CALL)
#undef CALL
  } else {
#define CALL(K) CALL_E(K, 4)
    LZ_DISPATCH_K(a.op.k, CALL)
#undef CALL
  }
#undef CALL_E
  return cudaGetLastError();
}

cudaError_t launch_b_tma(const Args& a, int ncta, cudaStream_t s) {
#define CALL(K)                                                                              \
  do {                                                                                       \
    static const cudaError_t attr = set_smem_attrs<K, 4>();                                  \
    if (attr != cudaSuccess) return attr;                                                    \
    k_lz_b_tma<K><<<ncta, WS_THREADS, NST_B * LayoutB<K>::STAGE_BYTES, s>>>(a);             \
  } while (0)
  LZ_DISPATCH_K(a.op.k, CALL)
#undef CALL
  return cudaGetLastError();
}

cudaError_t launch_fin(const Args& a, cudaStream_t s) {
#define CALL(K) k_lz_fin<K><<<1, TILE_PX, 0, s>>>(a)
  LZ_DISPATCH_K(a.op.k, CALL)
#undef CALL
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_assemble(const Args& a, int ncta, cudaStream_t s) {
#define CALL(K) k_lz_assemble<K, T><<<ncta, NT, 0, s>>>(a)
  LZ_DISPATCH_K(a.op.k, CALL)
#undef CALL
  return cudaGetLastError();
}

template <typename T>
int occupancy(int kind, int k, int E) {
  int nb = 0;
  auto take = [&](const void* fn) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, NT, 0) != cudaSuccess) nb = 1;
  };
  auto take_ws = [&](const void* fn, int smem) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, WS_THREADS, smem) != cudaSuccess)
      nb = 1;
  };
  auto body = [&]() -> cudaError_t {
#define CALL(K)                                                                   \
  do {                                                                            \
    if (kind == 0) take(E == 4 ? (const void*)k_lz_a<K, 4, T> : (const void*)k_lz_a<K, 0, T>); \
    else if (kind == 1) take((const void*)k_lz_b<K, T>);                          \
    else if (kind == 2) take((const void*)k_lz_assemble<K, T>);                   \
    else if (kind == 3)                                                           \
      take(E == 4 ? (const void*)k_lz_start<K, 4, T> : (const void*)k_lz_start<K, 0, T>); \
    else if (kind == 4 && E == 12) {                                              \
      if (set_smem_attrs<K, 12>() != cudaSuccess) nb = 1;                         \
      else take_ws((const void*)k_lz_a_tma<K, 12>,                                \
                   LayoutA<K, 12>::NST * LayoutA<K, 12>::STAGE_BYTES);            \
    } else if (kind == 4) {                                                       \
      if (set_smem_attrs<K, 4>() != cudaSuccess) nb = 1;                          \
      else take_ws((const void*)k_lz_a_tma<K, 4>,                                 \
                   LayoutA<K, 4>::NST * LayoutA<K, 4>::STAGE_BYTES);              \
    } else {                                                                      \
      if (set_smem_attrs<K, 4>() != cudaSuccess) nb = 1;                          \
      else take_ws((const void*)k_lz_b_tma<K>, NST_B * LayoutB<K>::STAGE_BYTES);  \
    }                                                                             \
  } while (0)
    LZ_DISPATCH_K(k, CALL)
#undef CALL
    return cudaSuccess;
  };
  body();
  return nb > 0 ? nb : 1;
}

}  // namespace lz
}  // namespace sylv

// =============================================================================================
// host side
// =============================================================================================
using namespace sylv;
using namespace sylv::lz;

namespace {

int lz_fail(int code, const std::string& msg) {
  set_last_error(msg.c_str());
  return code;
}

int lz_cuda(cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  (void)cudaGetLastError();
  return lz_fail(e == cudaErrorMemoryAllocation ? SYLV_E_NOMEM : SYLV_E_CUDA, m);
}

#define LK(call)                                        \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return lz_cuda(_e, #call);   \
  } while (0)

struct Work {   // per inner type
  int elt = 0;                 // sizeof(T)
  int cap_blocks = 0;
  void* basis = nullptr;
  void* wbuf = nullptr;
  double* partial = nullptr;
  float* partAB = nullptr;     // staged passes: pass A | pass B partial sums
  int gpA = 0, gpB = 0;
  Ctl* ctl = nullptr;
  Coef* co = nullptr;
  double* hist = nullptr;      // histH | histB | (spare) | G, each cap x k*k
  Ctl* h_ctl = nullptr;        // pinned
  double* h_hist = nullptr;    // pinned, 3 x cap x k*k
  double* h_tot = nullptr;     // pinned, NVMAX
  double* h_G = nullptr;       // pinned, cap x k*k
  int ncta[6] = {0, 0, 0, 0, 0, 0};  // pass A, pass B, assembly, start, staged A, staged B
  int staged = 0;                     // FP32 passes run the bulk-copy staged kernels
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_iters = 0, graph_profile = 0;
  std::vector<cudaEvent_t> events;   // profile: 2 per step + 1
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evs0 = nullptr, evs1 = nullptr;
  ~Work() {
    cudaFree(basis);
    cudaFree(wbuf);
    cudaFree(partial);
    cudaFree(partAB);
    cudaFree(ctl);
    cudaFree(co);
    cudaFree(hist);
    cudaFreeHost(h_ctl);
    cudaFreeHost(h_hist);
    cudaFreeHost(h_tot);
    cudaFreeHost(h_G);
    if (graph) cudaGraphExecDestroy(graph);
    for (auto e : events) cudaEventDestroy(e);
    for (auto e : {ev0, ev1, evs0, evs1})
      if (e) cudaEventDestroy(e);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
};

struct Cache {
  int checked = 0;
  int status = SYLV_OK;        // SYLV_E_UNSUPPORTED when the problem is not separable
  std::string why;
  int k = 0, m = 0;
  double kappa0 = 0;
  std::vector<double> t, phi, rho, U, Uinv;   // U, Uinv row-major k x k
  double* nu64 = nullptr;
  double* nuinv64 = nullptr;
  float* nu32 = nullptr;
  float* nuinv32 = nullptr;
  std::unique_ptr<Work> work[2];
  ~Cache() {
    cudaFree(nu64);
    cudaFree(nuinv64);
    cudaFree(nu32);
    cudaFree(nuinv32);
  }
};

std::mutex g_mu;
std::map<sylv_handle, std::unique_ptr<Cache>> g_cache;

// Symmetric eigendecomposition of a small matrix by cyclic Jacobi rotations (FP64).
void jacobi_eig(int k, std::vector<double> A, std::vector<double>& w, std::vector<double>& V) {
  V.assign(k * k, 0.0);
  for (int i = 0; i < k; ++i) V[i * k + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int p = 0; p < k; ++p)
      for (int q = 0; q < k; ++q) {
        tot += A[p * k + q] * A[p * k + q];
        if (p != q) off += A[p * k + q] * A[p * k + q];
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) {
        const double apq = A[p * k + q];
        if (apq == 0.0) continue;
        const double theta = (A[q * k + q] - A[p * k + p]) / (2.0 * apq);
        const double tt = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(tt * tt + 1.0), s = tt * c;
        for (int r = 0; r < k; ++r) {
          const double arp = A[r * k + p], arq = A[r * k + q];
          A[r * k + p] = c * arp - s * arq;
          A[r * k + q] = s * arp + c * arq;
        }
        for (int r = 0; r < k; ++r) {
          const double apr = A[p * k + r], aqr = A[q * k + r];
          A[p * k + r] = c * apr - s * aqr;
          A[q * k + r] = s * apr + c * aqr;
        }
        for (int r = 0; r < k; ++r) {
          const double vrp = V[r * k + p], vrq = V[r * k + q];
          V[r * k + p] = c * vrp - s * vrq;
          V[r * k + q] = s * vrp + c * vrq;
        }
      }
  }
  w.resize(k);
  for (int i = 0; i < k; ++i) w[i] = A[i * k + i];
}

// S = R^T R (upper R) on the host; false when not positive definite.
bool hchol_upper(int k, const double* S, double* R) {
  for (int j = 0; j < k; ++j) {
    double d = S[j * k + j];
    for (int p = 0; p < j; ++p) d -= R[p * k + j] * R[p * k + j];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    const double r = std::sqrt(d);
    R[j * k + j] = r;
    for (int i = j + 1; i < k; ++i) {
      double v = S[j * k + i];
      for (int p = 0; p < j; ++p) v -= R[p * k + j] * R[p * k + i];
      R[j * k + i] = v / r;
    }
    for (int i = 0; i < j; ++i) R[j * k + i] = 0.0;
  }
  return true;
}

void hsolve(int k, const double* R, const double* b, double* x) {
  std::vector<double> y(k);
  for (int i = 0; i < k; ++i) {
    double v = b[i];
    for (int p = 0; p < i; ++p) v -= R[p * k + i] * y[p];
    y[i] = v / R[i * k + i];
  }
  for (int i = k - 1; i >= 0; --i) {
    double v = y[i];
    for (int p = i + 1; p < k; ++p) v -= R[i * k + p] * x[p];
    x[i] = v / R[i * k + i];
  }
}

void hinv_upper(int k, const double* R, double* Ri) {
  for (int c = 0; c < k; ++c)
    for (int r = k - 1; r >= 0; --r) {
      double v = r == c ? 1.0 : 0.0;
      for (int p = r + 1; p < k; ++p) v -= R[r * k + p] * Ri[p * k + c];
      Ri[r * k + c] = r > c ? 0.0 : v / R[r * k + r];
    }
}

// Separability test and the quantities of eq. Axb-Sylv that do not depend on the right-hand side.
int prepare(sylv_handle h, const OpData& op, Cache& C, cudaStream_t s) {
  C.checked = 1;
  C.k = op.k;
  C.m = op.m;
  const int k = op.k, m = op.m;
  for (int j = 1; j < k; ++j)
    if (op.kappa64[j] != op.kappa64[0]) {
      C.status = SYLV_E_UNSUPPORTED;
      C.why = "Sylvester solver: the prior shapes differ (kappa_j not all equal)";
      return SYLV_OK;
    }
  C.kappa0 = op.kappa64[0];
  // t_c from pixel 0
  std::vector<double> d0(m);
  LK(cudaMemcpy2DAsync(d0.data(), sizeof(double), op.D64, (size_t)op.ld * sizeof(double),
                       sizeof(double), m, cudaMemcpyDeviceToHost, s));
  LK(cudaStreamSynchronize(s));
  if (!(d0[0] > 0.0)) {
    C.status = SYLV_E_UNSUPPORTED;
    C.why = "Sylvester solver: the noise weight d_0i must be positive (N invertible)";
    return SYLV_OK;
  }
  C.t.resize(m);
  for (int c = 0; c < m; ++c) C.t[c] = d0[c] / d0[0];
  const size_t ld = (size_t)op.ld;
  LK(cudaMalloc(&C.nu64, ld * sizeof(double)));
  LK(cudaMalloc(&C.nuinv64, ld * sizeof(double)));
  LK(cudaMalloc(&C.nu32, ld * sizeof(float)));
  LK(cudaMalloc(&C.nuinv32, ld * sizeof(float)));
  int dev = 0, nsm = 0;
  LK(cudaGetDevice(&dev));
  LK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int ncta = std::max(1, std::min<int>(nsm * 4, (int)((op.n + NT - 1) / NT)));
  double *dt = nullptr, *ddev = nullptr;
  LK(cudaMalloc(&dt, MMAX * sizeof(double)));
  cudaError_t e = cudaMalloc(&ddev, (size_t)ncta * MMAX * sizeof(double));
  if (e != cudaSuccess) {
    cudaFree(dt);
    return lz_cuda(e, "cudaMalloc");
  }
  std::vector<double> tpad(MMAX, 0.0), devh((size_t)ncta * MMAX);
  for (int c = 0; c < m; ++c) tpad[c] = C.t[c];
  e = cudaMemcpyAsync(dt, tpad.data(), MMAX * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_sep<<<ncta, NT, 0, s>>>(op, dt, C.nu64, C.nuinv64, C.nu32, C.nuinv32, ddev);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(devh.data(), ddev, devh.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dt);
  cudaFree(ddev);
  if (e != cudaSuccess) return lz_cuda(e, "separability check");
  double worst = 0.0;
  for (double v : devh) worst = std::max(worst, std::isnan(v) ? INFINITY : v);
  if (!(worst <= 1e-10)) {
    C.status = SYLV_E_UNSUPPORTED;
    char buf[160];
    std::snprintf(buf, sizeof(buf),
                  "Sylvester solver: noise precision is not separable (d_ci != t_c d_0i, "
                  "relative deviation %.3g)", worst);
    C.why = buf;
    return SYLV_OK;
  }
  // Lhat = A^T T A P^{-1} = U diag(rho) U^{-1}, U = P^{1/2} Ut, from the symmetric matrix
  // P^{-1/2} A^T T A P^{-1/2} = Ut diag(rho) Ut^T (the second Lemma of Sec. 3.3)
  C.phi.assign(op.tau64, op.tau64 + k);
  std::vector<double> Sm(k * k, 0.0), Ut;
  for (int p = 0; p < k; ++p)
    for (int q = 0; q < k; ++q) {
      double v = 0.0;
      for (int c = 0; c < m; ++c) v += op.A64[c * k + p] * C.t[c] * op.A64[c * k + q];
      Sm[p * k + q] = v / std::sqrt(C.phi[p] * C.phi[q]);
    }
  jacobi_eig(k, Sm, C.rho, Ut);
  C.U.assign(k * k, 0.0);
  C.Uinv.assign(k * k, 0.0);
  for (int p = 0; p < k; ++p)
    for (int q = 0; q < k; ++q) {
      C.U[p * k + q] = std::sqrt(C.phi[p]) * Ut[p * k + q];
      C.Uinv[q * k + p] = Ut[p * k + q] / std::sqrt(C.phi[p]);   // U^T P^{-1}
    }
  C.status = SYLV_OK;
  return SYLV_OK;
}

size_t env_mb(const char* name, size_t dflt) {
  const char* v = std::getenv(name);
  if (!v || !*v) return dflt;
  return (size_t)std::strtoull(v, nullptr, 10);
}

template <typename T>
int ensure_work(const OpData& op, Cache& C, int maxit, std::unique_ptr<Work>& slot) {
  const int k = op.k;
  const size_t block = (size_t)k * op.ld * sizeof(T);
  size_t free_b = 0, total_b = 0;
  LK(cudaMemGetInfo(&free_b, &total_b));
  // basis budget: SYLV_LZ_BASIS_MB, else 60 % of the free memory, at most 384 blocks
  size_t budget = env_mb("SYLV_LZ_BASIS_MB", 0) << 20;
  if (budget == 0) budget = (size_t)(0.6 * (double)free_b);
  long want = std::min<long>((long)maxit + 1, 384);
  if (slot) {
    const size_t have_budget = (size_t)slot->cap_blocks * block;
    if (slot->cap_blocks >= want || have_budget >= budget) return SYLV_OK;
  }
  slot.reset();
  long cap = std::min<long>(want, (long)(budget / block));
  if (cap < 2) return lz_fail(SYLV_E_NOMEM, "Sylvester solver: no room for two basis blocks");
  std::unique_ptr<Work> w(new Work());
  w->elt = sizeof(T);
  w->cap_blocks = (int)cap;
  LK(cudaMalloc(&w->basis, (size_t)cap * block));
  LK(cudaMalloc(&w->wbuf, block));
  int dev = 0, nsm = 0;
  LK(cudaGetDevice(&dev));
  LK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t ntiles = (op.n + NT - 1) / NT;
  // SYLV_LZ_STAGED=0 keeps the FP32 passes on the plain kernels
  const char* sv = std::getenv("SYLV_LZ_STAGED");
  w->staged = sizeof(T) == 4 && staged_available(op) && !(sv && sv[0] == '0');
  for (int kind = 0; kind < 6; ++kind) {
    if (kind >= 4 && !w->staged) continue;
    const int occ = occupancy<T>(kind, k, op.E);
    w->ncta[kind] = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * occ, ntiles));
  }
  const int maxcta = *std::max_element(w->ncta, w->ncta + 6);
  LK(cudaMalloc(&w->partial, (size_t)maxcta * NVMAX * sizeof(double)));
  if (w->staged) {   // value-major, stride rounded up to 32 CTAs; the padding stays zero
    w->gpA = (w->ncta[4] + 31) / 32 * 32;
    w->gpB = (w->ncta[5] + 31) / 32 * 32;
    const size_t nf = (size_t)(w->gpA + w->gpB) * NSMAX;
    LK(cudaMalloc(&w->partAB, nf * sizeof(float)));
    LK(cudaMemset(w->partAB, 0, nf * sizeof(float)));
  }
  LK(cudaMalloc(&w->ctl, sizeof(Ctl)));
  LK(cudaMemset(w->ctl, 0, sizeof(Ctl)));
  LK(cudaMalloc(&w->co, sizeof(Coef)));
  LK(cudaMemset(w->co, 0, sizeof(Coef)));
  LK(cudaMalloc(&w->hist, (size_t)4 * cap * k * k * sizeof(double)));
  LK(cudaMallocHost(&w->h_ctl, sizeof(Ctl)));
  LK(cudaMallocHost(&w->h_hist, (size_t)3 * cap * k * k * sizeof(double)));
  LK(cudaMallocHost(&w->h_tot, NVMAX * sizeof(double)));
  LK(cudaMallocHost(&w->h_G, (size_t)cap * k * k * sizeof(double)));
  LK(cudaStreamCreateWithFlags(&w->cap_stream, cudaStreamNonBlocking));
  LK(cudaEventCreate(&w->ev0));
  LK(cudaEventCreate(&w->ev1));
  LK(cudaEventCreate(&w->evs0));
  LK(cudaEventCreate(&w->evs1));
  slot = std::move(w);
  return SYLV_OK;
}

template <typename T>
Args make_args(const OpData& op, const Cache& C, Work& w) {
  Args a;
  std::memset(&a, 0, sizeof(a));
  a.op = op;
  a.nu64 = C.nu64;
  a.nuinv64 = C.nuinv64;
  a.nu32 = C.nu32;
  a.nuinv32 = C.nuinv32;
  a.basis = w.basis;
  a.bstride = (int64_t)op.k * op.ld;
  a.wbuf = w.wbuf;
  a.partial = w.partial;
  a.partA = w.partAB;
  a.partB = w.partAB ? w.partAB + (size_t)w.gpA * NSMAX : nullptr;
  a.gpA = w.gpA;
  a.gpB = w.gpB;
  a.ctl = w.ctl;
  a.co = w.co;
  const size_t kk = (size_t)op.k * op.k;
  a.histH = w.hist;
  a.histB = w.hist + (size_t)w.cap_blocks * kk;
  a.G = w.hist + (size_t)3 * w.cap_blocks * kk;
  a.kap2 = C.kappa0 * C.kappa0;
  for (int j = 0; j < op.k; ++j) a.phinv[j] = 1.0 / C.phi[j];
  for (int p = 0; p < op.k; ++p)
    for (int q = 0; q < op.k; ++q) a.U[p * KMAX + q] = C.U[p * op.k + q];
  return a;
}

template <typename T>
int launch_steps(Work& w, const Args& a, int iters, cudaStream_t s, bool capture, bool prof) {
  for (int it = 0; it < iters; ++it) {
    if (w.staged) LK(launch_a_tma(a, w.ncta[4], s));
    else LK(launch_a<T>(a, w.ncta[0], s));
    if (prof)
      LK(capture ? cudaEventRecordWithFlags(w.events[2 * it + 1], s, cudaEventRecordExternal)
                 : cudaEventRecord(w.events[2 * it + 1], s));
    if (w.staged) LK(launch_b_tma(a, w.ncta[5], s));
    else LK(launch_b<T>(a, w.ncta[1], s));
    // staged passes: the factor of the chunk's last step, for the poll
    if (w.staged && it == iters - 1) LK(launch_fin(a, s));
    if (prof)
      LK(capture ? cudaEventRecordWithFlags(w.events[2 * it + 2], s, cudaEventRecordExternal)
                 : cudaEventRecord(w.events[2 * it + 2], s));
  }
  return SYLV_OK;
}

template <typename T>
int ensure_graph(Work& w, const Args& a, int iters, int profile) {
  if (w.graph && w.graph_iters == iters && w.graph_profile == profile) return SYLV_OK;
  if (w.graph) {
    cudaGraphExecDestroy(w.graph);
    w.graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  LK(cudaStreamBeginCapture(w.cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = SYLV_OK;
  if (profile) {
    cudaError_t e = cudaEventRecordWithFlags(w.events[0], w.cap_stream, cudaEventRecordExternal);
    if (e != cudaSuccess) rc = lz_cuda(e, "event record in capture");
  }
  if (rc == SYLV_OK) rc = launch_steps<T>(w, a, iters, w.cap_stream, true, profile != 0);
  cudaError_t e = cudaStreamEndCapture(w.cap_stream, &g);
  if (rc != SYLV_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return lz_cuda(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&w.graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return lz_cuda(e, "cudaGraphInstantiate");
  w.graph_iters = iters;
  w.graph_profile = profile;
  return SYLV_OK;
}

// Residual estimate of Algorithm 5, advanced one Lanczos step at a time: for every shift rho_l
// the block LDL^T of T_s + rho_l I gains one pivot block D_s = H_s + rho_l I - B_s D_{s-1}^{-1}
// B_s^T and the forward substitution of E_1 c_l one block y_s = -B_s D_{s-1}^{-1} y_{s-1}; the
// last block of the shifted solution is z_l = D_s^{-1} y_s and gamma = sum_l ||B_{s+1} z_l||^2.
struct ShiftGamma {
  int k = 0, s = 0;
  std::vector<double> rho, D, y, R;   // per shift: D_s (k x k), y_s (k), chol factor of D_s
  void start(int k_, const double* c /*k x k, column l*/, const std::vector<double>& rho_) {
    k = k_;
    s = 0;
    rho = rho_;
    D.assign((size_t)k * k * k, 0.0);
    R.assign((size_t)k * k * k, 0.0);
    y.assign((size_t)k * k, 0.0);
    for (int l = 0; l < k; ++l)
      for (int a = 0; a < k; ++a) y[l * k + a] = c[a * k + l];
  }
  // H: H_{s+1}; Bprev: B_{s+1} (unused on the first step); Bnext: B_{s+2}.  Returns false if a
  // pivot block is not positive definite.
  bool advance(const double* H, const double* Bprev, const double* Bnext, double* gamma) {
    const size_t kk = (size_t)k * k;
    std::vector<double> X(kk), tmp(k), tmp2(k), Dn(kk), yn(k), z(k);
    double g = 0.0;
    for (int l = 0; l < k; ++l) {
      double* Dl = D.data() + l * kk;
      double* Rl = R.data() + l * kk;
      double* yl = y.data() + l * k;
      if (s == 0) {
        for (size_t t = 0; t < kk; ++t) Dn[t] = H[t];
        for (int a = 0; a < k; ++a) yn[a] = yl[a];
      } else {
        for (int c = 0; c < k; ++c) {   // X = D_{s-1}^{-1} B^T
          for (int a = 0; a < k; ++a) tmp[a] = Bprev[c * k + a];
          hsolve(k, Rl, tmp.data(), tmp2.data());
          for (int a = 0; a < k; ++a) X[a * k + c] = tmp2[a];
        }
        for (int a = 0; a < k; ++a) {
          double v = 0.0;
          for (int b = 0; b < k; ++b) v -= X[b * k + a] * yl[b];
          yn[a] = v;
        }
        for (int a = 0; a < k; ++a)
          for (int b = 0; b < k; ++b) {
            double v = 0.0;
            for (int p = 0; p < k; ++p) v += Bprev[a * k + p] * X[p * k + b];
            Dn[a * k + b] = H[a * k + b] - v;
          }
        for (int a = 0; a < k; ++a)
          for (int b = a + 1; b < k; ++b) Dn[a * k + b] = Dn[b * k + a] = 0.5 * (Dn[a * k + b] + Dn[b * k + a]);
      }
      for (int a = 0; a < k; ++a) Dn[a * k + a] += rho[l];
      if (!hchol_upper(k, Dn.data(), Rl)) return false;
      for (size_t t = 0; t < kk; ++t) Dl[t] = Dn[t];
      for (int a = 0; a < k; ++a) yl[a] = yn[a];
      hsolve(k, Rl, yl, z.data());
      for (int a = 0; a < k; ++a) {
        double v = 0.0;
        for (int b = a; b < k; ++b) v += Bnext[a * k + b] * z[b];
        g += v * v;
      }
    }
    ++s;
    *gamma = g;
    return std::isfinite(g);
  }
};

// Z of eq. soln-constr from the stored H_s, B_{s+1}: for each shift l the block LDL^T solve of
// (T_j + rho_l I) zhat_l = E_1 c_l, then Z = Zhat U^{-1} and G'_s = N_s Z_s.
void coefficients(int k, int j, const Cache& C, const double* c /*k x k*/, const double* hH,
                  const double* hB, const double* hN, double* Gp) {
  const size_t kk = (size_t)k * k;
  std::vector<double> Zh((size_t)j * kk, 0.0);   // block s: k x k, column l
  std::vector<double> Rf((size_t)j * kk), Xs((size_t)j * kk), y((size_t)j * k), D(kk), tmp(k),
      tmp2(k);
  for (int l = 0; l < k; ++l) {
    const double rho = C.rho[l];
    for (int s = 0; s < j; ++s) {
      const double* H = hH + s * kk;
      if (s == 0) {
        for (size_t t = 0; t < kk; ++t) D[t] = H[t];
        for (int a = 0; a < k; ++a) y[a] = c[a * k + l];
      } else {
        const double* Bs = hB + (s - 1) * kk;            // B_{s+1} in 1-based step numbering
        double* X = Xs.data() + s * kk;                   // D_{s-1}^{-1} B^T
        const double* Rp = Rf.data() + (s - 1) * kk;
        for (int cc = 0; cc < k; ++cc) {
          for (int a = 0; a < k; ++a) tmp[a] = Bs[cc * k + a];
          hsolve(k, Rp, tmp.data(), tmp2.data());
          for (int a = 0; a < k; ++a) X[a * k + cc] = tmp2[a];
        }
        for (int a = 0; a < k; ++a) {
          double v = 0.0;
          for (int b = 0; b < k; ++b) v -= X[b * k + a] * y[(s - 1) * k + b];
          y[s * k + a] = v;
        }
        for (int a = 0; a < k; ++a)
          for (int b = 0; b < k; ++b) {
            double v = 0.0;
            for (int p = 0; p < k; ++p) v += Bs[a * k + p] * X[p * k + b];
            D[a * k + b] = H[a * k + b] - v;
          }
        for (int a = 0; a < k; ++a)
          for (int b = a + 1; b < k; ++b) {
            const double mm = 0.5 * (D[a * k + b] + D[b * k + a]);
            D[a * k + b] = D[b * k + a] = mm;
          }
      }
      for (int a = 0; a < k; ++a) D[a * k + a] += rho;
      if (!hchol_upper(k, D.data(), Rf.data() + s * kk)) {
        // cannot happen for an SPD T_j; keep the partial sum finite
        for (size_t t = 0; t < kk; ++t) Rf[s * kk + t] = (t % (k + 1) == 0) ? 1e300 : 0.0;
      }
    }
    // back substitution: z_j = D_j^{-1} y_j, z_s = D_s^{-1} y_s - X_{s+1} z_{s+1}
    std::vector<double> z((size_t)j * k);
    for (int s = j - 1; s >= 0; --s) {
      hsolve(k, Rf.data() + s * kk, y.data() + s * k, z.data() + s * k);
      if (s + 1 < j) {
        const double* X = Xs.data() + (s + 1) * kk;
        for (int a = 0; a < k; ++a) {
          double v = 0.0;
          for (int b = 0; b < k; ++b) v += X[a * k + b] * z[(s + 1) * k + b];
          z[s * k + a] -= v;
        }
      }
    }
    for (int s = 0; s < j; ++s)
      for (int a = 0; a < k; ++a) Zh[s * kk + a * k + l] = z[s * k + a];
  }
  for (int s = 0; s < j; ++s) {
    double Zs[KMAX * KMAX];
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) {
        double v = 0.0;
        for (int p = 0; p < k; ++p) v += Zh[s * kk + a * k + p] * C.Uinv[p * k + b];
        Zs[a * k + b] = v;
      }
    const double* N = hN + s * kk;
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) {
        double v = 0.0;
        for (int p = a; p < k; ++p) v += N[a * k + p] * Zs[p * k + b];
        Gp[s * kk + a * k + b] = v;
      }
  }
}

template <typename T>
int run(sylv_handle h, const OpData& op, Cache& C, const double* B, double* X, int nrhs,
        const sylv_opts& o, sylv_info* info, cudaStream_t s) {
  std::unique_ptr<Work>& slot = C.work[sizeof(T) == 8 ? 1 : 0];
  int rc = ensure_work<T>(op, C, o.maxit, slot);
  if (rc != SYLV_OK) return rc;
  Work& w = *slot;
  const int k = op.k;
  const size_t kk = (size_t)k * k;
  const int iters = o.check_every > 0 ? o.check_every : 8;
  const bool prof = o.profile != 0;
  if (prof && (int)w.events.size() < 2 * iters + 1) {
    for (auto e : w.events) cudaEventDestroy(e);
    w.events.assign(2 * iters + 1, nullptr);
    for (auto& e : w.events) LK(cudaEventCreate(&e));
    if (w.graph) {
      cudaGraphExecDestroy(w.graph);
      w.graph = nullptr;
    }
  }
  Args a = make_args<T>(op, C, w);
  if (o.use_graph) {
    rc = ensure_graph<T>(w, a, iters, prof ? 1 : 0);
    if (rc != SYLV_OK) return rc;
  }
  sylv_info inf;
  std::memset(&inf, 0, sizeof(inf));
  inf.status = SYLV_OK;
  inf.tile = NT;
  inf.slots_mult = 1;
  inf.apply_staged = w.staged;
  inf.update_staged = w.staged;
  double ms_a = 0, ms_b = 0, ms_res = 0;
  long launches = 0;
  int polls = 0;
  LK(cudaEventRecord(w.ev0, s));
  if (!o.use_x0) LK(cudaMemsetAsync(X, 0, (size_t)nrhs * k * op.ldu * sizeof(double), s));
  int worst = SYLV_OK;
  for (int r = 0; r < nrhs; ++r) {
    a.B = B + (size_t)r * k * op.ldu;
    a.X = X + (size_t)r * k * op.ldu;
    a.ldu = op.ldu;
    int total = 0, outer = 0, status = SYLV_E_NOT_CONVERGED;
    double bnorm2 = 0.0, relres = 0.0;
    bool first = true;
    while (true) {
      a.x0_zero = (first && !o.use_x0) ? 1 : 0;
      if (prof) LK(cudaEventRecord(w.evs0, s));
      LK(launch_start<T>(a, w.ncta[3], s));
      if (prof) LK(cudaEventRecord(w.evs1, s));
      ++launches;
      LK(cudaMemcpyAsync(w.h_tot, w.co->tot, NVMAX * sizeof(double), cudaMemcpyDeviceToHost, s));
      LK(cudaStreamSynchronize(s));
      ++polls;
      if (prof) {
        float ms = 0;
        LK(cudaEventElapsedTime(&ms, w.evs0, w.evs1));
        ms_res += ms;
        ++inf.n_residual;
      }
      const int NS = k * (k + 1) / 2;
      const double rr = w.h_tot[NS];
      if (first) bnorm2 = w.h_tot[NS + 1];
      first = false;
      if (!std::isfinite(rr)) {
        status = SYLV_E_BREAKDOWN;
        break;
      }
      relres = bnorm2 > 0.0 ? std::sqrt(rr / bnorm2) : 0.0;
      if (bnorm2 == 0.0 || relres <= o.tol) {
        status = SYLV_OK;
        break;
      }
      if (outer >= o.max_outer || total >= o.maxit) break;
      // start block: Gram matrix of C = Yhat U, column scaling, Cholesky QR
      double Gm[KMAX * KMAX], Sh[KMAX * KMAX], Rb[KMAX * KMAX], sc[KMAX];
      int t = 0;
      for (int p = 0; p < k; ++p)
        for (int q = p; q < k; ++q, ++t) Gm[p * k + q] = Gm[q * k + p] = w.h_tot[t];
      bool ok = true;
      for (int p = 0; p < k; ++p) {
        sc[p] = std::sqrt(Gm[p * k + p]);
        if (!(sc[p] > 0.0) || !std::isfinite(sc[p])) ok = false;
      }
      if (ok) {
        for (int p = 0; p < k; ++p)
          for (int q = 0; q < k; ++q) Sh[p * k + q] = Gm[p * k + q] / (sc[p] * sc[q]);
        ok = hchol_upper(k, Sh, Rb);
      }
      if (!ok) {
        status = SYLV_E_BREAKDOWN;
        break;
      }
      // the start block C = Yhat U is raw block 1: C = V_1 B_1 with B_1 = Rb Sigma, which is
      // also B_0 U (Yhat = V_1 Rb Sigma U^{-1})
      Coef init;
      std::memset(&init, 0, sizeof(init));
      double cU[KMAX * KMAX];
      for (int p = 0; p < k; ++p) {
        for (int q = 0; q < k; ++q) {
          cU[p * k + q] = Rb[p * k + q] * sc[q];
          init.Rc[p * KMAX + q] = cU[p * k + q];
        }
        init.rci[p] = 1.0 / cU[p * k + p];
      }
      std::memcpy(init.R2[1], init.Rc, sizeof(init.Rc));   // staged passes read slot 1 at s = 1
      std::memcpy(init.ri2[1], init.rci, sizeof(init.rci));
      double nB0 = 0.0;   // ||B_0||_F^2, B_0 = (B_0 U) U^{-1}
      for (int p = 0; p < k; ++p)
        for (int q = 0; q < k; ++q) {
          double v = 0.0;
          for (int u = 0; u < k; ++u) v += cU[p * k + u] * C.Uinv[u * k + q];
          nB0 += v * v;
        }
      // inner target: the residual reduction still needed (safety 0.5), no finer than the
      // inner precision delivers in one run
      const double need = 0.5 * o.tol / relres;
      const double eps = o.precision == SYLV_PREC_MIXED ? std::max(o.inner_tol, need) : need;
      const double thr = eps * eps * nB0;
      Ctl c0;
      std::memset(&c0, 0, sizeof(c0));
      c0.cap = std::min(w.cap_blocks - 1, o.maxit - total);
      LK(cudaMemcpyAsync(w.co, &init, sizeof(Coef) - sizeof(init.tot), cudaMemcpyHostToDevice, s));
      *w.h_ctl = c0;
      LK(cudaMemcpyAsync(w.ctl, w.h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, s));
      ++outer;
      // Lanczos steps in chunks of `iters`; at every poll the host reads the new H_s, B_{s+1}
      // and advances the residual estimate; the run ends at the first step that meets it
      const size_t cb = (size_t)w.cap_blocks * kk;
      ShiftGamma sg;
      sg.start(k, cU, C.rho);
      const long max_chunks = (long)c0.cap / iters + 2;
      long chunks = 0;
      int j = 0, seen = 0;
      bool stop = false;
      while (!stop) {
        if (o.use_graph) {
          LK(cudaGraphLaunch(w.graph, s));
        } else {
          if (prof) LK(cudaEventRecord(w.events[0], s));
          rc = launch_steps<T>(w, a, iters, s, false, prof);
          if (rc != SYLV_OK) return rc;
        }
        launches += 2L * iters + (w.staged ? 1 : 0);
        const int cnt = std::min(iters, c0.cap - seen);
        LK(cudaMemcpyAsync(w.h_ctl, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        if (cnt > 0) {
          LK(cudaMemcpyAsync(w.h_hist + seen * kk, a.histH + seen * kk, cnt * kk * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
          LK(cudaMemcpyAsync(w.h_hist + cb + seen * kk, a.histB + seen * kk,
                             cnt * kk * sizeof(double), cudaMemcpyDeviceToHost, s));
        }
        LK(cudaStreamSynchronize(s));
        ++polls;
        ++chunks;
        if (prof) {
          for (int it = 0; it < iters; ++it) {
            float x = 0, y = 0;
            LK(cudaEventElapsedTime(&x, w.events[2 * it], w.events[2 * it + 1]));
            LK(cudaEventElapsedTime(&y, w.events[2 * it + 1], w.events[2 * it + 2]));
            ms_a += x;
            ms_b += y;
          }
        }
        if (w.h_ctl->err)
          return lz_fail(SYLV_E_TIMEOUT, "Sylvester solver: a bounded device-side wait expired");
        const int step = w.h_ctl->step;
        const int done = w.h_ctl->done;
        // steps with B_{s+1} recorded (a breakdown step has none)
        const int usable = done == BREAKDOWN ? step - 1 : step;
        while (seen < usable && !stop) {
          double g = 0.0;
          const double* Bprev = seen > 0 ? w.h_hist + cb + (seen - 1) * kk : nullptr;
          if (!sg.advance(w.h_hist + seen * kk, Bprev, w.h_hist + cb + seen * kk, &g)) {
            stop = true;
            j = seen;
            break;
          }
          ++seen;
          if (g <= thr) {
            stop = true;
            j = seen;
          }
        }
        if (!stop && done != RUNNING) {
          stop = true;
          j = step;
        }
        if (!stop && chunks > max_chunks) {
          stop = true;
          j = seen;
        }
      }
      if (prof) {
        inf.n_apply += (int)(chunks * iters);
        inf.n_update += (int)(chunks * iters);
      }
      total += j;
      if (j == 0) {
        status = SYLV_E_BREAKDOWN;
        break;
      }
      // H_s of a breakdown step was recorded by its pass A but not yet copied
      if (j > seen)
        LK(cudaMemcpyAsync(w.h_hist + seen * kk, a.histH + seen * kk,
                           (size_t)(j - seen) * kk * sizeof(double), cudaMemcpyDeviceToHost, s));
      // coefficients on the host, then X += sum_s Vt_s G'_s
      LK(cudaStreamSynchronize(s));
      // normalizers N_s = B_s^{-1} of the raw blocks (B_1 = Rb Sigma, B_s = recorded B for s > 1)
      double* hN = w.h_hist + 2 * cb;
      for (int t = 0; t < j; ++t)
        hinv_upper(k, t == 0 ? cU : w.h_hist + cb + (size_t)(t - 1) * kk, hN + (size_t)t * kk);
      coefficients(k, j, C, cU, w.h_hist, w.h_hist + cb, hN, w.h_G);
      LK(cudaMemcpyAsync((void*)a.G, w.h_G, (size_t)j * kk * sizeof(double), cudaMemcpyHostToDevice, s));
      a.nsteps = j;
      if (prof) LK(cudaEventRecord(w.evs0, s));
      LK(launch_assemble<T>(a, w.ncta[2], s));
      if (prof) LK(cudaEventRecord(w.evs1, s));
      ++launches;
      if (prof) {
        LK(cudaStreamSynchronize(s));
        float ms = 0;
        LK(cudaEventElapsedTime(&ms, w.evs0, w.evs1));
        ms_res += ms;
      }
    }
    inf.iterations = std::max(inf.iterations, total);
    inf.outer = std::max(inf.outer, outer);
    inf.relres = std::max(inf.relres, relres);
    if (status != SYLV_OK && (worst == SYLV_OK || status == SYLV_E_BREAKDOWN)) worst = status;
  }
  LK(cudaEventRecord(w.ev1, s));
  LK(cudaEventSynchronize(w.ev1));
  float ms_total = 0;
  LK(cudaEventElapsedTime(&ms_total, w.ev0, w.ev1));
  inf.status = worst;
  inf.polls = polls;
  inf.ms_total = ms_total;
  inf.ms_apply = ms_a;
  inf.ms_update = ms_b;
  inf.ms_residual = ms_res;
  inf.launches = (int)std::min<long>(launches, INT32_MAX);
  if (info) *info = inf;
  if (worst == SYLV_E_NOT_CONVERGED) set_last_error("Sylvester solver: tolerance not reached");
  if (worst == SYLV_E_BREAKDOWN) set_last_error("Sylvester solver: breakdown (non-finite or singular block)");
  return worst;
}

}  // namespace

namespace sylv {
void lanczos_release(sylv_handle h) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache.erase(h);
}
}  // namespace sylv

extern "C" int sylv_solve_sylvester(sylv_handle h, const double* B, double* X, int nrhs,
                                    const sylv_opts* o_in, sylv_info* info, sylv_stream s) {
  if (!h || !B || !X) return lz_fail(SYLV_E_INVALID, "NULL handle or buffer");
  if (nrhs < 1 || nrhs > RMAX) return lz_fail(SYLV_E_INVALID, "nrhs out of 1..SYLV_MAX_RHS");
  sylv_opts o;
  if (o_in) o = *o_in;
  else sylv_opts_default(&o);
  if (!(o.tol > 0.0) || !(o.tol < 1.0)) return lz_fail(SYLV_E_INVALID, "opts.tol must be in (0,1)");
  if (o.precision == SYLV_PREC_MIXED && (!(o.inner_tol > 0.0) || !(o.inner_tol < 1.0)))
    return lz_fail(SYLV_E_INVALID, "opts.inner_tol must be in (0,1)");
  if (o.precision != SYLV_PREC_MIXED && o.precision != SYLV_PREC_F64)
    return lz_fail(SYLV_E_INVALID, "opts.precision");
  if (o.maxit < 1 || o.max_outer < 1) return lz_fail(SYLV_E_INVALID, "opts.maxit/max_outer");
  if (o.check_every < 0 || o.check_every > 4096) return lz_fail(SYLV_E_INVALID, "opts.check_every");
  OpData op;
  int device = 0;
  int rc = handle_view(h, &op, &device);
  if (rc != SYLV_OK) return lz_fail(rc, "invalid handle");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  std::lock_guard<std::mutex> lk(g_mu);
  auto& cp = g_cache[h];
  if (!cp) cp.reset(new Cache());
  Cache& C = *cp;
  cudaStream_t st = (cudaStream_t)s;
  if (!C.checked) rc = prepare(h, op, C, st);
  if (rc == SYLV_OK && C.status != SYLV_OK) rc = lz_fail(C.status, C.why);
  if (rc == SYLV_OK)
    rc = o.precision == SYLV_PREC_F64 ? run<double>(h, op, C, B, X, nrhs, o, info, st)
                                      : run<float>(h, op, C, B, X, nrhs, o, info, st);
  if (prev != device) cudaSetDevice(prev);
  return rc;
}
