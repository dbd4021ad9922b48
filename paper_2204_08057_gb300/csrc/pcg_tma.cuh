// FP32 inner-iteration kernels with bulk-copy (TMA) staging and warp specialisation.
//
// Same arithmetic as k_inner_apply / k_inner_update, restructured for the memory system.
// A unit is one (tile, column) pair; every contiguous stream a unit needs (its rows of z, p, q
// or r, q, the noise maps D, the ELL rows of L and its diagonal, or the stored preconditioner
// factor; TILE_PX values each) is brought into shared memory by cp.async.bulk
// copies.  One producer warp issues the copies of unit u into stage u % NSTAGE once the
// consumers have released that stage (an "empty" mbarrier with one arrival per consumer
// warp), and the copies complete on the stage's "full" mbarrier.  Eight consumer warps (one
// pixel per thread) wait only on "full", compute, and release the stage: there is no
// CTA-wide barrier per unit, so warps drift independently and the copies stay in flight.
// The loads need no registers while in flight; the only per-thread global loads left are the
// stencil gathers that fall outside the tile (neighbours one image row away) and, in the
// operator kernel, the pixel's row of d (coalesced; d += alpha p of the previous iteration is
// done there, where p is read anyway, instead of in the update kernel).
//
// With one active column, units run tile after tile and dot products accumulate in registers
// until the end; with several, the columns of a tile run back to back (so the tile's operator
// rows are re-read from L2, not HBM) and each unit's products are folded into the per-warp
// sums of its column.
//
// Every mbarrier wait is bounded (about a second of SM clock).  When one expires the warp
// stops, the CTA records SYLV_E_TIMEOUT in Control::error, thread 0 waits (bounded) for the
// copies still in flight, and the CTA leaves without publishing partial sums.
#pragma once

#include "pcg_kernels.cuh"

namespace sylv {
namespace tma {

constexpr int NSTAGE = 2;   // stages of the staged kernels' rings (stand-alone apply: NST_X)
constexpr int NST_X = 3;
constexpr int MAXST = 3;
constexpr long long WAIT_BUDGET_CYCLES = 2000000000LL;

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)),
               "r"(bytes)
               : "memory");
}

// Global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(saddr(dst)), "l"(src), "r"(bytes), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase of the given parity, for at most `budget` SM clock cycles.  The waits of
// a pipeline (a stage to fill or to be released) take the kernel's budget (Control::
// wait_budget, shortened only to test the timeout path); the waits that drain copies already
// in flight before a CTA leaves keep the full default, so no copy outlives its CTA.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long budget = WAIT_BUDGET_CYCLES) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

// The pipeline wait budget of a kernel launched with this control word.
__device__ __forceinline__ long long pipe_budget(const Control* ctl) {
  const long long b = ctl->wait_budget;
  return b > 0 ? b : WAIT_BUDGET_CYCLES;
}

// Units of a CTA: its tiles (slot, slot + nslots, ...) times its active columns; unit u is
// tile u / nact and active column u % nact.
struct Units {
  int ntl;   // tiles of this CTA
  int nact;  // active columns
  int n;     // units = ntl * nact
};

__device__ __forceinline__ Units count_units(const SysDesc& sd, int slot, int nslots, int nact) {
  Units u;
  u.ntl = slot < sd.ntiles ? (sd.ntiles - slot + nslots - 1) / nslots : 0;
  u.nact = nact;
  u.n = u.ntl * nact;
  return u;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

constexpr int NCONS = TILE_PX / 32;     // consumer warps
constexpr int WS_THREADS = TILE_PX + 32;

// Shared state of a warp-specialised CTA.
struct PipeShared {
  uint64_t full[MAXST];
  uint64_t empty[MAXST];
  int cols[RMAX];
  int nact;
  int bad;
  int issued;
};

template <int NST = NSTAGE>
__device__ __forceinline__ void pipe_init(PipeShared& ps) {
  for (int s = 0; s < NST; ++s) {
    mbar_init(&ps.full[s], 1);
    mbar_init(&ps.empty[s], NCONS);
  }
  ps.bad = 0;
  ps.issued = 0;
  fence_mbar_init();
}

// Producer loop over units u0 .. u1 - 1: waits for stage release (from the second round of the
// ring on), then issues unit u with issue(u, stage).  NST: stages of the ring.
template <int NST = NSTAGE, typename Issue>
__device__ __forceinline__ void producer_loop_range(PipeShared& ps, int u0, int u1, Issue&& issue,
                                                    long long budget = WAIT_BUDGET_CYCLES) {
  const int lane = threadIdx.x & 31;
  for (int u = u0; u < u1; ++u) {
    const int st = u % NST;
    if (u >= NST) {
      bool ok = true;
      if (lane == 0) ok = mbar_wait_bounded(&ps.empty[st], ((u / NST) - 1) & 1, budget);
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

// After both roles are done: on a recorded timeout, flag it, wait (bounded) for the copies
// still in flight and report true (the caller leaves without partial sums).
template <int NST = NSTAGE>
__device__ __forceinline__ bool pipe_failed(PipeShared& ps, int consumed, Control* ctl) {
  __syncthreads();
  if (!ps.bad) return false;
  if (threadIdx.x == 0) {
    atomicOr(&ctl->error, 1u);
    for (int u = consumed; u < ps.issued; ++u)
      mbar_wait_bounded(&ps.full[u % NST], (u / NST) & 1);
  }
  __syncthreads();
  return true;
}

// ---- consumer-side sums (modes 1 and 2 of the staged kernels) -------------------------------
// In mode 0 the last CTA of a system to finish (atomic counter) sums the CTAs' partials and
// updates the column states.  In modes 1 and 2 no CTA waits for the others at its end: every
// CTA writes its partials, and every CTA of the NEXT kernel sums them itself at its start while
// its producer warp already fills the stage ring (mode 2), then applies the state change to its
// own copy of the column states.  All CTAs add in the same order, so the copies agree.  The
// states are double-buffered: operator kernels read ColState st (written by the update kernel,
// the residual kernel and the chunk-closing kernel) and their slot-0 CTA writes st2; update
// kernels read st2 and their slot-0 CTA writes st.  So no kernel reads a state it writes, and
// the counters of active and unfinished columns are kept by slot 0 alone.

// Columns a system may have for the consumer-side protocol (the host uses it up to this many;
// the copies live in shared memory next to the stage ring, which leaves little room).
constexpr int CS_RMAX = 2;

__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(TILE_PX) : "memory");
}

// tot[r][v] = sum over the system's slots of src[(slot R + r) NPART + v] for the columns with
// want[r], in a fixed order: thread t adds slots t, t + TILE_PX, ..., then FP64 warp trees and
// a tree over the warps.  Run by the TILE_PX consumer threads.
template <int NV>
__device__ __forceinline__ void sum_slots(const double* src, int nslots, int R, const int* want,
                                          double* red, double (*tot)[NPART]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = 0; r < R; ++r) {
    if (!want[r]) continue;
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    for (int sl = threadIdx.x; sl < nslots; sl += TILE_PX) {
      const double* p = src + ((size_t)sl * R + r) * NPART;
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += __ldcg(p + v);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double w = warp_sum(acc[v]);
      if (lane == 0) red[warp * NV + v] = w;
    }
    consumers_sync();
    if (warp == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double w = warp_sum(lane < NCONS ? red[lane * NV + v] : 0.0);
        if (lane == 0) tot[r][v] = w;
      }
    }
    consumers_sync();
  }
}

// Copies issued ahead for a column list that the state change altered: wait (bounded) until
// they landed, then start the ring afresh (thread 0; the caller synchronises).
__device__ __forceinline__ void pipe_restart(PipeShared& ps) {
  for (int u = 0; u < ps.issued; ++u) mbar_wait_bounded(&ps.full[u % NSTAGE], (u / NSTAGE) & 1);
  for (int q = 0; q < NSTAGE; ++q) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(saddr(&ps.full[q])) : "memory");
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(saddr(&ps.empty[q])) : "memory");
  }
  pipe_init(ps);
}

// Stage layouts.  Rows hold TILE_PX entries of 4 bytes (FP16 factor rows hold half2 pairs).
template <int K, int M, int E>
struct ApplyLayout {
  static constexpr int Z = 0, P = K, Q = 2 * K, D = 3 * K, VAL = 3 * K + M,
                       DIAG = 3 * K + M + E, COL = 3 * K + M + E + 1;
  static constexpr int ROWS = 3 * K + M + 2 * E + 1;
  static constexpr int STAGE_BYTES = ROWS * TILE_PX * 4;
};

template <int K, int M>
struct UpdateLayout {
  static constexpr int NB = K * (K + 1) / 2, NB2 = (NB + 1) / 2;
  static constexpr int R = 0, Q = K, S = 2 * K, L16 = 3 * K;
  static constexpr int ROWS = 3 * K + NB2;
  static constexpr int NOPREC_ROWS = 2 * K;
  static constexpr int STAGE_BYTES = ROWS * TILE_PX * 4;
};

// Operator value of one pixel from its staged data (Sec. 3.1): w_j = tau_j kappa_j^2 x_j +
// tau_j (L x_j) (lap holds L_ii x_j, the neighbours' values are nb with ELL weights v) +
// sum_c a_cj d_c (a_c . x); dcol: the pixel's noise weights in the stage (stride TILE_PX).
template <int K, int M, int E, int NV>
__device__ __forceinline__ void pixel_operator_ws(const CtaShared<float, NV>& sh, const float* dcol,
                                                  const float (&zi)[K], float (&lap)[K],
                                                  const float (&v)[E], const float (&nb)[E][K],
                                                  float (&w)[K]) {
  if constexpr (K % 2 == 0) {
    // the same arithmetic on pairs of sources with the packed FP32 FMA of sm_100+
    // (fma.rn.f32x2): the stencil, the prior diagonal and the block mapping
    constexpr int K2 = K / 2;
    float2 z2[K2], l2[K2], w2[K2];
#pragma unroll
    for (int q = 0; q < K2; ++q) {
      z2[q] = make_float2(zi[2 * q], zi[2 * q + 1]);
      l2[q] = make_float2(lap[2 * q], lap[2 * q + 1]);
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const float2 ve = make_float2(v[e], v[e]);
#pragma unroll
      for (int q = 0; q < K2; ++q)
        l2[q] = __ffma2_rn(ve, make_float2(nb[e][2 * q], nb[e][2 * q + 1]), l2[q]);
    }
#pragma unroll
    for (int q = 0; q < K2; ++q) {
      const float2 tk = make_float2(sh.tk2[2 * q], sh.tk2[2 * q + 1]);
      const float2 ta = make_float2(sh.tau[2 * q], sh.tau[2 * q + 1]);
      w2[q] = __ffma2_rn(tk, z2[q], __fmul2_rn(ta, l2[q]));
    }
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const float d = dcol[c * TILE_PX];
      const float2* arow = reinterpret_cast<const float2*>(sh.A[c]);
      float2 a2[K2];
#pragma unroll
      for (int q = 0; q < K2; ++q) a2[q] = arow[q];
      float2 acc = __fmul2_rn(a2[0], z2[0]);
#pragma unroll
      for (int q = 1; q < K2; ++q) acc = __ffma2_rn(a2[q], z2[q], acc);
      const float s = (acc.x + acc.y) * d;
      const float2 s2 = make_float2(s, s);
#pragma unroll
      for (int q = 0; q < K2; ++q) w2[q] = __ffma2_rn(a2[q], s2, w2[q]);
    }
#pragma unroll
    for (int q = 0; q < K2; ++q) {
      w[2 * q] = w2[q].x;
      w[2 * q + 1] = w2[q].y;
    }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int j = 0; j < K; ++j) lap[j] += v[e] * nb[e][j];
#pragma unroll
    for (int j = 0; j < K; ++j) w[j] = sh.tk2[j] * zi[j] + sh.tau[j] * lap[j];
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const float d = dcol[c * TILE_PX];
      float a[K];
      load_row<K, float>(sh.A[c], a);
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < K; ++j) s += a[j] * zi[j];
      s *= d;
#pragma unroll
      for (int j = 0; j < K; ++j) w[j] += a[j] * s;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// inner_apply (staged): d += alpha p (the previous iteration's step), p = z + beta p,
// q = G z + beta q, partial p . q
// ---------------------------------------------------------------------------------------------
// mode 0: the last CTA sets alpha (last-CTA protocol); mode 1: column states as stored in st;
// mode 2: first the state change of the previous update kernel, from its partials.
template <int K, int M, int E>
__global__ void __launch_bounds__(WS_THREADS, 3)
k_inner_apply_tma(const SysDesc* __restrict__ descs, const CtaRef* __restrict__ ctas,
                  Control* ctl, int mode) {
  using L = ApplyLayout<K, M, E>;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ CtaShared<float, 1> sh;
  __shared__ __align__(8) PipeShared ps;
  __shared__ ColState cst[CS_RMAX];
  __shared__ double tot2[CS_RMAX][NPART];
  const CtaRef cr = ctas[blockIdx.x];
  if (cr.sys < 0) return;  // idle CTA of a reassigned launch
  const SysDesc& sd = descs[cr.sys];
  const OpData& op = sd.op;
  const int R = sd.R;
  const bool newp = mode != 0 && R <= CS_RMAX;
  int act = 0;
  if (threadIdx.x < RMAX) {
    const int r = threadIdx.x;
    if (r < R) {
      const ColState& cs = sd.st[r];
      if (newp) cst[r] = cs;
      act = cs.phase == PH_INNER;
      sh.sc[r] = float(cs.beta);
      sh.sc2[r] = float(cs.alpha);   // (the update kernels' state change keeps alpha)
      sh.aux[r] = cs.first;
    }
    sh.act[r] = act;
  }
  stage_operator<float, 1>(op, K, sh);
  zero_wacc<float, 1>(sh, R);
  if (threadIdx.x == 0) {
    int na = 0;
    for (int r = 0; r < R; ++r)
      if (sh.act[r]) ps.cols[na++] = r;
    ps.nact = na;
    pipe_init(ps);
  }
  if (!__syncthreads_or(act)) {
    if (newp && cr.slot == 0 && threadIdx.x < R) sd.st2[threadIdx.x] = cst[threadIdx.x];
    return;
  }

  const int64_t ld = op.ld, n = op.n;
  Units U = count_units(sd, cr.slot, sd.nslots[0], ps.nact);
  const float* zg = (const float*)sd.vz;
  float* pg = (float*)sd.vp;
  float* qg = (float*)sd.vq;
  float* dgl = (float*)sd.vd;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int consumed = 0;
  auto issue = [&](int u, int st) {
    const int tile = cr.slot + (u / U.nact) * sd.nslots[0];
    const int r = ps.cols[u % U.nact];
    const bool first = sh.aux[r] != 0;
    const int64_t base = (int64_t)tile * TILE_PX;
    float* stage = reinterpret_cast<float*>(dsm + (size_t)st * L::STAGE_BYTES);
    const uint32_t rowb = TILE_PX * 4;
    const int nrows = first ? L::ROWS - 2 * K : L::ROWS;
    if (lane == 0) {
      fence_proxy_async();
      mbar_expect_tx(&ps.full[st], (uint32_t)nrows * rowb);
    }
    __syncwarp();
    const size_t voff = (size_t)r * K * ld;
    for (int q = lane; q < L::ROWS; q += 32) {
      const void* src = nullptr;
      if (q < K) src = zg + voff + (size_t)q * ld + base;
      else if (q < 2 * K) src = first ? nullptr : pg + voff + (size_t)(q - K) * ld + base;
      else if (q < 3 * K) src = first ? nullptr : qg + voff + (size_t)(q - 2 * K) * ld + base;
      else if (q < L::VAL) src = op.D32 + (size_t)(q - L::D) * ld + base;
      else if (q < L::DIAG) src = op.ell_val32 + (size_t)(q - L::VAL) * ld + base;
      else if (q == L::DIAG) src = op.diag32 + base;
      else src = op.ell_col + (size_t)(q - L::COL) * ld + base;
      if (src) bulk_load(stage + (size_t)q * TILE_PX, src, rowb, &ps.full[st]);
    }
    // the unit's d rows, which the consumers load directly: into L2 ahead of them
    if (!first && lane < K) bulk_prefetch_l2(dgl + voff + (size_t)lane * ld + base, rowb);
  };
  int head = 0;
  if (newp) {
    // the first ring of copies goes out for the columns active as stored; meanwhile the
    // consumers apply the previous update's state change (which keeps p, q and first as they are)
    head = U.n < NSTAGE ? U.n : NSTAGE;
    if (warp == NCONS) {
      if (!(ctl->inject_stall & STALL_APPLY))
        producer_loop_range(ps, 0, head, issue, pipe_budget(ctl));
    } else if (mode == 2) {
      sum_slots<2>(sd.partial2, sd.nslots[1], R, sh.act, sh.red, tot2);
      if (threadIdx.x < R && sh.act[threadIdx.x]) {
        const int r = threadIdx.x;
        after_update(cst[r], tot2[r][0], tot2[r][1], ctl, cr.slot == 0);
      }
    }
    __syncthreads();
    if (cr.slot == 0 && threadIdx.x < R) sd.st2[threadIdx.x] = cst[threadIdx.x];
    if (threadIdx.x == 0) {
      int na = 0;
      bool same = true;
      for (int r = 0; r < R; ++r) {
        const int a2 = cst[r].phase == PH_INNER;
        if (a2 != sh.act[r]) same = false;
        sh.act[r] = a2;
        sh.sc[r] = float(cst[r].beta);
        if (a2) ps.cols[na++] = r;
      }
      if (!same) {   // a column ended: restart the ring for the columns still running
        pipe_restart(ps);
        ps.nact = na;
        sh.flag = 1;
      } else {
        sh.flag = 0;
      }
    }
    __syncthreads();
    if (sh.flag) {
      if (ps.nact == 0) return;
      U = count_units(sd, cr.slot, sd.nslots[0], ps.nact);
      head = 0;
    }
  }

  if (warp == NCONS) {
    if (!(ctl->inject_stall & STALL_APPLY))
      producer_loop_range(ps, head, U.n, issue, pipe_budget(ctl));
  } else {
    const int t = threadIdx.x;
    float acc = 0.f;   // this thread's p . q over its units of one column (FP32)
    for (int u = 0; u < U.n; ++u) {
      const int st = u % NSTAGE;
      if (!mbar_wait_bounded(&ps.full[st], (u / NSTAGE) & 1, pipe_budget(ctl)) || ps.bad) {
        ps.bad = 1;
        break;
      }
      const int tile = cr.slot + (u / U.nact) * sd.nslots[0];
      const int r = ps.cols[u % U.nact];
      const int64_t base = (int64_t)tile * TILE_PX;
      const int64_t i = base + t;
      const float* stage = reinterpret_cast<const float*>(dsm + (size_t)st * L::STAGE_BYTES);
      const int32_t* scol = reinterpret_cast<const int32_t*>(stage + (size_t)L::COL * TILE_PX);
      const size_t voff = (size_t)r * K * ld;
      const bool first = sh.aux[r] != 0;
      float zi[K], lap[K];
#pragma unroll
      for (int j = 0; j < K; ++j) zi[j] = stage[(L::Z + j) * TILE_PX + t];
      const float dg = stage[L::DIAG * TILE_PX + t];
#pragma unroll
      for (int j = 0; j < K; ++j) lap[j] = dg * zi[j];
      // neighbour values: from the staged tile when the neighbour is in it, else from global
      // memory; generic pointers keep the loads branch-free so all E*K of them issue at once
      const float* src[E];
      int64_t stride[E];
      float v[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int64_t c = scol[e * TILE_PX + t];
        v[e] = stage[(L::VAL + e) * TILE_PX + t];
        const uint32_t loc = (uint32_t)(c - base);
        const bool in_tile = loc < (uint32_t)TILE_PX;
        src[e] = in_tile ? stage + (size_t)L::Z * TILE_PX + loc : zg + voff + c;
        stride[e] = in_tile ? (int64_t)TILE_PX : ld;
      }
      float nb[E][K];
#pragma unroll
      for (int e = 0; e < E; ++e)
#pragma unroll
        for (int j = 0; j < K; ++j) nb[e][j] = src[e][j * stride[e]];
      float w[K];
      pixel_operator_ws<K, M, E>(sh, stage + (size_t)L::D * TILE_PX + t, zi, lap, v, nb, w);
      const float beta = sh.sc[r], alpha = sh.sc2[r];
      float pq = 0.f;
      if (i < n) {
        float dv[K];   // the pixel's d, all loads in flight before the first use
#pragma unroll
        for (int j = 0; j < K; ++j) dv[j] = first ? 0.f : dgl[voff + (size_t)j * ld + i];
#pragma unroll
        for (int j = 0; j < K; ++j) {
          float pj = zi[j], qj = w[j];
          if (!first) {
            const float po = stage[(L::P + j) * TILE_PX + t];
            dgl[voff + (size_t)j * ld + i] = dv[j] + alpha * po;
            pj += beta * po;
            qj += beta * stage[(L::Q + j) * TILE_PX + t];
          }
          pg[voff + (size_t)j * ld + i] = pj;
          qg[voff + (size_t)j * ld + i] = qj;
          pq += pj * qj;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&ps.empty[st]);
      consumed = u + 1;
      acc += pq;
      if (U.nact > 1 || u + 1 == U.n) {
        const float v1[1] = {acc};
        warp_accumulate_f32<float, 1>(sh, r, v1);
        acc = 0.f;
      }
    }
  }
  if (pipe_failed(ps, consumed, ctl)) return;
  if (newp) {
    write_cta_partials<float, 1>(sd.partial, cr.slot, sh, R);
    return;
  }
  double tot[RMAX][1];
  if (!finish_partials<float, 1>(sd, cr.slot, sd.nslots[0], sh, R, tot)) return;
  if (threadIdx.x == 0) {
    for (int r = 0; r < R; ++r)
      if (sh.act[r]) after_apply(sd.st[r], tot[r][0], ctl, true);
    *sd.counter = 0u;
  }
}

// ---------------------------------------------------------------------------------------------
// inner_update (staged): r -= alpha q, z = P^{-1} r, partial r . z and r . r (d += alpha p is
// the next operator kernel's)
// ---------------------------------------------------------------------------------------------
// mode 0: the last CTA sets beta, gamma and the stopping state (last-CTA protocol); mode 1:
// column states as stored in st2 (alpha included); mode 2: first alpha (the operator kernel's
// state change) from its partials.
template <int K, int M>
__global__ void __launch_bounds__(WS_THREADS, 2)
k_inner_update_tma(const SysDesc* __restrict__ descs, const CtaRef* __restrict__ ctas,
                   Control* ctl, int mode) {
  using L = UpdateLayout<K, M>;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ CtaShared<float, 2> sh;  // (mixing rows unused here: the factor is stored)
  __shared__ __align__(8) PipeShared ps;
  __shared__ ColState cst[CS_RMAX];
  __shared__ double tot1[CS_RMAX][NPART];
  const CtaRef cr = ctas[blockIdx.x];
  if (cr.sys < 0) return;  // idle CTA of a reassigned launch
  const SysDesc& sd = descs[cr.sys];
  const OpData& op = sd.op;
  const int R = sd.R;
  const bool newp = mode != 0 && R <= CS_RMAX;
  int act = 0;
  if (threadIdx.x < RMAX) {
    const int r = threadIdx.x;
    if (r < R) {
      const ColState& cs = newp ? sd.st2[r] : sd.st[r];
      if (newp) cst[r] = cs;
      act = cs.phase == PH_INNER;
      sh.sc[r] = float(cs.alpha);
    }
    sh.act[r] = act;
  }
  zero_wacc<float, 2>(sh, R);
  if (threadIdx.x == 0) {
    int na = 0;
    for (int r = 0; r < R; ++r)
      if (sh.act[r]) ps.cols[na++] = r;
    ps.nact = na;
    pipe_init(ps);
  }
  if (!__syncthreads_or(act)) {
    if (newp && cr.slot == 0 && threadIdx.x < R) sd.st[threadIdx.x] = cst[threadIdx.x];
    return;
  }

  const int64_t ld = op.ld, n = op.n;
  const bool prec = ctl->precond == SYLV_PRECOND_BLOCK_JACOBI;
  Units U = count_units(sd, cr.slot, sd.nslots[1], ps.nact);
  float* rg = (float*)sd.vr;
  float* zg = (float*)sd.vz;
  const float* qg = (const float*)sd.vq;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int consumed = 0;
  auto issue = [&](int u, int st) {
    const int tile = cr.slot + (u / U.nact) * sd.nslots[1];
    const int r = ps.cols[u % U.nact];
    const int64_t base = (int64_t)tile * TILE_PX;
    float* stage = reinterpret_cast<float*>(dsm + (size_t)st * L::STAGE_BYTES);
    const uint32_t rowb = TILE_PX * 4;
    const int nrows = prec ? L::ROWS : L::NOPREC_ROWS;
    if (lane == 0) {
      fence_proxy_async();
      mbar_expect_tx(&ps.full[st], (uint32_t)nrows * rowb);
    }
    __syncwarp();
    const size_t voff = (size_t)r * K * ld;
    for (int q = lane; q < nrows; q += 32) {
      const void* src;
      if (q < L::Q) src = rg + voff + (size_t)(q - L::R) * ld + base;
      else if (q < L::S) src = qg + voff + (size_t)(q - L::Q) * ld + base;
      else if (q < L::L16) src = op.fs32 + (size_t)(q - L::S) * ld + base;
      else src = op.fl16 + (size_t)(q - L::L16) * ld + base;
      bulk_load(stage + (size_t)q * TILE_PX, src, rowb, &ps.full[st]);
    }
  };
  int head = 0;
  if (newp) {
    // the first ring of copies goes out for the columns active as stored; meanwhile the
    // consumers form alpha from the operator kernel's partial sums
    head = U.n < NSTAGE ? U.n : NSTAGE;
    if (warp == NCONS) {
      if (!(ctl->inject_stall & STALL_UPDATE))
        producer_loop_range(ps, 0, head, issue, pipe_budget(ctl));
    } else if (mode == 2) {
      sum_slots<1>(sd.partial, sd.nslots[0], R, sh.act, sh.red, tot1);
      if (threadIdx.x < R && sh.act[threadIdx.x]) {
        const int r = threadIdx.x;
        after_apply(cst[r], tot1[r][0], ctl, cr.slot == 0);
      }
    }
    __syncthreads();
    if (cr.slot == 0 && threadIdx.x < R) sd.st[threadIdx.x] = cst[threadIdx.x];
    if (threadIdx.x == 0) {
      int na = 0;
      bool same = true;
      for (int r = 0; r < R; ++r) {
        const int a2 = cst[r].phase == PH_INNER;
        if (a2 != sh.act[r]) same = false;
        sh.act[r] = a2;
        sh.sc[r] = float(cst[r].alpha);
        if (a2) ps.cols[na++] = r;
      }
      if (!same) {   // a column ended: restart the ring for the columns still running
        pipe_restart(ps);
        ps.nact = na;
        sh.flag = 1;
      } else {
        sh.flag = 0;
      }
    }
    __syncthreads();
    if (sh.flag) {
      if (ps.nact == 0) return;
      U = count_units(sd, cr.slot, sd.nslots[1], ps.nact);
      head = 0;
    }
  }

  if (warp == NCONS) {
    if (!(ctl->inject_stall & STALL_UPDATE))
      producer_loop_range(ps, head, U.n, issue, pipe_budget(ctl));
  } else {
    const int t = threadIdx.x;
    float acc_rz = 0.f, acc_rr = 0.f;   // over this thread's units of one column (FP32)
    for (int u = 0; u < U.n; ++u) {
      const int st = u % NSTAGE;
      if (!mbar_wait_bounded(&ps.full[st], (u / NSTAGE) & 1, pipe_budget(ctl)) || ps.bad) {
        ps.bad = 1;
        break;
      }
      const int tile = cr.slot + (u / U.nact) * sd.nslots[1];
      const int r = ps.cols[u % U.nact];
      const int64_t i = (int64_t)tile * TILE_PX + t;
      const float* stage = reinterpret_cast<const float*>(dsm + (size_t)st * L::STAGE_BYTES);
      const float alpha = sh.sc[r];
      const size_t voff = (size_t)r * K * ld;
      float ri[K], zi[K];
#pragma unroll
      for (int j = 0; j < K; ++j)
        ri[j] = stage[(L::R + j) * TILE_PX + t] - alpha * stage[(L::Q + j) * TILE_PX + t];
      if (prec) {
        BlockChol<K, float> f;
        const __half2* sl = reinterpret_cast<const __half2*>(stage + (size_t)L::L16 * TILE_PX);
#pragma unroll
        for (int x = 0; x < K; ++x) f.s[x] = stage[(L::S + x) * TILE_PX + t];
#pragma unroll
        for (int x = 0; x < L::NB; x += 2) {
          const float2 v = __half22float2(sl[(x / 2) * TILE_PX + t]);
          f.l[x] = v.x;
          if (x + 1 < L::NB) f.l[x + 1] = v.y;
        }
        block_solve<K, float>(f, ri, zi);
      } else {
#pragma unroll
        for (int j = 0; j < K; ++j) zi[j] = ri[j];
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&ps.empty[st]);   // stage fully read
      consumed = u + 1;
      float rz = 0.f, rr = 0.f;
      if (i < n) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
          rg[voff + (size_t)j * ld + i] = ri[j];
          zg[voff + (size_t)j * ld + i] = zi[j];
          rz += ri[j] * zi[j];
          rr += ri[j] * ri[j];
        }
      }
      acc_rz += rz;
      acc_rr += rr;
      if (U.nact > 1 || u + 1 == U.n) {
        const float v2[2] = {acc_rz, acc_rr};
        warp_accumulate_f32<float, 2>(sh, r, v2);
        acc_rz = acc_rr = 0.f;
      }
    }
  }
  if (pipe_failed(ps, consumed, ctl)) return;
  if (newp) {
    write_cta_partials<float, 2>(sd.partial2, cr.slot, sh, R);
    return;
  }
  double tot[RMAX][2];
  if (!finish_partials<float, 2>(sd, cr.slot, sd.nslots[1], sh, R, tot)) return;
  if (threadIdx.x == 0) {
    for (int r = 0; r < R; ++r)
      if (sh.act[r]) after_update(sd.st[r], tot[r][0], tot[r][1], ctl, true);
    *sd.counter = 0u;
  }
}

// ---------------------------------------------------------------------------------------------
// residual (staged, mixed precision): r64 = B - G X in FP64, r = r64 rounded to FP32, d = 0,
// z = P^{-1} r; partial ||r64||^2, ||B||^2, r . z, r . r; the last CTA decides (after_residual)
// ---------------------------------------------------------------------------------------------
// The FP64 operator is the pixel-block form (k(k+1) FMAs per pixel for the block plus the
// stencil), which keeps this kernel on the FP64 pipe (1/64 of the FP32 rate on GB300): staging
// every stream it reads lets the consumer warps wait only on that pipe.  Stage: X and B of the
// tile (the caller's FP64 rows), the FP64 pixel block, the FP64 ELL values, the ELL columns,
// and the FP32 scaling and FP16 factor of the preconditioner.  Used when the caller's rows can
// be copied whole (n a multiple of TILE_PX, even ldu, 16-byte aligned X and B).
template <int K, int E>
struct ResidLayout {
  static constexpr int NB = K * (K + 1) / 2, NB2 = (NB + 1) / 2;
  // byte offsets of the regions; rows hold TILE_PX entries
  static constexpr int X = 0;                          // K rows, FP64
  static constexpr int B = X + K * TILE_PX * 8;        // K rows, FP64
  static constexpr int BLK = B + K * TILE_PX * 8;      // NB rows, FP64
  static constexpr int VAL = BLK + NB * TILE_PX * 8;   // E rows, FP64
  static constexpr int COL = VAL + E * TILE_PX * 8;    // E rows, int32
  static constexpr int FS = COL + E * TILE_PX * 4;     // K rows, FP32
  static constexpr int FL = FS + K * TILE_PX * 4;      // NB2 rows, half2
  static constexpr int STAGE_BYTES = FL + NB2 * TILE_PX * 4;
};

template <int K, int M, int E>
__global__ void __launch_bounds__(WS_THREADS, 1)
k_residual_tma(const SysDesc* __restrict__ descs, const CtaRef* __restrict__ ctas,
               Control* ctl) {
  using L = ResidLayout<K, E>;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ CtaShared<double, 4> sh;
  __shared__ __align__(8) PipeShared ps;
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
  if (threadIdx.x == 0) {
    int na = 0;
    for (int r = 0; r < R; ++r)
      if (sh.act[r]) ps.cols[na++] = r;
    ps.nact = na;
    pipe_init(ps);
  }
  if (!__syncthreads_or(act)) return;

  const int64_t ld = op.ld, ldu = op.ldu, n = op.n;
  const bool prec = ctl->precond == SYLV_PRECOND_BLOCK_JACOBI;
  const bool x0_zero = ctl->x0_zero != 0;
  const Units U = count_units(sd, cr.slot, sd.nslots[3], ps.nact);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int consumed = 0;

  if (warp == NCONS) {
    producer_loop_range(ps, 0, (ctl->inject_stall & STALL_RESIDUAL) ? 0 : U.n, [&](int u, int st) {
      const int tile = cr.slot + (u / U.nact) * sd.nslots[3];
      const int r = ps.cols[u % U.nact];
      const bool noop = x0_zero && sh.aux[r] == PH_START;   // X = 0: no operator term
      const int64_t base = (int64_t)tile * TILE_PX;
      unsigned char* stage = dsm + (size_t)st * L::STAGE_BYTES;
      const uint32_t row8 = TILE_PX * 8, row4 = TILE_PX * 4;
      const uint32_t bytes = K * row8 + (noop ? 0u : K * row8 + L::NB * row8 + E * (row8 + row4)) +
                             (prec ? K * row4 + L::NB2 * row4 : 0u);
      if (lane == 0) {
        fence_proxy_async();
        mbar_expect_tx(&ps.full[st], bytes);
      }
      __syncwarp();
      const size_t uoff = (size_t)r * K * ldu;
      constexpr int NROWS = 2 * K + L::NB + 2 * E + K + L::NB2;
      for (int q = lane; q < NROWS; q += 32) {
        const void* src = nullptr;
        void* dst = nullptr;
        uint32_t nb = row8;
        int x = q;
        if (x < K) {
          src = sd.B + uoff + (size_t)x * ldu + base;
          dst = stage + L::B + (size_t)x * row8;
        } else if ((x -= K) < K) {
          if (!noop) src = sd.X + uoff + (size_t)x * ldu + base;
          dst = stage + L::X + (size_t)x * row8;
        } else if ((x -= K) < L::NB) {
          if (!noop) src = op.blk64 + (size_t)x * ld + base;
          dst = stage + L::BLK + (size_t)x * row8;
        } else if ((x -= L::NB) < E) {
          if (!noop) src = op.ell_val64 + (size_t)x * ld + base;
          dst = stage + L::VAL + (size_t)x * row8;
        } else if ((x -= E) < E) {
          if (!noop) src = op.ell_col + (size_t)x * ld + base;
          dst = stage + L::COL + (size_t)x * row4;
          nb = row4;
        } else if ((x -= E) < K) {
          if (prec) src = op.fs32 + (size_t)x * ld + base;
          dst = stage + L::FS + (size_t)x * row4;
          nb = row4;
        } else {
          x -= K;
          if (prec) src = op.fl16 + (size_t)x * ld + base;
          dst = stage + L::FL + (size_t)x * row4;
          nb = row4;
        }
        if (src) bulk_load(dst, src, nb, &ps.full[st]);
      }
    }, pipe_budget(ctl));
  } else {
    const int t = threadIdx.x;
    double a_rr64 = 0.0, a_bb = 0.0, a_rz = 0.0, a_rr = 0.0;
    for (int u = 0; u < U.n; ++u) {
      const int st = u % NSTAGE;
      if (!mbar_wait_bounded(&ps.full[st], (u / NSTAGE) & 1, pipe_budget(ctl)) || ps.bad) {
        ps.bad = 1;
        break;
      }
      const int tile = cr.slot + (u / U.nact) * sd.nslots[3];
      const int r = ps.cols[u % U.nact];
      const bool noop = x0_zero && sh.aux[r] == PH_START;
      const int64_t base = (int64_t)tile * TILE_PX;
      const int64_t i = base + t;
      const unsigned char* stage = dsm + (size_t)st * L::STAGE_BYTES;
      const double* sx = reinterpret_cast<const double*>(stage + L::X);
      const double* sb = reinterpret_cast<const double*>(stage + L::B);
      const double* sblk = reinterpret_cast<const double*>(stage + L::BLK);
      const double* sval = reinterpret_cast<const double*>(stage + L::VAL);
      const int32_t* scol = reinterpret_cast<const int32_t*>(stage + L::COL);
      const size_t uoff = (size_t)r * K * ldu, off = (size_t)r * K * ld;
      double gx[K];
#pragma unroll
      for (int j = 0; j < K; ++j) gx[j] = 0.0;
      if (!noop) {
        double xi[K];
#pragma unroll
        for (int j = 0; j < K; ++j) xi[j] = sx[j * TILE_PX + t];
        // neighbours of the stencil: staged when in the tile, else the caller's X
        const double* src[E];
        int64_t stride[E];
        double v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int64_t c = scol[e * TILE_PX + t];
          v[e] = sval[e * TILE_PX + t];
          const uint32_t loc = (uint32_t)(c - base);
          const bool in_tile = loc < (uint32_t)TILE_PX;
          src[e] = in_tile ? sx + loc : sd.X + uoff + c;
          stride[e] = in_tile ? (int64_t)TILE_PX : ldu;
        }
        double nb[E][K];
#pragma unroll
        for (int e = 0; e < E; ++e)
#pragma unroll
          for (int j = 0; j < K; ++j) nb[e][j] = src[e][j * stride[e]];
        // pixel block (packed lower triangle, row-major)
#pragma unroll
        for (int a = 0; a < K; ++a) {
#pragma unroll
          for (int b = 0; b <= a; ++b) {
            const double pab = sblk[(a * (a + 1) / 2 + b) * TILE_PX + t];
            gx[a] += pab * xi[b];
            if (b != a) gx[b] += pab * xi[a];
          }
        }
        double lap[K];
#pragma unroll
        for (int j = 0; j < K; ++j) lap[j] = 0.0;
#pragma unroll
        for (int e = 0; e < E; ++e)
#pragma unroll
          for (int j = 0; j < K; ++j) lap[j] += v[e] * nb[e][j];
#pragma unroll
        for (int j = 0; j < K; ++j) gx[j] += sh.tau[j] * lap[j];
      }
      float ri[K], zi[K];
      double rr64 = 0.0, bb = 0.0;
      const bool start = sh.aux[r] == PH_START;   // ||B||^2 is used by the first residual only
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const double bj = sb[j * TILE_PX + t];
        const double r64 = bj - gx[j];
        rr64 += r64 * r64;
        if (start) bb += bj * bj;
        ri[j] = float(r64);
      }
      if (prec) {
        BlockChol<K, float> f;
        const float* sfs = reinterpret_cast<const float*>(stage + L::FS);
        const __half2* sfl = reinterpret_cast<const __half2*>(stage + L::FL);
#pragma unroll
        for (int x = 0; x < K; ++x) f.s[x] = sfs[x * TILE_PX + t];
#pragma unroll
        for (int x = 0; x < L::NB; x += 2) {
          const float2 w2 = __half22float2(sfl[(x / 2) * TILE_PX + t]);
          f.l[x] = w2.x;
          if (x + 1 < L::NB) f.l[x + 1] = w2.y;
        }
        block_solve<K, float>(f, ri, zi);
      } else {
#pragma unroll
        for (int j = 0; j < K; ++j) zi[j] = ri[j];
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&ps.empty[st]);
      consumed = u + 1;
      float rzt = 0.f, rrt = 0.f;   // products in the inner type, like the inner kernels
      if (i < n) {
        float* rv = (float*)sd.vr + off;
        float* dv = (float*)sd.vd + off;
        float* zv = (float*)sd.vz + off;
#pragma unroll
        for (int j = 0; j < K; ++j) {
          rv[(size_t)j * ld + i] = ri[j];
          dv[(size_t)j * ld + i] = 0.f;
          zv[(size_t)j * ld + i] = zi[j];
          rzt += ri[j] * zi[j];
          rrt += ri[j] * ri[j];
        }
      } else {
        rr64 = bb = 0.0;
      }
      a_rr64 += rr64;
      a_bb += bb;
      a_rz += double(rzt);
      a_rr += double(rrt);
      if (U.nact > 1 || u + 1 == U.n) {
        const double v4[4] = {a_rr64, a_bb, a_rz, a_rr};
        warp_accumulate<double, 4>(sh, r, v4);
        a_rr64 = a_bb = a_rz = a_rr = 0.0;
      }
    }
  }
  if (pipe_failed(ps, consumed, ctl)) return;
  double tot[RMAX][4];
  if (!finish_partials<double, 4>(sd, cr.slot, sd.nslots[3], sh, R, tot)) return;
  if (threadIdx.x == 0) {
    for (int r = 0; r < R; ++r)
      if (sh.act[r]) after_residual(sd.st[r], tot[r], ctl);
    *sd.counter = 0u;
  }
}

// ---------------------------------------------------------------------------------------------
// stand-alone operator apply (staged): Y = G X for FP32 caller vectors (nrhs columns)
// ---------------------------------------------------------------------------------------------
// Stage: x of the tile (K rows), D, ELL values, diagonal, ELL columns.  Used when n is a
// multiple of TILE_PX and every caller row starts 16-byte aligned (whole-tile copies then stay
// inside the caller's rows).  Units run tile-major, so with several right-hand sides the
// tile's operator rows come from L2 after the first.
template <int K, int M, int E>
struct ApplyXLayout {
  static constexpr int X = 0, D = K, VAL = K + M, DIAG = K + M + E, COL = K + M + E + 1;
  static constexpr int ROWS = K + M + 2 * E + 1;
  static constexpr int STAGE_BYTES = ROWS * TILE_PX * 4;
};

template <int K, int M, int E>
__global__ void __launch_bounds__(WS_THREADS, 3)
k_apply_tma(OpData op, const float* __restrict__ X, float* __restrict__ Y, int R,
            unsigned int* ctr) {
  // ctr[0]: timeout flag; ctr[1]: next tile; ctr[2]: CTAs done (both zero between launches).
  // Tiles are taken from ctr[1] one ahead, so CTAs on faster SMs take more of them; there are
  // no partial sums here, so how the tiles are split changes nothing in the result.  A tile
  // index >= ntiles stops the consumers.  A tile's columns run back to back.
  using L = ApplyXLayout<K, M, E>;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ CtaShared<float, 1> sh;
  __shared__ __align__(8) PipeShared ps;
  __shared__ int utile[NST_X], ucol[NST_X];
  stage_operator<float, 1>(op, K, sh);
  if (threadIdx.x == 0) pipe_init<NST_X>(ps);
  __syncthreads();
  const int64_t ldu = op.ldu;
  const int ntiles = (int)(op.n / TILE_PX);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int consumed = 0;
  if (warp == NCONS) {
    int next = 0, u = 0;
    if (lane == 0) next = (int)atomicAdd(ctr + 1, 1u);
    bool stop = false;
    while (!stop) {
      const int tile = __shfl_sync(0xffffffffu, next, 0);
      const bool end = tile >= ntiles;
      if (!end && lane == 0) next = (int)atomicAdd(ctr + 1, 1u);
      const int nu = end ? 1 : R;
      for (int r = 0; r < nu; ++r, ++u) {
        const int st = u % NST_X;
        if (u >= NST_X) {
          bool ok = true;
          if (lane == 0) ok = mbar_wait_bounded(&ps.empty[st], ((u / NST_X) - 1) & 1);
          ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
          if (!ok || ps.bad) {
            if (lane == 0) ps.bad = 1;
            stop = true;
            break;
          }
        }
        if (lane == 0) {
          utile[st] = end ? -1 : tile;
          ucol[st] = r;
        }
        __syncwarp();
        if (end) {
          if (lane == 0) mbar_arrive(&ps.full[st]);
        } else {
          const int64_t base = (int64_t)tile * TILE_PX;
          float* stage = reinterpret_cast<float*>(dsm + (size_t)st * L::STAGE_BYTES);
          const uint32_t rowb = TILE_PX * 4;
          if (lane == 0) {
            fence_proxy_async();
            mbar_expect_tx(&ps.full[st], (uint32_t)L::ROWS * rowb);
          }
          __syncwarp();
          const size_t xoff = (size_t)r * K * ldu;
          for (int q = lane; q < L::ROWS; q += 32) {
            const void* src;
            if (q < K) src = X + xoff + (size_t)q * ldu + base;
            else if (q < L::VAL) src = op.D32 + (size_t)(q - L::D) * op.ld + base;
            else if (q < L::DIAG) src = op.ell_val32 + (size_t)(q - L::VAL) * op.ld + base;
            else if (q == L::DIAG) src = op.diag32 + base;
            else src = op.ell_col + (size_t)(q - L::COL) * op.ld + base;
            bulk_load(stage + (size_t)q * TILE_PX, src, rowb, &ps.full[st]);
          }
        }
        if (lane == 0) ps.issued = u + 1;
      }
      if (end) stop = true;
    }
  } else {
    const int t = threadIdx.x;
    for (int u = 0;; ++u) {
      const int st = u % NST_X;
      if (!mbar_wait_bounded(&ps.full[st], (u / NST_X) & 1) || ps.bad) {
        ps.bad = 1;
        break;
      }
      const int tile = utile[st];
      if (tile < 0) {
        consumed = u + 1;
        break;
      }
      const int r = ucol[st];
      const int64_t base = (int64_t)tile * TILE_PX;
      const int64_t i = base + t;
      const float* stage = reinterpret_cast<const float*>(dsm + (size_t)st * L::STAGE_BYTES);
      const int32_t* scol = reinterpret_cast<const int32_t*>(stage + (size_t)L::COL * TILE_PX);
      const size_t xoff = (size_t)r * K * ldu;
      float xi[K], lap[K];
#pragma unroll
      for (int j = 0; j < K; ++j) xi[j] = stage[(L::X + j) * TILE_PX + t];
      const float dg = stage[L::DIAG * TILE_PX + t];
#pragma unroll
      for (int j = 0; j < K; ++j) lap[j] = dg * xi[j];
      const float* src[E];
      int64_t stride[E];
      float v[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int64_t c = scol[e * TILE_PX + t];
        v[e] = stage[(L::VAL + e) * TILE_PX + t];
        const uint32_t loc = (uint32_t)(c - base);
        const bool in_tile = loc < (uint32_t)TILE_PX;
        src[e] = in_tile ? stage + (size_t)L::X * TILE_PX + loc : X + xoff + c;
        stride[e] = in_tile ? (int64_t)TILE_PX : ldu;
      }
      float nb[E][K];
#pragma unroll
      for (int e = 0; e < E; ++e)
#pragma unroll
        for (int j = 0; j < K; ++j) nb[e][j] = src[e][j * stride[e]];
      float w[K];
      pixel_operator_ws<K, M, E>(sh, stage + (size_t)L::D * TILE_PX + t, xi, lap, v, nb, w);
      __syncwarp();
      if (lane == 0) mbar_arrive(&ps.empty[st]);
      consumed = u + 1;
#pragma unroll
      for (int j = 0; j < K; ++j) Y[xoff + (size_t)j * ldu + i] = w[j];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (ps.bad) {
      atomicOr(ctr, 1u);
      for (int u = consumed; u < ps.issued; ++u)
        mbar_wait_bounded(&ps.full[u % NST_X], (u / NST_X) & 1);
    }
    // every CTA's producer has finished taking tiles when its CTA gets here; the last CTA
    // resets the counters for the next launch
    __threadfence();
    if (atomicAdd(ctr + 2, 1u) == gridDim.x - 1u) {
      ctr[1] = 0u;
      ctr[2] = 0u;
      __threadfence();
    }
  }
}

}  // namespace tma
}  // namespace sylv
