// Multi-column staged FP32 kernels: several right-hand sides ("columns") of one system share
// every read of the tile's operator data.
//
// The operator of Sec. 3.1 (the block mapping of eq. block-vector-mapping-matvec with the
// neighbour stencil of Algorithm 1) and the pixel-block preconditioner are the same for every
// right-hand side; only the vectors differ.  These kernels stage a tile's operator rows (the
// noise maps D, the ELL rows of L and its diagonal; or the preconditioner's scaling and factor)
// ONCE, into an operator slot, and each (tile, column) unit's vector rows into a separate ring
// of vector stages.  A consumer thread (one pixel) moves its pixel's operator data from the
// slot into registers when it starts a tile and releases the slot at once; then it runs every
// column of the tile from registers.  For the operator that data is the k x k pixel block
//
//     P_i = diag_j(tau_j (kappa_j^2 + L_ii)) + sum_c d_ci a_c a_c^T       (formed once per pixel)
//
// with the ELL weights and the places of the neighbours, so a column costs k^2 + E k FMAs
// (w = P_i z_i + tau o sum_e v_e z_{col_e}) instead of the (2k + 1) m + 2k + E k of the
// one-column form; for the update it is the factor of P_i.  Units run tile-major: tile lt of
// the CTA, then its active columns one after another, so the tile's gathers of neighbours one
// image row away also serve all columns from L2.
//
// Dot products: each unit's per-warp sums go to the column's per-warp accumulators, the last CTA
// of a system sums them in a fixed order (the last-CTA protocol of pcg_kernels.cuh).  Every
// mbarrier wait is bounded; on expiry the CTA records SYLV_E_TIMEOUT, thread 0 waits (bounded)
// for the copies still in flight (the last ring-depth vector units and MC_NOP operator slots
// issued are the only ones that can be), and the CTA leaves without publishing partial sums.
#pragma once

#include "pcg_tma.cuh"

namespace sylv {
namespace tma {

constexpr int MC_NOP = 2;   // operator slots
constexpr int MC_NVS = 2;   // vector stages of the inner kernels (12-32 KB each)
constexpr int MC_NVS_X = 4; // vector stages of the stand-alone apply (2k rows each: two
                            // columns per unit, so a warp keeps both columns' gathers in flight)

template <int NVS = MC_NVS>
struct McPipe {
  uint64_t ofull[MC_NOP], oempty[MC_NOP];
  uint64_t vfull[NVS], vempty[NVS];
  int otile[MC_NOP];        // tile staged in an operator slot (-1: no more tiles)
  int cols[RMAX];           // active columns
  int nact;
  int bad;
  int o_issued;             // operator slots issued (tiles, sentinel included)
  int v_issued;             // vector units issued
};

template <int NVS>
__device__ __forceinline__ void mc_init(McPipe<NVS>& mp) {
  for (int s = 0; s < MC_NOP; ++s) {
    mbar_init(&mp.ofull[s], 1);
    mbar_init(&mp.oempty[s], NCONS);
  }
  for (int s = 0; s < NVS; ++s) {
    mbar_init(&mp.vfull[s], 1);
    mbar_init(&mp.vempty[s], NCONS);
  }
  mp.bad = 0;
  mp.o_issued = 0;
  mp.v_issued = 0;
  fence_mbar_init();
}

// Producer side: lane 0 waits (bounded) for the consumers to release a slot or stage; the
// result is broadcast to the warp.  false: give up (timeout, or the consumers gave up).
template <int NVS>
__device__ __forceinline__ bool mc_wait_release(McPipe<NVS>& mp, uint64_t* bar,
                                                uint32_t parity, long long budget) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  if (lane == 0) ok = mbar_wait_bounded(bar, parity, budget);
  ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  if (!ok || mp.bad) {
    if (lane == 0) mp.bad = 1;
    return false;
  }
  return true;
}

// Producer warp.  next_tile(lt) gives the CTA's lt-th tile (< 0: none left).  op_issue(tile,
// slot, bar) issues the tile's operator rows into the slot and arms bar with their bytes;
// vec_issue(tile, col, stage, bar) the same for one column's vector rows.  After the last
// tile a sentinel slot (tile -1, no copies) tells the consumers to stop.
template <int NVS, typename NextTile, typename OpIssue, typename VecIssue>
__device__ __forceinline__ void mc_produce(McPipe<NVS>& mp, unsigned char* opbuf,
                                           int op_bytes,
                                           unsigned char* vecbuf, int vec_bytes,
                                           NextTile&& next_tile, OpIssue&& op_issue,
                                           VecIssue&& vec_issue,
                                           long long budget = WAIT_BUDGET_CYCLES) {
  const int lane = threadIdx.x & 31;
  const int na = mp.nact;
  int u = 0;
  for (int lt = 0;; ++lt) {
    const int tile = next_tile(lt);
    const int os = lt % MC_NOP;
    if (lt >= MC_NOP && !mc_wait_release(mp, &mp.oempty[os], ((lt / MC_NOP) - 1) & 1, budget))
      return;
    if (lane == 0) mp.otile[os] = tile;
    __syncwarp();
    if (tile < 0) {
      if (lane == 0) {
        mbar_arrive(&mp.ofull[os]);
        mp.o_issued = lt + 1;
      }
      return;
    }
    fence_proxy_async();   // the consumers' reads of the slot before the copies into it
    op_issue(tile, opbuf + (size_t)os * op_bytes, &mp.ofull[os]);
    if (lane == 0) mp.o_issued = lt + 1;
    for (int a = 0; a < na; ++a, ++u) {
      const int vs = u % NVS;
      if (u >= NVS && !mc_wait_release(mp, &mp.vempty[vs], ((u / NVS) - 1) & 1, budget))
        return;
      fence_proxy_async();
      vec_issue(tile, mp.cols[a], vecbuf + (size_t)vs * vec_bytes, &mp.vfull[vs]);
      if (lane == 0) mp.v_issued = u + 1;
    }
  }
}

// Consumer warps.  on_tile(tile, slot) reads the slot into registers (the slot is released
// right after); on_unit(tile, col, stage, release) computes one column of the tile from the
// stage and calls release() once it has read the stage.
template <int NVS, typename OnTile, typename OnUnit>
__device__ __forceinline__ void mc_consume(McPipe<NVS>& mp, const unsigned char* opbuf,
                                           int op_bytes,
                                           const unsigned char* vecbuf, int vec_bytes,
                                           OnTile&& on_tile, OnUnit&& on_unit,
                                           long long budget = WAIT_BUDGET_CYCLES) {
  const int lane = threadIdx.x & 31;
  const int na = mp.nact;
  int u = 0;
  for (int lt = 0;; ++lt) {
    const int os = lt % MC_NOP;
    if (!mbar_wait_bounded(&mp.ofull[os], (lt / MC_NOP) & 1, budget) || mp.bad) {
      mp.bad = 1;
      return;
    }
    const int tile = mp.otile[os];
    if (tile < 0) return;
    on_tile(tile, opbuf + (size_t)os * op_bytes);
    __syncwarp();
    if (lane == 0) mbar_arrive(&mp.oempty[os]);
    for (int a = 0; a < na; ++a, ++u) {
      const int vs = u % NVS;
      if (!mbar_wait_bounded(&mp.vfull[vs], (u / NVS) & 1, budget) || mp.bad) {
        mp.bad = 1;
        return;
      }
      auto release = [&]() {
        __syncwarp();
        if (lane == 0) mbar_arrive(&mp.vempty[vs]);
      };
      on_unit(tile, mp.cols[a], vecbuf + (size_t)vs * vec_bytes, release);
    }
  }
}

// After both roles: on a recorded timeout, flag it, wait (bounded) for the copies that can
// still be in flight and report true (the caller leaves without partial sums).
template <int NVS>
__device__ __forceinline__ bool mc_failed(McPipe<NVS>& mp, unsigned int* err) {
  __syncthreads();
  if (!mp.bad) return false;
  if (threadIdx.x == 0) {
    atomicOr(err, 1u);
    for (int u = mp.v_issued > NVS ? mp.v_issued - NVS : 0; u < mp.v_issued; ++u)
      mbar_wait_bounded(&mp.vfull[u % NVS], (u / NVS) & 1);
    for (int t = mp.o_issued > MC_NOP ? mp.o_issued - MC_NOP : 0; t < mp.o_issued; ++t)
      mbar_wait_bounded(&mp.ofull[t % MC_NOP], (t / MC_NOP) & 1);
  }
  __syncthreads();
  return true;
}

// Issues `rows` rows of TILE_PX 4-byte entries, row q from src(q), into dst (lane-strided);
// lane 0 arms bar with their bytes first.
template <typename Src>
__device__ __forceinline__ void issue_rows(float* dst, int rows, uint64_t* bar, Src&& src) {
  const int lane = threadIdx.x & 31;
  const uint32_t rowb = TILE_PX * 4;
  if (lane == 0) mbar_expect_tx(bar, (uint32_t)rows * rowb);
  __syncwarp();
  for (int q = lane; q < rows; q += 32) bulk_load(dst + (size_t)q * TILE_PX, src(q), rowb, bar);
}

// ---------------------------------------------------------------------------------------------
// Operator data of one pixel in registers
// ---------------------------------------------------------------------------------------------
template <int K, int E>
struct PixelOp {
  static constexpr int NB = K * (K + 1) / 2;
  float P[NB];        // pixel block, packed lower triangle, row-major
  float v[E];         // ELL weights of the off-diagonal entries of L
  int32_t c[E];       // neighbour e: its pixel index, or its position in the tile
  uint32_t in_tile;   // bit e: neighbour e lies in this tile
};

// Operator slot rows of the operator kernels: D (M), ELL values (E), diagonal (1), ELL columns.
template <int M, int E>
struct McOpRows {
  static constexpr int D = 0, VAL = M, DIAG = M + E, COL = M + E + 1, ROWS = M + 2 * E + 1;
  static constexpr int BYTES = ROWS * TILE_PX * 4;
};

// P_i and the stencil entries of pixel t of the tile starting at `base` from an operator slot.
template <int K, int M, int E, int NV>
__device__ __forceinline__ void load_pixel_op(const CtaShared<float, NV>& sh, const float* slot,
                                              int t, int64_t base, PixelOp<K, E>& po) {
  using OR = McOpRows<M, E>;
#pragma unroll
  for (int q = 0; q < PixelOp<K, E>::NB; ++q) po.P[q] = 0.f;
#pragma unroll
  for (int c = 0; c < M; ++c) {
    const float d = slot[(OR::D + c) * TILE_PX + t];
    float a[K];
    load_row<K, float>(sh.A[c], a);
#pragma unroll
    for (int x = 0; x < K; ++x) {
      const float da = d * a[x];
#pragma unroll
      for (int y = 0; y <= x; ++y) po.P[x * (x + 1) / 2 + y] += da * a[y];
    }
  }
  const float dg = slot[OR::DIAG * TILE_PX + t];
#pragma unroll
  for (int j = 0; j < K; ++j) po.P[j * (j + 1) / 2 + j] += sh.tk2[j] + sh.tau[j] * dg;
  const int32_t* scol = reinterpret_cast<const int32_t*>(slot + (size_t)OR::COL * TILE_PX);
  po.in_tile = 0u;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int64_t col = scol[e * TILE_PX + t];
    po.v[e] = slot[(OR::VAL + e) * TILE_PX + t];
    const uint32_t loc = (uint32_t)(col - base);
    const bool in = loc < (uint32_t)TILE_PX;
    po.c[e] = in ? (int32_t)loc : (int32_t)col;
    po.in_tile |= (in ? 1u : 0u) << e;
  }
}

// w = G z at the pixel for UC columns at once (all their neighbour loads issued before any
// arithmetic): zi the pixel's values (from the stages), sz the stages' z rows (stride
// TILE_PX), zg the columns' vectors in global memory (stride ld).
template <int K, int E, int UC, int NV>
__device__ __forceinline__ void pixel_apply_mcn(const CtaShared<float, NV>& sh,
                                                const PixelOp<K, E>& po,
                                                const float* const (&sz)[UC],
                                                const float* const (&zg)[UC], int64_t ld,
                                                const float (&zi)[UC][K], float (&w)[UC][K]) {
  float nb[UC][E][K];
#pragma unroll
  for (int u = 0; u < UC; ++u) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const bool in = (po.in_tile >> e) & 1u;
      const float* src = in ? sz[u] + po.c[e] : zg[u] + po.c[e];
      const int64_t stride = in ? (int64_t)TILE_PX : ld;
#pragma unroll
      for (int j = 0; j < K; ++j) nb[u][e][j] = src[j * stride];
    }
  }
#pragma unroll
  for (int u = 0; u < UC; ++u) {
    float lap[K];
#pragma unroll
    for (int j = 0; j < K; ++j) lap[j] = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int j = 0; j < K; ++j) lap[j] += po.v[e] * nb[u][e][j];
#pragma unroll
    for (int j = 0; j < K; ++j) w[u][j] = sh.tau[j] * lap[j];
#pragma unroll
    for (int x = 0; x < K; ++x) {
#pragma unroll
      for (int y = 0; y <= x; ++y) {
        const float pxy = po.P[x * (x + 1) / 2 + y];
        w[u][x] += pxy * zi[u][y];
        if (y != x) w[u][y] += pxy * zi[u][x];
      }
    }
  }
}

// The same for one column.
template <int K, int E, int NV>
__device__ __forceinline__ void pixel_apply_mc(const CtaShared<float, NV>& sh,
                                               const PixelOp<K, E>& po, const float* sz,
                                               const float* zg, int64_t ld,
                                               const float (&zi)[K], float (&w)[K]) {
  const float* const szs[1] = {sz};
  const float* const zgs[1] = {zg};
  float zi1[1][K], w1[1][K];
#pragma unroll
  for (int j = 0; j < K; ++j) zi1[0][j] = zi[j];
  pixel_apply_mcn<K, E, 1, NV>(sh, po, szs, zgs, ld, zi1, w1);
#pragma unroll
  for (int j = 0; j < K; ++j) w[j] = w1[0][j];
}

// ---------------------------------------------------------------------------------------------
// inner_apply, several columns: d += alpha p (the previous iteration's step), p = z + beta p,
// q = G z + beta q, partial p . q (last CTA sets alpha)
// ---------------------------------------------------------------------------------------------
template <int K>
struct McApplyVec {
  static constexpr int Z = 0, P = K, Q = 2 * K, Dv = 3 * K, ROWS = 4 * K;
  static constexpr int BYTES = ROWS * TILE_PX * 4;
};

template <int K, int M, int E>
constexpr size_t mc_apply_smem() {
  return (size_t)MC_NOP * McOpRows<M, E>::BYTES + (size_t)MC_NVS * McApplyVec<K>::BYTES;
}

template <int K, int M, int E>
__global__ void __launch_bounds__(WS_THREADS, 2)
k_inner_apply_mc(const SysDesc* __restrict__ descs, const CtaRef* __restrict__ ctas,
                 Control* ctl) {
  using OR = McOpRows<M, E>;
  using VR = McApplyVec<K>;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ CtaShared<float, 1> sh;
  __shared__ __align__(8) McPipe<> mp;
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
      sh.sc[r] = float(cs.beta);
      sh.sc2[r] = float(cs.alpha);
      sh.aux[r] = cs.first;
    }
    sh.act[r] = act;
  }
  stage_operator<float, 1>(op, K, sh);
  zero_wacc<float, 1>(sh, R);
  if (threadIdx.x == 0) {
    int na = 0;
    for (int r = 0; r < R; ++r)
      if (sh.act[r]) mp.cols[na++] = r;
    mp.nact = na;
    mc_init(mp);
  }
  if (!__syncthreads_or(act)) return;

  const int64_t ld = op.ld, n = op.n;
  const int nsl = sd.nslots[0];
  float* zg = (float*)sd.vz;
  float* pg = (float*)sd.vp;
  float* qg = (float*)sd.vq;
  float* dgl = (float*)sd.vd;
  unsigned char* opbuf = dsm;
  unsigned char* vecbuf = dsm + (size_t)MC_NOP * OR::BYTES;
  const int warp = threadIdx.x >> 5;
  if (warp == NCONS) {
    if (!(ctl->inject_stall & STALL_APPLY))
      mc_produce(
          mp, opbuf, OR::BYTES, vecbuf, VR::BYTES,
          [&](int lt) {
            const int tile = cr.slot + lt * nsl;
            return tile < sd.ntiles ? tile : -1;
          },
          [&](int tile, unsigned char* slot, uint64_t* bar) {
            const int64_t base = (int64_t)tile * TILE_PX;
            issue_rows(reinterpret_cast<float*>(slot), OR::ROWS, bar, [&](int q) -> const void* {
              if (q < OR::VAL) return op.D32 + (size_t)(q - OR::D) * ld + base;
              if (q < OR::DIAG) return op.ell_val32 + (size_t)(q - OR::VAL) * ld + base;
              if (q == OR::DIAG) return op.diag32 + base;
              return op.ell_col + (size_t)(q - OR::COL) * ld + base;
            });
          },
          [&](int tile, int r, unsigned char* stage, uint64_t* bar) {
            const int64_t base = (int64_t)tile * TILE_PX;
            const size_t voff = (size_t)r * K * ld;
            const bool first = sh.aux[r] != 0;   // p, q and d are not read on a first iteration
            issue_rows(reinterpret_cast<float*>(stage), first ? K : VR::ROWS, bar,
                       [&](int q) -> const void* {
                         if (q < VR::P) return zg + voff + (size_t)(q - VR::Z) * ld + base;
                         if (q < VR::Q) return pg + voff + (size_t)(q - VR::P) * ld + base;
                         if (q < VR::Dv) return qg + voff + (size_t)(q - VR::Q) * ld + base;
                         return dgl + voff + (size_t)(q - VR::Dv) * ld + base;
                       });
          },
          pipe_budget(ctl));
  } else {
    const int t = threadIdx.x;
    PixelOp<K, E> po;
    int64_t base = 0;
    mc_consume(
        mp, opbuf, OR::BYTES, vecbuf, VR::BYTES,
        [&](int tile, const unsigned char* slot) {
          base = (int64_t)tile * TILE_PX;
          load_pixel_op<K, M, E>(sh, reinterpret_cast<const float*>(slot), t, base, po);
        },
        [&](int tile, int r, const unsigned char* stage_b, auto&& release) {
          const float* stage = reinterpret_cast<const float*>(stage_b);
          const int64_t i = base + t;
          const size_t voff = (size_t)r * K * ld;
          const bool first = sh.aux[r] != 0;
          float zi[K], w[K];
#pragma unroll
          for (int j = 0; j < K; ++j) zi[j] = stage[(VR::Z + j) * TILE_PX + t];
          pixel_apply_mc<K, E>(sh, po, stage + (size_t)VR::Z * TILE_PX, zg + voff, ld, zi, w);
          const float beta = sh.sc[r], alpha = sh.sc2[r];
          float pn[K], qn[K], dv[K];
#pragma unroll
          for (int j = 0; j < K; ++j) {
            pn[j] = zi[j];
            qn[j] = w[j];
            dv[j] = 0.f;
            if (!first) {
              const float po = stage[(VR::P + j) * TILE_PX + t];
              dv[j] = stage[(VR::Dv + j) * TILE_PX + t] + alpha * po;
              pn[j] += beta * po;
              qn[j] += beta * stage[(VR::Q + j) * TILE_PX + t];
            }
          }
          release();
          float pq = 0.f;
          if (i < n) {
#pragma unroll
            for (int j = 0; j < K; ++j) {
              if (!first) dgl[voff + (size_t)j * ld + i] = dv[j];
              pg[voff + (size_t)j * ld + i] = pn[j];
              qg[voff + (size_t)j * ld + i] = qn[j];
              pq += pn[j] * qn[j];
            }
          }
          const float v1[1] = {pq};
          warp_accumulate_f32<float, 1>(sh, r, v1);
        },
        pipe_budget(ctl));
  }
  if (mc_failed(mp, &ctl->error)) return;
  double tot[RMAX][1];
  if (!finish_partials<float, 1>(sd, cr.slot, nsl, sh, R, tot)) return;
  if (threadIdx.x == 0) {
    for (int r = 0; r < R; ++r)
      if (sh.act[r]) after_apply(sd.st[r], tot[r][0], ctl, true);
    *sd.counter = 0u;
  }
}

// ---------------------------------------------------------------------------------------------
// inner_update, several columns: r -= alpha q, z = P^{-1} r, partial r . z and r . r (last CTA
// sets beta, gamma and the stopping state; d += alpha p is the next operator kernel's)
// ---------------------------------------------------------------------------------------------
template <int K>
struct McUpdateRows {
  static constexpr int NB = K * (K + 1) / 2, NB2 = (NB + 1) / 2;
  static constexpr int S = 0, L16 = K, OP_ROWS = K + NB2;            // operator slot
  static constexpr int R = 0, Q = K, VEC_ROWS = 2 * K;                 // vector stage
  static constexpr int OP_BYTES = OP_ROWS * TILE_PX * 4, VEC_BYTES = VEC_ROWS * TILE_PX * 4;
};

template <int K>
constexpr size_t mc_update_smem() {
  return (size_t)MC_NOP * McUpdateRows<K>::OP_BYTES +
         (size_t)MC_NVS * McUpdateRows<K>::VEC_BYTES;
}

template <int K, int M>
__global__ void __launch_bounds__(WS_THREADS, 2)
k_inner_update_mc(const SysDesc* __restrict__ descs, const CtaRef* __restrict__ ctas,
                  Control* ctl) {
  using L = McUpdateRows<K>;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ CtaShared<float, 2> sh;   // (mixing rows unused here: the factor is stored)
  __shared__ __align__(8) McPipe<> mp;
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
      sh.sc[r] = float(cs.alpha);
    }
    sh.act[r] = act;
  }
  zero_wacc<float, 2>(sh, R);
  if (threadIdx.x == 0) {
    int na = 0;
    for (int r = 0; r < R; ++r)
      if (sh.act[r]) mp.cols[na++] = r;
    mp.nact = na;
    mc_init(mp);
  }
  if (!__syncthreads_or(act)) return;

  const int64_t ld = op.ld, n = op.n;
  const int nsl = sd.nslots[1];
  const bool prec = ctl->precond == SYLV_PRECOND_BLOCK_JACOBI;
  float* rg = (float*)sd.vr;
  float* zg = (float*)sd.vz;
  const float* qg = (const float*)sd.vq;
  unsigned char* opbuf = dsm;
  unsigned char* vecbuf = dsm + (size_t)MC_NOP * L::OP_BYTES;
  const int warp = threadIdx.x >> 5;
  if (warp == NCONS) {
    if (!(ctl->inject_stall & STALL_UPDATE))
      mc_produce(
          mp, opbuf, L::OP_BYTES, vecbuf, L::VEC_BYTES,
          [&](int lt) {
            const int tile = cr.slot + lt * nsl;
            return tile < sd.ntiles ? tile : -1;
          },
          [&](int tile, unsigned char* slot, uint64_t* bar) {
            const int64_t base = (int64_t)tile * TILE_PX;
            issue_rows(reinterpret_cast<float*>(slot), prec ? L::OP_ROWS : 0, bar,
                       [&](int q) -> const void* {
                         if (q < K) return op.fs32 + (size_t)q * ld + base;
                         return op.fl16 + (size_t)(q - K) * ld + base;
                       });
          },
          [&](int tile, int r, unsigned char* stage, uint64_t* bar) {
            const int64_t base = (int64_t)tile * TILE_PX;
            const size_t voff = (size_t)r * K * ld;
            issue_rows(reinterpret_cast<float*>(stage), L::VEC_ROWS, bar,
                       [&](int q) -> const void* {
                         if (q < L::Q) return rg + voff + (size_t)(q - L::R) * ld + base;
                         return qg + voff + (size_t)(q - L::Q) * ld + base;
                       });
          },
          pipe_budget(ctl));
  } else {
    const int t = threadIdx.x;
    BlockChol<K, float> f;
    int64_t base = 0;
    mc_consume(
        mp, opbuf, L::OP_BYTES, vecbuf, L::VEC_BYTES,
        [&](int tile, const unsigned char* slot_b) {
          base = (int64_t)tile * TILE_PX;
          if (prec) {
            const float* slot = reinterpret_cast<const float*>(slot_b);
            const __half2* sl = reinterpret_cast<const __half2*>(slot + (size_t)L::L16 * TILE_PX);
#pragma unroll
            for (int x = 0; x < K; ++x) f.s[x] = slot[(L::S + x) * TILE_PX + t];
#pragma unroll
            for (int x = 0; x < L::NB; x += 2) {
              const float2 v = __half22float2(sl[(x / 2) * TILE_PX + t]);
              f.l[x] = v.x;
              if (x + 1 < L::NB) f.l[x + 1] = v.y;
            }
          }
        },
        [&](int tile, int r, const unsigned char* stage_b, auto&& release) {
          const float* stage = reinterpret_cast<const float*>(stage_b);
          const int64_t i = base + t;
          const size_t voff = (size_t)r * K * ld;
          const float alpha = sh.sc[r];
          float ri[K], zi[K];
#pragma unroll
          for (int j = 0; j < K; ++j)
            ri[j] = stage[(L::R + j) * TILE_PX + t] - alpha * stage[(L::Q + j) * TILE_PX + t];
          release();
          if (prec) {
            block_solve<K, float>(f, ri, zi);
          } else {
#pragma unroll
            for (int j = 0; j < K; ++j) zi[j] = ri[j];
          }
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
          const float v2[2] = {rz, rr};
          warp_accumulate_f32<float, 2>(sh, r, v2);
        },
        pipe_budget(ctl));
  }
  if (mc_failed(mp, &ctl->error)) return;
  double tot[RMAX][2];
  if (!finish_partials<float, 2>(sd, cr.slot, nsl, sh, R, tot)) return;
  if (threadIdx.x == 0) {
    for (int r = 0; r < R; ++r)
      if (sh.act[r]) after_update(sd.st[r], tot[r][0], tot[r][1], ctl, true);
    *sd.counter = 0u;
  }
}

// ---------------------------------------------------------------------------------------------
// stand-alone operator apply, several columns: Y = G X for FP32 caller vectors
// ---------------------------------------------------------------------------------------------
// Tiles come from a counter (ctr[1], one ahead), so CTAs on faster SMs take more of them (no
// partial sums here: the split changes nothing in the result).  ctr[0]: timeout flag; ctr[2]:
// CTAs done (the last one zeroes ctr[1] and ctr[2] for the next launch).  Used when n is a
// multiple of TILE_PX and every caller row starts 16-byte aligned.
template <int K>
struct McXVec {
  static constexpr int BYTES = 2 * K * TILE_PX * 4;   // x rows of a column pair
};

template <int K, int M, int E>
constexpr size_t mc_applyx_smem() {
  return (size_t)MC_NOP * McOpRows<M, E>::BYTES + (size_t)MC_NVS_X * McXVec<K>::BYTES;
}

template <int K, int M, int E>
__global__ void __launch_bounds__(WS_THREADS, 2)
k_apply_mc(OpData op, const float* __restrict__ X, float* __restrict__ Y, int R,
           unsigned int* ctr) {
  using OR = McOpRows<M, E>;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ CtaShared<float, 1> sh;
  __shared__ __align__(8) McPipe<MC_NVS_X> mp;
  stage_operator<float, 1>(op, K, sh);
  const int npair = (R + 1) / 2;   // a unit is a pair of columns (the last may be single)
  if (threadIdx.x == 0) {
    for (int a = 0; a < npair; ++a) mp.cols[a] = a;
    mp.nact = npair;
    mc_init(mp);
  }
  __syncthreads();
  const int64_t ldu = op.ldu, ld = op.ld;
  const int ntiles = (int)(op.n / TILE_PX);
  unsigned char* opbuf = dsm;
  unsigned char* vecbuf = dsm + (size_t)MC_NOP * OR::BYTES;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == NCONS) {
    int ahead = 0;
    if (lane == 0) ahead = (int)atomicAdd(ctr + 1, 1u);
    mc_produce(
        mp, opbuf, OR::BYTES, vecbuf, McXVec<K>::BYTES,
        [&](int) {
          const int tile = __shfl_sync(0xffffffffu, ahead, 0);
          if (tile >= ntiles) return -1;
          if (lane == 0) ahead = (int)atomicAdd(ctr + 1, 1u);
          return tile;
        },
        [&](int tile, unsigned char* slot, uint64_t* bar) {
          const int64_t base = (int64_t)tile * TILE_PX;
          issue_rows(reinterpret_cast<float*>(slot), OR::ROWS, bar, [&](int q) -> const void* {
            if (q < OR::VAL) return op.D32 + (size_t)(q - OR::D) * ld + base;
            if (q < OR::DIAG) return op.ell_val32 + (size_t)(q - OR::VAL) * ld + base;
            if (q == OR::DIAG) return op.diag32 + base;
            return op.ell_col + (size_t)(q - OR::COL) * ld + base;
          });
        },
        [&](int tile, int a, unsigned char* stage, uint64_t* bar) {
          const int64_t base = (int64_t)tile * TILE_PX;
          const int nc = 2 * a + 1 < R ? 2 : 1;
          const size_t xoff = (size_t)(2 * a) * K * ldu;   // the pair's K or 2K rows follow
          issue_rows(reinterpret_cast<float*>(stage), nc * K, bar, [&](int q) -> const void* {
            return X + xoff + (size_t)q * ldu + base;
          });
        });
  } else {
    const int t = threadIdx.x;
    PixelOp<K, E> po;
    int64_t base = 0;
    mc_consume(
        mp, opbuf, OR::BYTES, vecbuf, McXVec<K>::BYTES,
        [&](int tile, const unsigned char* slot) {
          base = (int64_t)tile * TILE_PX;
          load_pixel_op<K, M, E>(sh, reinterpret_cast<const float*>(slot), t, base, po);
        },
        [&](int tile, int a, const unsigned char* stage_b, auto&& release) {
          const float* stage = reinterpret_cast<const float*>(stage_b);
          const bool two = 2 * a + 1 < R;   // a single last column is computed twice
          const size_t x0 = (size_t)(2 * a) * K * ldu, x1 = two ? x0 + (size_t)K * ldu : x0;
          const float* const sz[2] = {stage, two ? stage + (size_t)K * TILE_PX : stage};
          const float* const zg[2] = {X + x0, X + x1};
          float xi[2][K], w[2][K];
#pragma unroll
          for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int j = 0; j < K; ++j) xi[u][j] = sz[u][j * TILE_PX + t];
          pixel_apply_mcn<K, E, 2>(sh, po, sz, zg, ldu, xi, w);
          release();
#pragma unroll
          for (int j = 0; j < K; ++j) Y[x0 + (size_t)j * ldu + base + t] = w[0][j];
          if (two) {
#pragma unroll
            for (int j = 0; j < K; ++j) Y[x1 + (size_t)j * ldu + base + t] = w[1][j];
          }
        });
  }
  const bool bad = mc_failed(mp, ctr);
  (void)bad;
  if (threadIdx.x == 0) {
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
