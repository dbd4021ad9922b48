// FP32 inner-iteration kernels with bulk-copy (TMA) staging of each tile's streams.
//
// Same arithmetic as k_inner_apply / k_inner_update, restructured for the memory system:
// every contiguous stream a tile needs (its own rows of z, p, q or d, p, r, q, the noise maps
// D, the ELL rows of L and its diagonal; TILE_PX values each) is brought into shared memory by
// cp.async.bulk copies that complete on an mbarrier, two units ahead of the computation.
// A unit is one (tile, column) pair.  The loads therefore need no registers while in flight,
// and the only per-thread global loads left are the stencil gathers that fall outside the
// tile (the neighbours one image row away); gathers inside the tile read the staged rows.
//
// Waits on an mbarrier are bounded (about a second of SM clock); when one expires the CTA
// records SYLV_E_TIMEOUT in Control::error, drains its own copies (again bounded) and leaves
// without publishing partial sums, so the host sees the error at its next poll.
#pragma once

#include "pcg_kernels.cuh"

namespace sylv {
namespace tma {

constexpr int NSTAGE = 2;
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

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > WAIT_BUDGET_CYCLES) return false;
  }
  return true;
}

// Units of a CTA: its tiles (slot, slot + nslots, ...) times its active columns.
struct Units {
  int ntl;     // tiles of this CTA
  int nact;    // active columns
  int n;       // units
};

__device__ __forceinline__ Units count_units(const SysDesc& sd, int slot, int nact) {
  Units u;
  u.ntl = slot < sd.ntiles ? (sd.ntiles - slot + sd.nslots - 1) / sd.nslots : 0;
  u.nact = nact;
  u.n = u.ntl * nact;
  return u;
}

// Shared-memory stage layouts (rows of TILE_PX entries of 4 bytes).
template <int K, int M, int E>
struct ApplyLayout {
  static constexpr int Z = 0, P = K, Q = 2 * K, D = 3 * K, VAL = 3 * K + M,
                       DIAG = 3 * K + M + E, COL = 3 * K + M + E + 1;
  static constexpr int ROWS = 3 * K + M + 2 * E + 1;
  static constexpr int STAGE_BYTES = ROWS * TILE_PX * 4;
};

// Update stage: d, p, r, q (4K float rows), the preconditioner scaling (K float rows) and its
// FP16 factor (K(K+1)/2 half rows, packed two per float row).
template <int K, int M>
struct UpdateLayout {
  static constexpr int Dv = 0, P = K, R = 2 * K, Q = 3 * K, S = 4 * K, L16 = 5 * K;
  static constexpr int NB = K * (K + 1) / 2;
  static constexpr int FLOAT_ROWS = 5 * K;
  static constexpr int STAGE_BYTES = FLOAT_ROWS * TILE_PX * 4 + NB * TILE_PX * 2;
  static constexpr int COPIES = 5 * K + NB;
  static constexpr int NOPREC_COPIES = 4 * K;
};

// On an expired wait: flag the error, drain this CTA's outstanding copies (bounded) and
// return true (the caller leaves).
__device__ __forceinline__ bool handle_timeout(bool ok, uint64_t* bars, int next_unit,
                                               int nunits, Control* ctl) {
  const bool bad = __syncthreads_or(!ok);
  if (!bad) return false;
  if (threadIdx.x == 0) {
    atomicOr(&ctl->error, 1u);
    for (int u = next_unit; u < nunits && u < next_unit + NSTAGE; ++u)
      mbar_wait_bounded(&bars[u % NSTAGE], (u / NSTAGE) & 1);
  }
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------------------------
// inner_apply (staged): p = z + beta p, q = G z + beta q, partial p . q
// ---------------------------------------------------------------------------------------------
template <int K, int M, int E>
__global__ void __launch_bounds__(TILE_PX, 2)
k_inner_apply_tma(const SysDesc* __restrict__ descs, const CtaRef* __restrict__ ctas,
                  Control* ctl) {
  using L = ApplyLayout<K, M, E>;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ CtaShared<float, 1> sh;
  __shared__ __align__(8) uint64_t bars[NSTAGE];
  __shared__ int s_cols[RMAX];
  __shared__ int s_nact;
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
      sh.aux[r] = cs.first;
    }
    sh.act[r] = act;
  }
  stage_operator<float, 1>(op, K, sh);
  zero_wacc<float, 1>(sh, R);
  if (threadIdx.x == 0) {
    int na = 0;
    for (int r = 0; r < R; ++r)
      if (sh.act[r]) s_cols[na++] = r;
    s_nact = na;
    for (int s = 0; s < NSTAGE; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  if (!__syncthreads_or(act)) return;

  const int64_t ld = op.ld, n = op.n;
  const Units U = count_units(sd, cr.slot, s_nact);
  const float* zg = (const float*)sd.vz;
  float* pg = (float*)sd.vp;
  float* qg = (float*)sd.vq;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // warp 0 issues the copies of unit u into stage u % NSTAGE
  auto issue = [&](int u) {
    const int st = u % NSTAGE;
    const int tile = cr.slot + (u / U.nact) * sd.nslots;
    const int r = s_cols[u % U.nact];
    const bool first = sh.aux[r] != 0;
    const int64_t base = (int64_t)tile * TILE_PX;
    float* stage = reinterpret_cast<float*>(dsm + (size_t)st * L::STAGE_BYTES);
    const uint32_t rowb = TILE_PX * 4;
    const int nrows = first ? L::ROWS - 2 * K : L::ROWS;
    if (lane == 0) {
      fence_proxy_async();
      mbar_expect_tx(&bars[st], (uint32_t)nrows * rowb);
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
      if (src) bulk_load(stage + (size_t)q * TILE_PX, src, rowb, &bars[st]);
    }
  };

  if (warp == 0) {
    for (int u = 0; u < NSTAGE && u < U.n; ++u) issue(u);
  }
  for (int u = 0; u < U.n; ++u) {
    const int st = u % NSTAGE;
    const bool ok = mbar_wait_bounded(&bars[st], (u / NSTAGE) & 1);
    if (handle_timeout(ok, bars, u, U.n, ctl)) return;
    const int tile = cr.slot + (u / U.nact) * sd.nslots;
    const int r = s_cols[u % U.nact];
    const int64_t base = (int64_t)tile * TILE_PX;
    const int t = threadIdx.x;
    const int64_t i = base + t;
    const float* stage = reinterpret_cast<const float*>(dsm + (size_t)st * L::STAGE_BYTES);
    const int32_t* scol = reinterpret_cast<const int32_t*>(stage + (size_t)L::COL * TILE_PX);
    const size_t voff = (size_t)r * K * ld;
    float zi[K], lap[K];
#pragma unroll
    for (int j = 0; j < K; ++j) zi[j] = stage[(L::Z + j) * TILE_PX + t];
    const float dg = stage[L::DIAG * TILE_PX + t];
#pragma unroll
    for (int j = 0; j < K; ++j) lap[j] = dg * zi[j];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int64_t c = scol[e * TILE_PX + t];
      const float v = stage[(L::VAL + e) * TILE_PX + t];
      const uint32_t loc = (uint32_t)(c - base);
      if (loc < (uint32_t)TILE_PX) {
#pragma unroll
        for (int j = 0; j < K; ++j) lap[j] += v * stage[(L::Z + j) * TILE_PX + loc];
      } else {
#pragma unroll
        for (int j = 0; j < K; ++j) lap[j] += v * __ldg(zg + voff + (size_t)j * ld + c);
      }
    }
    float w[K];
#pragma unroll
    for (int j = 0; j < K; ++j) w[j] = sh.tk2[j] * zi[j] + sh.tau[j] * lap[j];
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const float d = stage[(L::D + c) * TILE_PX + t];
      float a[K];
      load_row<K, float>(sh.A[c], a);
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < K; ++j) s += a[j] * zi[j];
      s *= d;
#pragma unroll
      for (int j = 0; j < K; ++j) w[j] += a[j] * s;
    }
    const bool first = sh.aux[r] != 0;
    const float beta = sh.sc[r];
    float pq = 0.f;
    if (i < n) {
#pragma unroll
      for (int j = 0; j < K; ++j) {
        float pj = zi[j], qj = w[j];
        if (!first) {
          pj += beta * stage[(L::P + j) * TILE_PX + t];
          qj += beta * stage[(L::Q + j) * TILE_PX + t];
        }
        pg[voff + (size_t)j * ld + i] = pj;
        qg[voff + (size_t)j * ld + i] = qj;
        pq += pj * qj;
      }
    }
    const double v1[1] = {double(pq)};
    warp_accumulate<float, 1>(sh, r, v1);
    __syncthreads();  // stage st fully read
    if (warp == 0 && u + NSTAGE < U.n) issue(u + NSTAGE);
  }
  double tot[RMAX][1];
  if (!finish_partials<float, 1>(sd, cr.slot, sh, R, tot)) return;
  if (threadIdx.x == 0) {
    for (int r = 0; r < R; ++r) {
      if (!sh.act[r]) continue;
      ColState& cs = sd.st[r];
      const double pq = tot[r][0];
      if (pq > 0.0 && isfinite(pq)) {
        cs.alpha = cs.gamma / pq;
        cs.first = 0;
      } else if (cs.rr_in == 0.0) {
        cs.phase = PH_INNER_DONE;
        atomicSub(&ctl->n_active, 1u);
      } else {
        cs.phase = PH_FAILED;
        cs.status = SYLV_E_BREAKDOWN;
        atomicSub(&ctl->n_active, 1u);
        atomicSub(&ctl->n_unfinished, 1u);
      }
    }
    *sd.counter = 0u;
  }
}

// ---------------------------------------------------------------------------------------------
// inner_update (staged): d += alpha p, r -= alpha q, z = P^{-1} r, partial r . z and r . r
// ---------------------------------------------------------------------------------------------
template <int K, int M>
__global__ void __launch_bounds__(TILE_PX, 2)
k_inner_update_tma(const SysDesc* __restrict__ descs, const CtaRef* __restrict__ ctas,
                   Control* ctl) {
  using L = UpdateLayout<K, M>;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ CtaShared<float, 2> sh;  // (mixing rows unused here: the factor is stored)
  __shared__ __align__(8) uint64_t bars[NSTAGE];
  __shared__ int s_cols[RMAX];
  __shared__ int s_nact;
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
  stage_operator<float, 2>(op, K, sh);
  zero_wacc<float, 2>(sh, R);
  if (threadIdx.x == 0) {
    int na = 0;
    for (int r = 0; r < R; ++r)
      if (sh.act[r]) s_cols[na++] = r;
    s_nact = na;
    for (int s = 0; s < NSTAGE; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  if (!__syncthreads_or(act)) return;

  const int64_t ld = op.ld, n = op.n;
  const bool prec = ctl->precond == SYLV_PRECOND_BLOCK_JACOBI;
  const Units U = count_units(sd, cr.slot, s_nact);
  float* dg_ = (float*)sd.vd;
  float* rg = (float*)sd.vr;
  float* zg = (float*)sd.vz;
  const float* pg = (const float*)sd.vp;
  const float* qg = (const float*)sd.vq;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  auto issue = [&](int u) {
    const int st = u % NSTAGE;
    const int tile = cr.slot + (u / U.nact) * sd.nslots;
    const int r = s_cols[u % U.nact];
    const int64_t base = (int64_t)tile * TILE_PX;
    float* stage = reinterpret_cast<float*>(dsm + (size_t)st * L::STAGE_BYTES);
    const uint32_t rowb = TILE_PX * 4;
    const int ncopies = prec ? L::COPIES : L::NOPREC_COPIES;
    const uint32_t bytes = prec ? (uint32_t)L::STAGE_BYTES : (uint32_t)(4 * K * rowb);
    if (lane == 0) {
      fence_proxy_async();
      mbar_expect_tx(&bars[st], bytes);
    }
    __syncwarp();
    const size_t voff = (size_t)r * K * ld;
    __half* stage_l16 = reinterpret_cast<__half*>(stage + (size_t)L::L16 * TILE_PX);
    for (int q = lane; q < ncopies; q += 32) {
      if (q < 5 * K) {
        const float* src;
        if (q < K) src = dg_ + voff + (size_t)q * ld + base;
        else if (q < 2 * K) src = pg + voff + (size_t)(q - K) * ld + base;
        else if (q < 3 * K) src = rg + voff + (size_t)(q - 2 * K) * ld + base;
        else if (q < 4 * K) src = qg + voff + (size_t)(q - 3 * K) * ld + base;
        else src = op.fs32 + (size_t)(q - 4 * K) * ld + base;
        bulk_load(stage + (size_t)q * TILE_PX, src, rowb, &bars[st]);
      } else {
        const int a = q - 5 * K;
        bulk_load(stage_l16 + (size_t)a * TILE_PX, op.fl16 + (size_t)a * ld + base,
                  TILE_PX * 2, &bars[st]);
      }
    }
  };

  if (warp == 0) {
    for (int u = 0; u < NSTAGE && u < U.n; ++u) issue(u);
  }
  int last_tile = -1;
  BlockChol<K, float> f;
  for (int u = 0; u < U.n; ++u) {
    const int st = u % NSTAGE;
    const bool ok = mbar_wait_bounded(&bars[st], (u / NSTAGE) & 1);
    if (handle_timeout(ok, bars, u, U.n, ctl)) return;
    const int tile = cr.slot + (u / U.nact) * sd.nslots;
    const int r = s_cols[u % U.nact];
    const int t = threadIdx.x;
    const int64_t i = (int64_t)tile * TILE_PX + t;
    const float* stage = reinterpret_cast<const float*>(dsm + (size_t)st * L::STAGE_BYTES);
    if (prec && tile != last_tile) {
      const __half* sl16 = reinterpret_cast<const __half*>(stage + (size_t)L::L16 * TILE_PX);
#pragma unroll
      for (int x = 0; x < K; ++x) f.s[x] = stage[(L::S + x) * TILE_PX + t];
#pragma unroll
      for (int x = 0; x < L::NB; ++x) f.l[x] = __half2float(sl16[x * TILE_PX + t]);
      last_tile = tile;
    }
    const float alpha = sh.sc[r];
    const size_t voff = (size_t)r * K * ld;
    float rz = 0.f, rr = 0.f;
    if (i < n) {
      float ri[K], zi[K];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const float dn = stage[(L::Dv + j) * TILE_PX + t] + alpha * stage[(L::P + j) * TILE_PX + t];
        ri[j] = stage[(L::R + j) * TILE_PX + t] - alpha * stage[(L::Q + j) * TILE_PX + t];
        dg_[voff + (size_t)j * ld + i] = dn;
        rg[voff + (size_t)j * ld + i] = ri[j];
      }
      if (prec) {
        block_solve<K, float>(f, ri, zi);
      } else {
#pragma unroll
        for (int j = 0; j < K; ++j) zi[j] = ri[j];
      }
#pragma unroll
      for (int j = 0; j < K; ++j) {
        zg[voff + (size_t)j * ld + i] = zi[j];
        rz += ri[j] * zi[j];
        rr += ri[j] * ri[j];
      }
    }
    const double v2[2] = {double(rz), double(rr)};
    warp_accumulate<float, 2>(sh, r, v2);
    __syncthreads();
    if (warp == 0 && u + NSTAGE < U.n) issue(u + NSTAGE);
  }
  double tot[RMAX][2];
  if (!finish_partials<float, 2>(sd, cr.slot, sh, R, tot)) return;
  if (threadIdx.x == 0) {
    for (int r = 0; r < R; ++r) {
      if (!sh.act[r]) continue;
      ColState& cs = sd.st[r];
      const double rz = tot[r][0], rr = tot[r][1];
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
    *sd.counter = 0u;
  }
}

}  // namespace tma
}  // namespace sylv
