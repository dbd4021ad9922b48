// True residual of the mixed-precision refinement in double-float arithmetic (df32.cuh).
//
// r = B - G X (Algorithm 2's residual, evaluated on the true FP64 iterate at every refinement
// step) with G in its pixel-block form: (G x)_i = P_i x_i + tau o (sum_e v_e x_{col_e}), P_i the
// k x k pixel block (prior diagonal and data term, eq. block-vector-mapping-matvec) and v_e the
// off-diagonal weights of L (Algorithm 1's stencil).  The handle keeps P_i and v_e split into
// FP32 (hi, lo) pairs (set-up); X and B are split here.  Each product is accumulated exactly in
// its leading part and with its rounding error in a compensation term (Dot2), so the residual
// comes out with about 2^-44 (|b| + |G||X|) accuracy per element although no FP64 operation is
// issued: on this GPU the FP64 unit (1/64 of FP32) bounds the FP64 form of this kernel.
//
// A pixel with an input outside the split's range, or a non-finite result, is recomputed in
// FP64 from the FP64 copies (apply_pixel_blk64).  The kernel then rounds r to FP32 for the inner
// solve, sets d = 0, applies the preconditioner and forms the partial sums of ||r||^2 (from the
// accurate residual), ||B||^2, r . z and r . r, like k_residual; the last CTA decides.
#pragma once

#include "df32.cuh"
#include "pcg_tma.cuh"

namespace sylv {

// Split FP64 values of this CTA's tile for one column: the pixels' own x in (hi, lo) rows,
// read by the stencil of in-tile neighbours (a hi of NaN marks a value outside the split range).
template <int K>
struct DfTile {
  float h[K][TILE_PX];
  float l[K][TILE_PX];
};

// lap_j += v_e * x_{col_e, j} for a batch of EC neighbours (split values), all sources j; for an
// even number of sources on pairs of sources with the packed instructions.
template <int K, int EC>
__device__ __forceinline__ void df_stencil(df::Acc (&lap)[K], const float (&vh)[EC],
                                           const float (&vl)[EC], const float (&nh)[EC][K],
                                           const float (&nl)[EC][K]) {
  if constexpr (K % 2 == 0) {
#pragma unroll
    for (int q = 0; q < K / 2; ++q) {
      df::Acc2 a{make_float2(lap[2 * q].s, lap[2 * q + 1].s),
                 make_float2(lap[2 * q].c, lap[2 * q + 1].c)};
#pragma unroll
      for (int e = 0; e < EC; ++e)
        df::fma2(a, make_float2(vh[e], vh[e]), make_float2(vl[e], vl[e]),
                 make_float2(nh[e][2 * q], nh[e][2 * q + 1]),
                 make_float2(nl[e][2 * q], nl[e][2 * q + 1]));
      lap[2 * q] = df::Acc{a.s.x, a.c.x};
      lap[2 * q + 1] = df::Acc{a.s.y, a.c.y};
    }
  } else {
#pragma unroll
    for (int e = 0; e < EC; ++e)
#pragma unroll
      for (int j = 0; j < K; ++j) df::fma(lap[j], vh[e], vl[e], nh[e][j], nl[e][j]);
  }
}

// r = b - (P x + tau o lap) at the pixel, normalised pairs; getp(q) gives the (hi, lo) of the
// packed lower-triangle entry q of the pixel block.  false: a non-finite result.
template <int K, typename GetP>
__device__ __forceinline__ bool df_finish(const df::Acc (&lap)[K], const float (&xh)[K],
                                          const float (&xl)[K], GetP&& getp,
                                          const float* tau_h, const float* tau_l,
                                          const float (&bh)[K], const float (&bl)[K],
                                          float (&rh)[K], float (&rl)[K]) {
  bool ok = true;
  if constexpr (K % 2 == 0) {
    // output pairs (2q, 2q + 1): sum over b of P_{2q+u, b} x_b, then tau o lap, then b - g
#pragma unroll
    for (int q = 0; q < K / 2; ++q) {
      df::Acc2 g = df::zero2();
#pragma unroll
      for (int b = 0; b < K; ++b) {
        const int a0 = 2 * q, a1 = 2 * q + 1;
        const int q0 = a0 >= b ? a0 * (a0 + 1) / 2 + b : b * (b + 1) / 2 + a0;
        const int q1 = a1 >= b ? a1 * (a1 + 1) / 2 + b : b * (b + 1) / 2 + a1;
        float p0h, p0l, p1h, p1l;
        getp(q0, p0h, p0l);
        getp(q1, p1h, p1l);
        df::fma2(g, make_float2(p0h, p1h), make_float2(p0l, p1l), make_float2(xh[b], xh[b]),
                 make_float2(xl[b], xl[b]));
      }
      float2 lh, ll;
      df::norm2(df::Acc2{make_float2(lap[2 * q].s, lap[2 * q + 1].s),
                         make_float2(lap[2 * q].c, lap[2 * q + 1].c)},
                lh, ll);
      df::fma2(g, make_float2(tau_h[2 * q], tau_h[2 * q + 1]),
               make_float2(tau_l[2 * q], tau_l[2 * q + 1]), lh, ll);
      float2 r2h, r2l;
      df::sub_from2(make_float2(bh[2 * q], bh[2 * q + 1]), make_float2(bl[2 * q], bl[2 * q + 1]),
                    g, r2h, r2l);
      rh[2 * q] = r2h.x;
      rh[2 * q + 1] = r2h.y;
      rl[2 * q] = r2l.x;
      rl[2 * q + 1] = r2l.y;
    }
  } else {
    df::Acc g[K];
#pragma unroll
    for (int j = 0; j < K; ++j) g[j] = df::zero();
#pragma unroll
    for (int a = 0; a < K; ++a) {
#pragma unroll
      for (int b = 0; b <= a; ++b) {
        float ph, pl;
        getp(a * (a + 1) / 2 + b, ph, pl);
        df::fma(g[a], ph, pl, xh[b], xl[b]);
        if (b != a) df::fma(g[b], ph, pl, xh[a], xl[a]);
      }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
      float lh, ll;
      df::norm(lap[j], lh, ll);
      df::fma(g[j], tau_h[j], tau_l[j], lh, ll);
      df::sub_from(bh[j], bl[j], g[j], rh[j], rl[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < K; ++j) ok &= isfinite(rh[j]) && isfinite(rl[j]);
  return ok;
}

// r = b - G x at pixel i of one column in double-float; xh, xl: the pixel's own split x;
// tile: the split x of the tile [base, base + tw) (in-tile neighbours), X: the column's FP64
// vector (out-of-tile neighbours), bh, bl: the split b.  false: recompute in FP64.
template <int K, int E>
__device__ __forceinline__ bool pixel_residual_df(const OpData& op, const float* tau_h,
                                                  const float* tau_l, const DfTile<K>& tile,
                                                  int64_t base, uint32_t tw, const double* X,
                                                  int64_t ldu,
                                                  int64_t i, const float (&xh)[K],
                                                  const float (&xl)[K], const float (&bh)[K],
                                                  const float (&bl)[K], float (&rh)[K],
                                                  float (&rl)[K]) {
  constexpr int NB = K * (K + 1) / 2;
  constexpr int EC = E > 0 ? E : 4;
  const int64_t ld = op.ld;
  const int Er = E > 0 ? E : op.E;
  bool ok = true;
  df::Acc lap[K];
#pragma unroll
  for (int j = 0; j < K; ++j) lap[j] = df::zero();
  for (int e0 = 0; e0 < Er; e0 += EC) {
    float nh[EC][K], nl[EC][K], vh[EC], vl[EC];
#pragma unroll
    for (int t = 0; t < EC; ++t) {
      const int e = E > 0 ? t : min(e0 + t, Er - 1);
      const int64_t c = __ldg(op.ell_col + (size_t)e * ld + i);
      vh[t] = __ldg(op.val_hl + (size_t)e * ld + i);
      vl[t] = __ldg(op.val_hl + (size_t)(Er + e) * ld + i);
      if (E == 0 && e0 + t >= Er) vh[t] = vl[t] = 0.f;
      const uint32_t loc = (uint32_t)(c - base);
      if (loc < tw) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
          nh[t][j] = tile.h[j][loc];
          nl[t][j] = tile.l[j][loc];
        }
      } else {
#pragma unroll
        for (int j = 0; j < K; ++j) ok &= df::split(X[(size_t)j * ldu + c], nh[t][j], nl[t][j]);
      }
    }
    df_stencil<K, EC>(lap, vh, vl, nh, nl);
  }
  ok &= df_finish<K>(lap, xh, xl,
                     [&](int q, float& ph, float& pl) {
                       ph = __ldg(op.blk_hl + (size_t)q * ld + i);
                       pl = __ldg(op.blk_hl + (size_t)(NB + q) * ld + i);
                     },
                     tau_h, tau_l, bh, bl, rh, rl);
  return ok;
}

// The same pixel in FP64 from the FP64 copies (the fallback), split into (rh, rl).
template <int K, int E, int NV>
__device__ __forceinline__ void pixel_residual_f64(const OpData& op,
                                                   const CtaShared<double, NV>& sh,
                                                   const double* X, const double* B,
                                                   int64_t ldu, int64_t i, bool with_op,
                                                   float (&rh)[K], float (&rl)[K]) {
  double gx[K];
#pragma unroll
  for (int j = 0; j < K; ++j) gx[j] = 0.0;
  if (with_op) {
    double xi[K];
#pragma unroll
    for (int j = 0; j < K; ++j) xi[j] = X[(size_t)j * ldu + i];
    apply_pixel_blk64<K, E, double, NV>(op, sh, X, ldu, i, xi, gx);
  }
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const double r = B[(size_t)j * ldu + i] - gx[j];
    rh[j] = float(r);
    rl[j] = float(r - double(rh[j]));
  }
}

// ---------------------------------------------------------------------------------------------
// residual (mixed precision, double-float): r = B - G X, r_in = fl32(r), d = 0, z = P^{-1} r_in;
// partial ||r||^2, ||B||^2, r . z, r . r; the last CTA decides (after_residual)
// ---------------------------------------------------------------------------------------------
template <int K, int M, int E>
__global__ void __launch_bounds__(TILE_PX, 2)
k_residual_df(const SysDesc* __restrict__ descs, const CtaRef* __restrict__ ctas, Control* ctl) {
  __shared__ CtaShared<double, 4> sh;   // FP64 tau for the fallback; per-warp sums
  __shared__ float tau_h[8], tau_l[8];
  __shared__ DfTile<K> tile;
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
  if (threadIdx.x < 8) {
    const int j = threadIdx.x;
    tau_h[j] = j < K ? op.tau_hl[0][j] : 0.f;
    tau_l[j] = j < K ? op.tau_hl[1][j] : 0.f;
  }
  stage_operator<double, 4>(op, K, sh);
  zero_wacc<double, 4>(sh, R);
  if (!__syncthreads_or(act)) return;

  const int64_t ld = op.ld, ldu = op.ldu, n = op.n;
  const bool prec = ctl->precond == SYLV_PRECOND_BLOCK_JACOBI;
  const bool x0_zero = ctl->x0_zero != 0;
  const int t = threadIdx.x;
  const uint32_t tw = blockDim.x;   // tile width of the plan (128 or TILE_PX)
  for (int tile_i = cr.slot; tile_i < sd.ntiles; tile_i += sd.nslots[2]) {
    const int64_t base = (int64_t)tile_i * tw;
    const int64_t i0 = base + t;
    const bool valid = i0 < n;
    const int64_t i = valid ? i0 : 0;
    BlockChol<K, float> f;
    if (prec) load_factor32<K>(op, i, f);
    for (int r = 0; r < R; ++r) {
      if (!sh.act[r]) continue;
      const bool with_op = !(x0_zero && sh.aux[r] == PH_START);   // X = 0: r = B
      const size_t off = (size_t)r * K * ld, offu = (size_t)r * K * ldu;
      const double* X = sd.X + offu;
      const double* B = sd.B + offu;
      float rh[K], rl[K], bh[K], bl[K], xh[K], xl[K];
      bool ok = true;
#pragma unroll
      for (int j = 0; j < K; ++j) ok &= df::split(B[(size_t)j * ldu + i], bh[j], bl[j]);
      if (with_op) {
        // the pixel's own x, split once and shared with the tile's stencils
        __syncthreads();   // the previous column's reads of the tile are done
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const bool okj = df::split(X[(size_t)j * ldu + i], xh[j], xl[j]);
          ok &= okj;
          tile.h[j][t] = okj ? xh[j] : __int_as_float(0x7fc00000);   // NaN: not split
          tile.l[j][t] = xl[j];
        }
        __syncthreads();
        ok &= pixel_residual_df<K, E>(op, tau_h, tau_l, tile, base, tw, X, ldu, i, xh, xl, bh,
                                      bl, rh, rl);
      } else {
#pragma unroll
        for (int j = 0; j < K; ++j) {
          rh[j] = bh[j];
          rl[j] = bl[j];
        }
      }
      if (!ok && valid) pixel_residual_f64<K, E, 4>(op, sh, X, B, ldu, i, with_op, rh, rl);
      float rr64 = 0.f, bb = 0.f, rz = 0.f, rr = 0.f;   // (FP32 partials, FP64 across warps)
      if (valid) {
        float ri[K], zi[K];
        float rr_px = 0.f, bb_px = 0.f;
#pragma unroll
        for (int j = 0; j < K; ++j) {
          ri[j] = __fadd_rn(rh[j], rl[j]);
          rr_px = fmaf(rh[j], rh[j], fmaf(2.f * rh[j], rl[j], rr_px));
          bb_px = fmaf(bh[j], bh[j], bb_px);
        }
        rr64 = rr_px;
        if (sh.aux[r] == PH_START) bb = bb_px;   // ||B||^2: first residual only
        {
          float* rv = (float*)sd.vr + off;
          float* dv = (float*)sd.vd + off;
          float* zv = (float*)sd.vz + off;
          if (prec) {
            block_solve<K, float>(f, ri, zi);
          } else {
#pragma unroll
            for (int j = 0; j < K; ++j) zi[j] = ri[j];
          }
          float rzt = 0.f, rrt = 0.f;   // products in the inner type, like the inner kernels
#pragma unroll
          for (int j = 0; j < K; ++j) {
            rv[(size_t)j * ld + i] = ri[j];
            dv[(size_t)j * ld + i] = 0.f;
            zv[(size_t)j * ld + i] = zi[j];
            rzt += ri[j] * zi[j];
            rrt += ri[j] * ri[j];
          }
          rz = rzt;
          rr = rrt;
        }
      }
      const float v[4] = {rr64, bb, rz, rr};
      warp_accumulate_f32<double, 4>(sh, r, v);
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
// the same residual with bulk-copy staging (the layout of k_residual_tma: X and B of the tile as
// the caller's FP64 rows, the pixel blocks and ELL values as FP32 pairs, the ELL columns, the
// preconditioner's scaling and factor), warp-specialised: one producer warp fills a two-stage
// ring, eight consumer warps compute.  Each thread splits every x it reads where it reads it:
// its own and its in-tile neighbours' from the stage, the others from the caller's X.  The
// in-tile splits are done twice (once per reader), but the consumer warps never wait for one
// another, so they drift apart and hide each other's latency (a shared buffer of split values
// needed a barrier per unit among them: same time on one column, 151 against 173 ms per
// 8-column solve of 50M pixels).  Same conditions as the FP64 staged kernel: whole tiles, an
// even ldu, 16-byte aligned X and B.
// ---------------------------------------------------------------------------------------------
template <int K, int M, int E>
__global__ void __launch_bounds__(tma::WS_THREADS, 1)
k_residual_tma_df(const SysDesc* __restrict__ descs, const CtaRef* __restrict__ ctas,
                  Control* ctl) {
  using namespace tma;
  using L = ResidLayout<K, E>;
  constexpr int NB = L::NB;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ CtaShared<double, 4> sh;
  __shared__ __align__(8) PipeShared ps;
  __shared__ float tau_h[8], tau_l[8];
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
  if (threadIdx.x < 8) {
    const int j = threadIdx.x;
    tau_h[j] = j < K ? op.tau_hl[0][j] : 0.f;
    tau_l[j] = j < K ? op.tau_hl[1][j] : 0.f;
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
      const uint32_t bytes = K * row8 + (noop ? 0u : K * row8 + NB * row8 + E * (row8 + row4)) +
                             (prec ? K * row4 + L::NB2 * row4 : 0u);
      if (lane == 0) {
        fence_proxy_async();
        mbar_expect_tx(&ps.full[st], bytes);
      }
      __syncwarp();
      const size_t uoff = (size_t)r * K * ldu;
      // rows: B (K, FP64), X (K, FP64), pixel blocks (2 NB, FP32 pairs), ELL values (2 E,
      // FP32 pairs), ELL columns (E), scaling (K), factor (NB2)
      constexpr int NROWS = 2 * K + 2 * NB + 2 * E + E + K + L::NB2;
      for (int q = lane; q < NROWS; q += 32) {
        const void* src = nullptr;
        void* dst = nullptr;
        uint32_t nbytes = row8;
        int x = q;
        if (x < K) {
          src = sd.B + uoff + (size_t)x * ldu + base;
          dst = stage + L::B + (size_t)x * row8;
        } else if ((x -= K) < K) {
          if (!noop) src = sd.X + uoff + (size_t)x * ldu + base;
          dst = stage + L::X + (size_t)x * row8;
        } else if ((x -= K) < 2 * NB) {
          if (!noop) src = op.blk_hl + (size_t)x * ld + base;
          dst = stage + L::BLK + (size_t)x * row4;
          nbytes = row4;
        } else if ((x -= 2 * NB) < 2 * E) {
          if (!noop) src = op.val_hl + (size_t)x * ld + base;
          dst = stage + L::VAL + (size_t)x * row4;
          nbytes = row4;
        } else if ((x -= 2 * E) < E) {
          if (!noop) src = op.ell_col + (size_t)x * ld + base;
          dst = stage + L::COL + (size_t)x * row4;
          nbytes = row4;
        } else if ((x -= E) < K) {
          if (prec) src = op.fs32 + (size_t)x * ld + base;
          dst = stage + L::FS + (size_t)x * row4;
          nbytes = row4;
        } else {
          x -= K;
          if (prec) src = op.fl16 + (size_t)x * ld + base;
          dst = stage + L::FL + (size_t)x * row4;
          nbytes = row4;
        }
        if (src) bulk_load(dst, src, nbytes, &ps.full[st]);
      }
    }, pipe_budget(ctl));
  } else {
    const int t = threadIdx.x;
    // ||r||^2, ||B||^2, r . z, r . r over this thread's units of one column: sums of FP32
    // products in FP32 (a stopping test needs a few digits; the sums of squares cannot cancel),
    // FP64 across warps and CTAs
    float a_rr64 = 0.f, a_bb = 0.f, a_rz = 0.f, a_rr = 0.f;
    for (int u = 0; u < U.n; ++u) {
      const int st = u % NSTAGE;
      if (!mbar_wait_bounded(&ps.full[st], (u / NSTAGE) & 1, pipe_budget(ctl)) || ps.bad) {
        ps.bad = 1;
        break;
      }
      const int tile = cr.slot + (u / U.nact) * sd.nslots[3];
      const int r = ps.cols[u % U.nact];
      const bool with_op = !(x0_zero && sh.aux[r] == PH_START);
      const int64_t base = (int64_t)tile * TILE_PX;
      const int64_t i = base + t;
      const unsigned char* stage = dsm + (size_t)st * L::STAGE_BYTES;
      const double* sx = reinterpret_cast<const double*>(stage + L::X);
      const double* sb = reinterpret_cast<const double*>(stage + L::B);
      const float* sph = reinterpret_cast<const float*>(stage + L::BLK);
      const float* spl = sph + (size_t)NB * TILE_PX;
      const float* svh = reinterpret_cast<const float*>(stage + L::VAL);
      const float* svl = svh + (size_t)E * TILE_PX;
      const int32_t* scol = reinterpret_cast<const int32_t*>(stage + L::COL);
      const size_t uoff = (size_t)r * K * ldu, off = (size_t)r * K * ld;
      const double* Xg = sd.X + uoff;
      float rh[K], rl[K], bh[K], bl[K];
      bool ok = true;
#pragma unroll
      for (int j = 0; j < K; ++j) ok &= df::split(sb[j * TILE_PX + t], bh[j], bl[j]);
      if (with_op) {
        float xh[K], xl[K];
#pragma unroll
        for (int j = 0; j < K; ++j) ok &= df::split(sx[j * TILE_PX + t], xh[j], xl[j]);
        // stencil: every neighbour's x split where it is read, in-tile ones from the stage,
        // the others from the caller's X (generic pointers: no branch, no barrier between the
        // consumer warps)
        df::Acc lap[K];
#pragma unroll
        for (int j = 0; j < K; ++j) lap[j] = df::zero();
        float nh[E][K], nl[E][K], vh[E], vl[E];
        const double* src[E];
        int64_t stride[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int64_t c = scol[e * TILE_PX + t];
          vh[e] = svh[e * TILE_PX + t];
          vl[e] = svl[e * TILE_PX + t];
          const uint32_t loc = (uint32_t)(c - base);
          const bool in = loc < (uint32_t)TILE_PX;
          src[e] = in ? sx + loc : Xg + c;
          stride[e] = in ? (int64_t)TILE_PX : ldu;
        }
#pragma unroll
        for (int e = 0; e < E; ++e)
#pragma unroll
          for (int j = 0; j < K; ++j) ok &= df::split(src[e][j * stride[e]], nh[e][j], nl[e][j]);
        df_stencil<K, E>(lap, vh, vl, nh, nl);
        ok &= df_finish<K>(lap, xh, xl,
                           [&](int q, float& ph, float& pl) {
                             ph = sph[q * TILE_PX + t];
                             pl = spl[q * TILE_PX + t];
                           },
                           tau_h, tau_l, bh, bl, rh, rl);
      } else {
#pragma unroll
        for (int j = 0; j < K; ++j) {
          rh[j] = bh[j];
          rl[j] = bl[j];
        }
      }
      if (!ok && i < n)
        pixel_residual_f64<K, E, 4>(op, sh, Xg, sd.B + uoff, ldu, i, with_op, rh, rl);
      float ri[K], zi[K];
      float rr_px = 0.f, bb_px = 0.f;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        ri[j] = __fadd_rn(rh[j], rl[j]);
        rr_px = fmaf(rh[j], rh[j], fmaf(2.f * rh[j], rl[j], rr_px));
        bb_px = fmaf(bh[j], bh[j], bb_px);
      }
      if (prec) {
        BlockChol<K, float> f;
        const float* sfs = reinterpret_cast<const float*>(stage + L::FS);
        const __half2* sfl = reinterpret_cast<const __half2*>(stage + L::FL);
#pragma unroll
        for (int x = 0; x < K; ++x) f.s[x] = sfs[x * TILE_PX + t];
#pragma unroll
        for (int x = 0; x < NB; x += 2) {
          const float2 w2 = __half22float2(sfl[(x / 2) * TILE_PX + t]);
          f.l[x] = w2.x;
          if (x + 1 < NB) f.l[x + 1] = w2.y;
        }
        block_solve<K, float>(f, ri, zi);
      } else {
#pragma unroll
        for (int j = 0; j < K; ++j) zi[j] = ri[j];
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&ps.empty[st]);
      consumed = u + 1;
      float rr64 = 0.f, bb = 0.f;
      float rzt = 0.f, rrt = 0.f;   // products in the inner type, like the inner kernels
      if (i < n) {
        rr64 = rr_px;
        if (sh.aux[r] == PH_START) bb = bb_px;   // ||B||^2: first residual only
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
      }
      a_rr64 += rr64;
      a_bb += bb;
      a_rz += rzt;
      a_rr += rrt;
      if (U.nact > 1 || u + 1 == U.n) {
        const float v4[4] = {a_rr64, a_bb, a_rz, a_rr};
        warp_accumulate_f32<double, 4>(sh, r, v4);
        a_rr64 = a_bb = a_rz = a_rr = 0.f;
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
// stand-alone residual R = B - G X (sylv_residual): the same double-float arithmetic, written
// in FP64 as h + l
// ---------------------------------------------------------------------------------------------
template <int K, int M, int E>
__global__ void __launch_bounds__(TILE_PX, 2)
k_residual_out(OpData op, const double* __restrict__ B, const double* __restrict__ X, int R,
               double* __restrict__ Rout, int use_df) {
  __shared__ CtaShared<double, 1> sh;
  __shared__ float tau_h[8], tau_l[8];
  __shared__ DfTile<K> tile;
  if (threadIdx.x < 8) {
    const int j = threadIdx.x;
    tau_h[j] = j < K ? op.tau_hl[0][j] : 0.f;
    tau_l[j] = j < K ? op.tau_hl[1][j] : 0.f;
  }
  stage_operator<double, 1>(op, K, sh);
  const int64_t ldu = op.ldu, n = op.n;
  const int t = threadIdx.x;
  const int ntiles = (int)((n + TILE_PX - 1) / TILE_PX);
  for (int tile_i = blockIdx.x; tile_i < ntiles; tile_i += gridDim.x) {
    const int64_t base = (int64_t)tile_i * TILE_PX;
    const bool valid = base + t < n;
    const int64_t i = valid ? base + t : 0;
    for (int r = 0; r < R; ++r) {
      const size_t offu = (size_t)r * K * ldu;
      const double* Xr = X + offu;
      const double* Br = B + offu;
      float rh[K], rl[K], bh[K], bl[K], xh[K], xl[K];
      bool ok = use_df != 0;
#pragma unroll
      for (int j = 0; j < K; ++j) ok &= df::split(Br[(size_t)j * ldu + i], bh[j], bl[j]);
      __syncthreads();
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const bool okj = df::split(Xr[(size_t)j * ldu + i], xh[j], xl[j]);
        ok &= okj;
        tile.h[j][t] = okj ? xh[j] : __int_as_float(0x7fc00000);
        tile.l[j][t] = xl[j];
      }
      __syncthreads();
      if (use_df)
        ok &= pixel_residual_df<K, E>(op, tau_h, tau_l, tile, base, TILE_PX, Xr, ldu, i, xh, xl,
                                      bh, bl, rh, rl);
      if (!ok && valid) pixel_residual_f64<K, E, 1>(op, sh, Xr, Br, ldu, i, true, rh, rl);
      if (valid) {
#pragma unroll
        for (int j = 0; j < K; ++j)
          Rout[offu + (size_t)j * ldu + i] = double(rh[j]) + double(rl[j]);
      }
    }
  }
}

}  // namespace sylv
