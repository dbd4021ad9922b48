// Stand-alone staged FP32 operator apply for three or more right-hand sides.
//
// Y = G X (Sec. 3.1, eq. block-vector-mapping-matvec with the stencil of Algorithm 1) for the
// caller's FP32 columns, as k_apply_tma (pcg_tma.cuh) computes it, with a tile's operator rows
// staged once for all its columns instead of once per column.
#pragma once

#include "pcg_tma.cuh"

namespace sylv {
namespace tma {

// Several right-hand sides (three or more): a tile's operator rows (D, ELL values, diagonal, ELL
// columns) go to one of NST_X operator slots, once per tile; each (tile, column) unit's x rows
// go through a ring of NST_X vector stages.  So the operator rows are staged once per tile,
// not once per column (8 columns: 3.3 -> 3.9 TB/s); with one column the single ring above is
// faster (5.4 against 4.8 TB/s).
template <int K, int M, int E>
struct ApplyXOpsLayout {
  static constexpr int D = 0, VAL = M, DIAG = M + E, COL = M + E + 1;   // operator slot rows
  static constexpr int OP_ROWS = M + 2 * E + 1;
  static constexpr int OP_BYTES = OP_ROWS * TILE_PX * 4;
  static constexpr int VEC_BYTES = K * TILE_PX * 4;                      // x rows of a unit
  static constexpr int SMEM = NST_X * (OP_BYTES + VEC_BYTES);
};

template <int K, int M, int E>
__global__ void __launch_bounds__(WS_THREADS, 3)
k_apply_tma_ops(OpData op, const float* __restrict__ X, float* __restrict__ Y, int R,
            unsigned int* ctr) {
  // ctr[0]: timeout flag; ctr[1]: next tile; ctr[2]: CTAs done (both zero between launches).
  // Tiles are taken from ctr[1] one ahead, so CTAs on faster SMs take more of them; there are
  // no partial sums here, so how the tiles are split changes nothing in the result.  A tile
  // index >= ntiles stops the consumers.  A tile's columns run back to back.
  using L = ApplyXOpsLayout<K, M, E>;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ CtaShared<float, 1> sh;
  __shared__ __align__(8) PipeShared ps;                 // vector ring
  __shared__ __align__(8) uint64_t op_full[NST_X], op_empty[NST_X];
  __shared__ int utile[NST_X], ucol[NST_X];
  __shared__ int op_issued, op_started;
  unsigned char* opbuf = dsm;                                       // NST_X operator slots
  unsigned char* vecbuf = dsm + (size_t)NST_X * L::OP_BYTES;        // NST_X vector stages
  stage_operator<float, 1>(op, K, sh);
  if (threadIdx.x == 0) {
    pipe_init<NST_X>(ps);
    for (int q = 0; q < NST_X; ++q) {
      mbar_init(&op_full[q], 1);
      mbar_init(&op_empty[q], NCONS);
    }
    op_issued = 0;
    op_started = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const int64_t ldu = op.ldu;
  const int ntiles = (int)(op.n / TILE_PX);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t rowb = TILE_PX * 4;
  int consumed = 0;
  if (warp == NCONS) {
    int next = 0, u = 0, lt = 0;
    if (lane == 0) next = (int)atomicAdd(ctr + 1, 1u);
    bool stop = false;
    while (!stop) {
      const int tile = __shfl_sync(0xffffffffu, next, 0);
      const bool end = tile >= ntiles;
      if (!end && lane == 0) next = (int)atomicAdd(ctr + 1, 1u);
      const int64_t base = (int64_t)tile * TILE_PX;
      if (!end) {   // the tile's operator rows into slot lt % NST_X, once released
        const int os = lt % NST_X;
        if (lt >= NST_X) {
          bool ok = true;
          if (lane == 0) ok = mbar_wait_bounded(&op_empty[os], ((lt / NST_X) - 1) & 1);
          ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
          if (!ok || ps.bad) {
            if (lane == 0) ps.bad = 1;
            break;
          }
        }
        float* slot = reinterpret_cast<float*>(opbuf + (size_t)os * L::OP_BYTES);
        if (lane == 0) {
          fence_proxy_async();
          mbar_expect_tx(&op_full[os], (uint32_t)L::OP_ROWS * rowb);
        }
        __syncwarp();
        for (int q = lane; q < L::OP_ROWS; q += 32) {
          const void* src;
          if (q < L::VAL) src = op.D32 + (size_t)(q - L::D) * op.ld + base;
          else if (q < L::DIAG) src = op.ell_val32 + (size_t)(q - L::VAL) * op.ld + base;
          else if (q == L::DIAG) src = op.diag32 + base;
          else src = op.ell_col + (size_t)(q - L::COL) * op.ld + base;
          bulk_load(slot + (size_t)q * TILE_PX, src, rowb, &op_full[os]);
        }
        if (lane == 0) op_issued = lt + 1;
      }
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
          float* stage = reinterpret_cast<float*>(vecbuf + (size_t)st * L::VEC_BYTES);
          if (lane == 0) {
            fence_proxy_async();
            mbar_expect_tx(&ps.full[st], (uint32_t)K * rowb);
          }
          __syncwarp();
          const size_t xoff = (size_t)r * K * ldu;
          for (int q = lane; q < K; q += 32)
            bulk_load(stage + (size_t)q * TILE_PX, X + xoff + (size_t)q * ldu + base, rowb,
                      &ps.full[st]);
        }
        if (lane == 0) ps.issued = u + 1;
      }
      ++lt;
      if (end) stop = true;
    }
  } else {
    const int t = threadIdx.x;
    int lt = 0;
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
      const int os = lt % NST_X;
      if (r == 0) {   // first column of a tile: its operator rows
        if (!mbar_wait_bounded(&op_full[os], (lt / NST_X) & 1) || ps.bad) {
          ps.bad = 1;
          break;
        }
        if (t == 0) op_started = lt + 1;
      }
      const int64_t base = (int64_t)tile * TILE_PX;
      const int64_t i = base + t;
      const float* stage = reinterpret_cast<const float*>(vecbuf + (size_t)st * L::VEC_BYTES);
      const float* slot = reinterpret_cast<const float*>(opbuf + (size_t)os * L::OP_BYTES);
      const int32_t* scol = reinterpret_cast<const int32_t*>(slot + (size_t)L::COL * TILE_PX);
      const size_t xoff = (size_t)r * K * ldu;
      float xi[K], lap[K];
#pragma unroll
      for (int j = 0; j < K; ++j) xi[j] = stage[j * TILE_PX + t];
      const float dg = slot[L::DIAG * TILE_PX + t];
#pragma unroll
      for (int j = 0; j < K; ++j) lap[j] = dg * xi[j];
      const float* src[E];
      int64_t stride[E];
      float v[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int64_t c = scol[e * TILE_PX + t];
        v[e] = slot[(L::VAL + e) * TILE_PX + t];
        const uint32_t loc = (uint32_t)(c - base);
        const bool in_tile = loc < (uint32_t)TILE_PX;
        src[e] = in_tile ? stage + loc : X + xoff + c;
        stride[e] = in_tile ? (int64_t)TILE_PX : ldu;
      }
      float nb[E][K];
#pragma unroll
      for (int e = 0; e < E; ++e)
#pragma unroll
        for (int j = 0; j < K; ++j) nb[e][j] = src[e][j * stride[e]];
      float w[K];
      pixel_operator_ws<K, M, E>(sh, slot + (size_t)L::D * TILE_PX + t, xi, lap, v, nb, w);
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&ps.empty[st]);
        if (r == R - 1) mbar_arrive(&op_empty[os]);   // the tile's last column: slot released
      }
      if (r == R - 1) ++lt;
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
      for (int q = op_started; q < op_issued; ++q)
        mbar_wait_bounded(&op_full[q % NST_X], (q / NST_X) & 1);
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
