// Iteration kernels with inner type float: the generic kernels and the bulk-copy staged ones.
#include <cstdlib>
#include <cstring>

#include "apply_ops.cuh"
#include "pcg_mc.cuh"
#include "resid_df.cuh"

namespace sylv {

bool tma_available(int k, int m, int e) { return special_shape(k, m, e); }

namespace tma {

// Chunk-closing kernel of the staged pair in modes 1 and 2 (launched over the update kernel's
// CTA list; the slot-0 CTA of each system works): the state change of the last update of a
// chunk, so that the host's poll and the next chunk see it.
__global__ void __launch_bounds__(TILE_PX)
k_inner_close(const SysDesc* __restrict__ descs, const CtaRef* __restrict__ ctas, Control* ctl) {
  __shared__ ColState cst[CS_RMAX];
  __shared__ int want[RMAX];
  __shared__ double red[32 * 2];
  __shared__ double tot[CS_RMAX][NPART];
  const CtaRef cr = ctas[blockIdx.x];
  if (cr.sys < 0 || cr.slot != 0) return;
  const SysDesc& sd = descs[cr.sys];
  const int R = sd.R;
  if (R > CS_RMAX) return;
  if (threadIdx.x < RMAX) {
    const int r = threadIdx.x;
    want[r] = 0;
    if (r < R) {
      cst[r] = sd.st[r];
      want[r] = cst[r].phase == PH_INNER;
    }
  }
  __syncthreads();
  sum_slots<2>(sd.partial2, sd.nslots[1], R, want, red, tot);
  if (threadIdx.x < R && want[threadIdx.x]) {
    const int r = threadIdx.x;
    after_update(cst[r], tot[r][0], tot[r][1], ctl, true);
    sd.st[r] = cst[r];
  }
}

}  // namespace tma

namespace {

template <int K, int M, int E>
size_t apply_tma_smem() {
  return (size_t)tma::NSTAGE * tma::ApplyLayout<K, M, E>::STAGE_BYTES;
}
template <int K, int M>
size_t update_tma_smem() {
  return (size_t)tma::NSTAGE * tma::UpdateLayout<K, M>::STAGE_BYTES;
}

template <int K, int M, int E>
cudaError_t apply_tma(int ncta, const SysDesc* d, const CtaRef* c, Control* ctl, int mode,
                      cudaStream_t s) {
  static bool attr = false;
  const size_t smem = apply_tma_smem<K, M, E>();
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tma::k_inner_apply_tma<K, M, E>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  tma::k_inner_apply_tma<K, M, E><<<ncta, tma::WS_THREADS, smem, s>>>(d, c, ctl, mode);
  return cudaGetLastError();
}

template <int K, int M>
cudaError_t update_tma(int ncta, const SysDesc* d, const CtaRef* c, Control* ctl, int mode,
                       cudaStream_t s) {
  static bool attr = false;
  const size_t smem = update_tma_smem<K, M>();
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tma::k_inner_update_tma<K, M>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  tma::k_inner_update_tma<K, M><<<ncta, tma::WS_THREADS, smem, s>>>(d, c, ctl, mode);
  return cudaGetLastError();
}

template <int K, int M, int E>
cudaError_t apply_mc(int ncta, const SysDesc* d, const CtaRef* c, Control* ctl, cudaStream_t s) {
  static bool attr = false;
  constexpr size_t smem = tma::mc_apply_smem<K, M, E>();
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tma::k_inner_apply_mc<K, M, E>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  tma::k_inner_apply_mc<K, M, E><<<ncta, tma::WS_THREADS, smem, s>>>(d, c, ctl);
  return cudaGetLastError();
}

template <int K, int M>
cudaError_t update_mc(int ncta, const SysDesc* d, const CtaRef* c, Control* ctl, cudaStream_t s) {
  static bool attr = false;
  constexpr size_t smem = tma::mc_update_smem<K>();
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tma::k_inner_update_mc<K, M>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  tma::k_inner_update_mc<K, M><<<ncta, tma::WS_THREADS, smem, s>>>(d, c, ctl);
  return cudaGetLastError();
}

template <int K, int M, int E>
int mc_occupancy(int kind) {
  int nb = 0;
  if (kind == 0) {
    constexpr size_t smem = tma::mc_apply_smem<K, M, E>();
    cudaFuncSetAttribute(tma::k_inner_apply_mc<K, M, E>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tma::k_inner_apply_mc<K, M, E>,
                                                  tma::WS_THREADS, smem);
  } else {
    constexpr size_t smem = tma::mc_update_smem<K>();
    cudaFuncSetAttribute(tma::k_inner_update_mc<K, M>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tma::k_inner_update_mc<K, M>,
                                                  tma::WS_THREADS, smem);
  }
  return nb < 1 ? 1 : nb;
}

template <int K, int M, int E>
int tma_occupancy(int kind) {
  int nb = 0;
  if (kind == 0) {
    cudaFuncSetAttribute(tma::k_inner_apply_tma<K, M, E>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)apply_tma_smem<K, M, E>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tma::k_inner_apply_tma<K, M, E>,
                                                  tma::WS_THREADS, apply_tma_smem<K, M, E>());
  } else {
    cudaFuncSetAttribute(tma::k_inner_update_tma<K, M>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)update_tma_smem<K, M>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tma::k_inner_update_tma<K, M>,
                                                  tma::WS_THREADS, update_tma_smem<K, M>());
  }
  return nb < 1 ? 1 : nb;
}

template <int K, int M, int E>
size_t residual_tma_smem() {
  return (size_t)tma::NSTAGE * tma::ResidLayout<K, E>::STAGE_BYTES;
}

template <int K, int M, int E>
cudaError_t residual_tma(int ncta, const SysDesc* d, const CtaRef* c, Control* ctl,
                         cudaStream_t s) {
  static bool attr = false;
  const size_t smem = residual_tma_smem<K, M, E>();
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tma::k_residual_tma<K, M, E>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  tma::k_residual_tma<K, M, E><<<ncta, tma::WS_THREADS, smem, s>>>(d, c, ctl);
  return cudaGetLastError();
}

template <int K, int M, int E>
int residual_tma_occupancy() {
  int nb = 0;
  cudaFuncSetAttribute(tma::k_residual_tma<K, M, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)residual_tma_smem<K, M, E>());
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tma::k_residual_tma<K, M, E>,
                                                tma::WS_THREADS, residual_tma_smem<K, M, E>());
  return nb < 1 ? 1 : nb;
}

// variant 0: one ring of whole stages (k_apply_tma); 1: operator slots once per tile and a
// ring of x rows (k_apply_tma_ops); 2: the multi-column kernel (k_apply_mc)
template <int K, int M, int E, int V>
cudaError_t apply_x_tma_impl(const OpData& op, const float* X, float* Y, int R, unsigned int* err,
                             cudaStream_t s) {
  static bool attr = false;
  static int grid = 0;
  const auto kern = V == 2 ? tma::k_apply_mc<K, M, E>
                           : (V == 1 ? tma::k_apply_tma_ops<K, M, E> : tma::k_apply_tma<K, M, E>);
  constexpr size_t ring = (size_t)tma::NST_X * tma::ApplyXLayout<K, M, E>::STAGE_BYTES;
  const size_t smem = V == 2 ? tma::mc_applyx_smem<K, M, E>()
                             : (V == 1 ? (size_t)tma::ApplyXOpsLayout<K, M, E>::SMEM : ring);
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0, dev = 0, nsm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, tma::WS_THREADS, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    grid = nsm * (occ < 1 ? 1 : occ);
    attr = true;
  }
  const int ntiles = (int)(op.n / TILE_PX);
  const int g = ntiles < grid ? ntiles : grid;
  kern<<<g, tma::WS_THREADS, smem, s>>>(op, X, Y, R, err);
  return cudaGetLastError();
}

// One or two columns: one ring of whole stages; three or more: the multi-column kernel
// (SYLV_APPLY_MANY=ops selects the kernel with operator slots and a ring of x rows instead).
const int g_apply_many = [] {
  const char* v = std::getenv("SYLV_APPLY_MANY");
  return (v && std::strcmp(v, "ops") == 0) ? 1 : 2;
}();

template <int K, int M, int E>
cudaError_t apply_x_tma(const OpData& op, const float* X, float* Y, int R, unsigned int* err,
                        cudaStream_t s) {
  if (R < 3) return apply_x_tma_impl<K, M, E, 0>(op, X, Y, R, err, s);
  return g_apply_many == 1 ? apply_x_tma_impl<K, M, E, 1>(op, X, Y, R, err, s)
                           : apply_x_tma_impl<K, M, E, 2>(op, X, Y, R, err, s);
}

}  // namespace

#define SYLV_TMA_APPLY_X_(K_, M_, E_) \
  if (k == K_ && m == M_ && e == E_) return apply_x_tma<K_, M_, E_>(op, X, Y, R, err, s);

// Staged stand-alone FP32 apply; cudaErrorNotSupported when the shape or the alignment does
// not allow it (the caller then uses the direct kernel).
cudaError_t launch_apply_staged(const OpData& op, const float* X, float* Y, int R,
                                unsigned int* err, cudaStream_t s) {
  const int k = op.k, m = op.m, e = op.E;
  const bool aligned = op.n > 0 && op.n % TILE_PX == 0 && op.ldu % 4 == 0 &&
                       ((uintptr_t)X & 15u) == 0 && ((uintptr_t)Y & 15u) == 0 && !op.has_w;
  if (aligned) {
    SYLV_SPECIAL_SHAPES(SYLV_TMA_APPLY_X_)
  }
  return cudaErrorNotSupported;
}

#define SYLV_TMA_APPLY_(K_, M_, E_)                                              \
  if (k == K_ && m == M_ && e == E_)                                             \
    return variant == 4 ? apply_mc<K_, M_, E_>(ncta, d, c, ctl, s)               \
                        : apply_tma<K_, M_, E_>(ncta, d, c, ctl, variant - 1, s);
#define SYLV_TMA_UPDATE_(K_, M_, E_)                                             \
  if (k == K_ && m == M_ && e == E_)                                             \
    return variant == 4 ? update_mc<K_, M_>(ncta, d, c, ctl, s)                  \
                        : update_tma<K_, M_>(ncta, d, c, ctl, variant - 1, s);
#define SYLV_TMA_OCC_(K_, M_, E_)                                                \
  if (k == K_ && m == M_ && e == E_)                                             \
    return variant == 2 ? mc_occupancy<K_, M_, E_>(kind) : tma_occupancy<K_, M_, E_>(kind);
#define SYLV_TMA_RESID_(K_, M_, E_) \
  if (k == K_ && m == M_ && e == E_) return residual_tma<K_, M_, E_>(ncta, d, c, ctl, s);
#define SYLV_TMA_RESID_OCC_(K_, M_, E_) \
  if (k == K_ && m == M_ && e == E_) return residual_tma_occupancy<K_, M_, E_>();

cudaError_t launch_residual_staged(int k, int m, int e, int ncta, const SysDesc* d,
                                   const CtaRef* c, Control* ctl, cudaStream_t s) {
  if (ncta <= 0) return cudaSuccess;
  SYLV_SPECIAL_SHAPES(SYLV_TMA_RESID_)
  return cudaErrorNotSupported;
}

template <>
cudaError_t launch_inner_apply<float>(int k, int m, int e, int variant, int ncta, int block,
                                      const SysDesc* d, const CtaRef* c, Control* ctl,
                                      cudaStream_t s) {
  if (ncta <= 0) return cudaSuccess;
  if (variant >= 1 && variant <= 4) {
    SYLV_SPECIAL_SHAPES(SYLV_TMA_APPLY_)
  }
  return launch_inner_apply_impl<float>(k, m, e, ncta, block, d, c, ctl, s);
}
template <>
cudaError_t launch_inner_update<float>(int k, int m, int e, int variant, int ncta, int block,
                                       const SysDesc* d, const CtaRef* c, Control* ctl,
                                       cudaStream_t s) {
  if (ncta <= 0) return cudaSuccess;
  if (variant >= 1 && variant <= 4) {
    SYLV_SPECIAL_SHAPES(SYLV_TMA_UPDATE_)
  }
  return launch_inner_update_impl<float>(k, m, e, ncta, block, d, c, ctl, s);
}
cudaError_t launch_residual_df(int k, int m, int e, int ncta, int block, const SysDesc* d,
                               const CtaRef* c, Control* ctl, cudaStream_t s) {
  if (ncta <= 0) return cudaSuccess;
#define CALL(K, M, E) k_residual_df<K, M, E><<<ncta, block, 0, s>>>(d, c, ctl)
  SYLV_DISPATCH_SHAPE(k, m, e)
#undef CALL
  return cudaGetLastError();
}

namespace {
template <int K, int M, int E>
size_t residual_tma_df_smem() {
  return (size_t)tma::NSTAGE * tma::ResidLayout<K, E>::STAGE_BYTES;
}

template <int K, int M, int E>
cudaError_t residual_tma_df(int ncta, const SysDesc* d, const CtaRef* c, Control* ctl,
                            cudaStream_t s) {
  static bool attr = false;
  const size_t smem = residual_tma_df_smem<K, M, E>();
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_residual_tma_df<K, M, E>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_residual_tma_df<K, M, E><<<ncta, tma::WS_THREADS, smem, s>>>(d, c, ctl);
  return cudaGetLastError();
}
}  // namespace

#define SYLV_TMA_RESID_DF_(K_, M_, E_) \
  if (k == K_ && m == M_ && e == E_) return residual_tma_df<K_, M_, E_>(ncta, d, c, ctl, s);

cudaError_t launch_residual_staged_df(int k, int m, int e, int ncta, const SysDesc* d,
                                      const CtaRef* c, Control* ctl, cudaStream_t s) {
  if (ncta <= 0) return cudaSuccess;
  SYLV_SPECIAL_SHAPES(SYLV_TMA_RESID_DF_)
  return cudaErrorNotSupported;
}

cudaError_t launch_residual_out(const OpData& op, const double* B, const double* X, int R,
                                double* Rout, int use_df, cudaStream_t s) {
  const int k = op.k, m = op.m, e = op.E;
  const int64_t ntiles = (op.n + TILE_PX - 1) / TILE_PX;
  const int grid = (int)(ntiles < 65536 ? ntiles : 65536);
#define CALL(K, M, E) \
  k_residual_out<K, M, E><<<grid, TILE_PX, 0, s>>>(op, B, X, R, Rout, use_df)
  SYLV_DISPATCH_SHAPE(k, m, e)
#undef CALL
  return cudaGetLastError();
}

template <>
cudaError_t launch_residual<float>(int k, int m, int e, int ncta, int block, const SysDesc* d,
                                   const CtaRef* c, Control* ctl, cudaStream_t s) {
  return launch_residual_impl<float>(k, m, e, ncta, block, d, c, ctl, s);
}
template <>
cudaError_t launch_update_x<float>(int k, int ncta, int block, const SysDesc* d, const CtaRef* c,
                                   cudaStream_t s) {
  return launch_update_x_impl<float>(k, ncta, block, d, c, s);
}
cudaError_t launch_inner_close(int ncta, const SysDesc* d, const CtaRef* c, Control* ctl,
                               cudaStream_t s) {
  if (ncta <= 0) return cudaSuccess;
  tma::k_inner_close<<<ncta, TILE_PX, 0, s>>>(d, c, ctl);
  return cudaGetLastError();
}

template <>
int occupancy<float>(int kind, int k, int m, int e, int variant, int block) {
  if (kind == 3) {
    SYLV_SPECIAL_SHAPES(SYLV_TMA_RESID_OCC_)
    kind = 2;
  }
  if (variant >= 1 && kind < 2) {
    SYLV_SPECIAL_SHAPES(SYLV_TMA_OCC_)
  }
  return occupancy_impl<float>(kind, k, m, e, block);
}

}  // namespace sylv
