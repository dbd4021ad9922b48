// Explicit instantiation of the iteration kernels with inner type float.
#include "pcg_kernels.cuh"

namespace sylv {

template <>
cudaError_t launch_inner_apply<float>(int k, int ntiles, int block, const SysDesc* d,
                                      const CtaRef* t, Control* c, cudaStream_t s) {
  return launch_inner_apply_impl<float>(k, ntiles, block, d, t, c, s);
}
template <>
cudaError_t launch_inner_update<float>(int k, int ntiles, int block, const SysDesc* d,
                                       const CtaRef* t, Control* c, cudaStream_t s) {
  return launch_inner_update_impl<float>(k, ntiles, block, d, t, c, s);
}
template <>
cudaError_t launch_residual<float>(int k, int ntiles, int block, const SysDesc* d,
                                   const CtaRef* t, Control* c, cudaStream_t s) {
  return launch_residual_impl<float>(k, ntiles, block, d, t, c, s);
}
template <>
cudaError_t launch_update_x<float>(int k, int ntiles, int block, const SysDesc* d,
                                   const CtaRef* t, cudaStream_t s) {
  return launch_update_x_impl<float>(k, ntiles, block, d, t, s);
}

template <>
int occupancy<float>(int k, int block) {
  return occupancy_impl<float>(k, block);
}

}  // namespace sylv
