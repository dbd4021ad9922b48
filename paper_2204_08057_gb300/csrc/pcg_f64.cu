// Explicit instantiation of the iteration kernels with inner type double.
#include "pcg_kernels.cuh"

namespace sylv {

template <>
cudaError_t launch_inner_apply<double>(int k, int ntiles, int block, const SysDesc* d,
                                      const CtaRef* t, Control* c, cudaStream_t s) {
  return launch_inner_apply_impl<double>(k, ntiles, block, d, t, c, s);
}
template <>
cudaError_t launch_inner_update<double>(int k, int ntiles, int block, const SysDesc* d,
                                       const CtaRef* t, Control* c, cudaStream_t s) {
  return launch_inner_update_impl<double>(k, ntiles, block, d, t, c, s);
}
template <>
cudaError_t launch_residual<double>(int k, int ntiles, int block, const SysDesc* d,
                                   const CtaRef* t, Control* c, cudaStream_t s) {
  return launch_residual_impl<double>(k, ntiles, block, d, t, c, s);
}
template <>
cudaError_t launch_update_x<double>(int k, int ntiles, int block, const SysDesc* d,
                                   const CtaRef* t, cudaStream_t s) {
  return launch_update_x_impl<double>(k, ntiles, block, d, t, s);
}

template <>
int occupancy<double>(int k, int block) {
  return occupancy_impl<double>(k, block);
}

}  // namespace sylv
