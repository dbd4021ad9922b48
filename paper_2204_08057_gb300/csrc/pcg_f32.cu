// Explicit instantiation of the iteration kernels with inner type float.
#include "pcg_kernels.cuh"

namespace sylv {

template <>
cudaError_t launch_inner_apply<float>(int k, int m, int e, int ncta, int block, const SysDesc* d,
                                     const CtaRef* c, Control* ctl, cudaStream_t s) {
  return launch_inner_apply_impl<float>(k, m, e, ncta, block, d, c, ctl, s);
}
template <>
cudaError_t launch_inner_update<float>(int k, int m, int e, int ncta, int block,
                                      const SysDesc* d, const CtaRef* c, Control* ctl,
                                      cudaStream_t s) {
  return launch_inner_update_impl<float>(k, m, e, ncta, block, d, c, ctl, s);
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
template <>
int occupancy<float>(int k, int m, int e, int block) {
  return occupancy_impl<float>(k, m, e, block);
}

}  // namespace sylv
