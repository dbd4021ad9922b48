// Explicit instantiation of the iteration kernels with inner type double.
#include "pcg_kernels.cuh"

namespace sylv {

template <>
cudaError_t launch_inner_apply<double>(int k, int m, int e, int variant, int ncta, int block,
                                       const SysDesc* d, const CtaRef* c, Control* ctl,
                                       cudaStream_t s) {
  (void)variant;
  return launch_inner_apply_impl<double>(k, m, e, ncta, block, d, c, ctl, s);
}
template <>
cudaError_t launch_inner_update<double>(int k, int m, int e, int variant, int ncta, int block,
                                        const SysDesc* d, const CtaRef* c, Control* ctl,
                                        cudaStream_t s) {
  (void)variant;
  return launch_inner_update_impl<double>(k, m, e, ncta, block, d, c, ctl, s);
}
template <>
cudaError_t launch_residual<double>(int k, int m, int e, int ncta, int block, const SysDesc* d,
                                  const CtaRef* c, Control* ctl, cudaStream_t s) {
  return launch_residual_impl<double>(k, m, e, ncta, block, d, c, ctl, s);
}
template <>
cudaError_t launch_update_x<double>(int k, int ncta, int block, const SysDesc* d, const CtaRef* c,
                                  cudaStream_t s) {
  return launch_update_x_impl<double>(k, ncta, block, d, c, s);
}
template <>
int occupancy<double>(int kind, int k, int m, int e, int variant, int block) {
  (void)variant;
  return occupancy_impl<double>(kind == 3 ? 2 : kind, k, m, e, block);
}

}  // namespace sylv
