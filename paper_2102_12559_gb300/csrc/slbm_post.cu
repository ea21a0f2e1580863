// Instantiations of the post-step kernel (interface conversion + ghost images).
#include "slbm_post.cuh"

namespace slbm {
template <>
cudaError_t launch_post<float, float>(const Params<float>& p, float* f0, float* f1,
                                      const uint8_t* flag_old, const uint8_t* flag_new,
                                      const BcDev& bc, int images, const uint8_t* mask_in,
                                      uint8_t* tile_mask,
                                      cudaStream_t st) {
  return launch_post_impl<float, float>(p, f0, f1, flag_old, flag_new, bc, images, mask_in, tile_mask,
                                         st);
}
template <>
cudaError_t launch_post<double, double>(const Params<double>& p, double* f0, double* f1,
                                        const uint8_t* flag_old, const uint8_t* flag_new,
                                        const BcDev& bc, int images, const uint8_t* mask_in,
                                      uint8_t* tile_mask,
                                      cudaStream_t st) {
  return launch_post_impl<double, double>(p, f0, f1, flag_old, flag_new, bc, images, mask_in, tile_mask,
                                         st);
}
template <>
cudaError_t launch_post<__half, float>(const Params<float>& p, __half* f0, __half* f1,
                                       const uint8_t* flag_old, const uint8_t* flag_new,
                                       const BcDev& bc, int images, const uint8_t* mask_in,
                                       uint8_t* tile_mask, cudaStream_t st) {
  return launch_post_impl<__half, float>(p, f0, f1, flag_old, flag_new, bc, images, mask_in,
                                         tile_mask, st);
}

template <>
cudaError_t launch_post<fx16, float>(const Params<float>& p, fx16* f0, fx16* f1,
                                     const uint8_t* flag_old, const uint8_t* flag_new,
                                     const BcDev& bc, int images, const uint8_t* mask_in,
                                     uint8_t* tile_mask, cudaStream_t st) {
  return launch_post_impl<fx16, float>(p, f0, f1, flag_old, flag_new, bc, images, mask_in,
                                       tile_mask, st);
}

#define SLBM_POSTSTEP_INST(S, R)                                                             \
  template <>                                                                                \
  cudaError_t launch_post_step<S, R>(const Params<R>& p, S* f0, S* f1,                       \
                                     const uint8_t* flag_old, const uint8_t* flag_new,       \
                                     const BcDev& bc, const int* work, const int* list,     \
                                     const int* nlist, const GhostTables& gt,               \
                                     cudaStream_t st) {                                      \
    return launch_post_step_impl<S, R>(p, f0, f1, flag_old, flag_new, bc, work, list, nlist, \
                                       gt, st);                                              \
  }
SLBM_POSTSTEP_INST(float, float)
SLBM_POSTSTEP_INST(double, double)
SLBM_POSTSTEP_INST(__half, float)
SLBM_POSTSTEP_INST(fx16, float)
#undef SLBM_POSTSTEP_INST
}  // namespace slbm
