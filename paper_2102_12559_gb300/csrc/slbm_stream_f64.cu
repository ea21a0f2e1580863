// Double-precision instantiation of the fused stream-collide kernel.
#include "slbm_stream.cuh"

namespace slbm {
template <>
cudaError_t launch_stream_collide<double, double>(const Params<double>& p, int P, const void* tm0,
                                          const void* tm1, double* fout0, double* fout1,
                                          const uint8_t* flag_cur, uint8_t* flag_nxt,
                                          const uint8_t* tile_mask, uint8_t* mask_next,
                                          const BcDev& bc, int* err, cudaStream_t st) {
  return launch_stream_collide_impl<double, double>(p, P, static_cast<const CUtensorMap*>(tm0),
                                            static_cast<const CUtensorMap*>(tm1), fout0, fout1,
                                            flag_cur, flag_nxt, tile_mask, mask_next, bc, err,
                                            st);
}
}  // namespace slbm
