// Single-precision instantiation of the fused stream-collide kernel.
#include "slbm_stream.cuh"

namespace slbm {
template <>
cudaError_t launch_stream_collide<float, float>(const Params<float>& p, int P, const float* fin0,
                                        const float* fin1, float* fout0, float* fout1,
                                        const uint8_t* flag_cur, uint8_t* flag_nxt,
                                        const uint8_t* tile_mask, uint8_t* mask_next,
                                        cudaStream_t st) {
  if (p.wrap_y)
    return launch_stream_collide_wrap<float, float>(p, P, fin0, fin1, fout0, fout1, flag_cur, flag_nxt,
                                               tile_mask, mask_next, st);
  return launch_stream_collide_impl<float, float, false>(p, P, fin0, fin1, fout0, fout1, flag_cur,
                                                   flag_nxt, tile_mask, mask_next, st);
}
}  // namespace slbm
