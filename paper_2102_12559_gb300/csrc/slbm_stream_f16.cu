// FP16-storage instantiation of the fused stream-collide kernel: populations
// stored as half-precision deviations s_i = f_i - W_i, arithmetic in FP32.
#include "slbm_stream.cuh"

namespace slbm {
template <>
cudaError_t launch_stream_collide<__half, float>(const Params<float>& p, int P, const __half* fin0,
                                        const __half* fin1, __half* fout0, __half* fout1,
                                        const uint8_t* flag_cur, uint8_t* flag_nxt,
                                        const uint8_t* tile_mask, uint8_t* mask_next,
                                        cudaStream_t st) {
  if (p.wrap_y)
    return launch_stream_collide_wrap<__half, float>(p, P, fin0, fin1, fout0, fout1, flag_cur, flag_nxt,
                                               tile_mask, mask_next, st);
  return launch_stream_collide_impl<__half, float, false>(p, P, fin0, fin1, fout0, fout1, flag_cur,
                                                   flag_nxt, tile_mask, mask_next, st);
}
}  // namespace slbm
