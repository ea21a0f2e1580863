// FP16-storage instantiation of the fused stream-collide kernel for grids whose
// periodic y rows are read through their images near the edges (wrap_y).
#include "slbm_stream.cuh"

namespace slbm {
template <>
cudaError_t launch_stream_collide_wrap<__half, float>(const Params<float>& p, int P, const __half* fin0,
                                             const __half* fin1, __half* fout0, __half* fout1,
                                             const uint8_t* flag_cur, uint8_t* flag_nxt,
                                             const uint8_t* tile_mask, uint8_t* mask_next,
                                             cudaStream_t st) {
  return launch_stream_collide_impl<__half, float, true>(p, P, fin0, fin1, fout0, fout1, flag_cur,
                                                  flag_nxt, tile_mask, mask_next, st);
}
}  // namespace slbm
