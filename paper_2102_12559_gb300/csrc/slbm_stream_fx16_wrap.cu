// Fixed-point instantiation of the fused stream-collide kernel for grids whose
// periodic y rows are read through their images near the edges (wrap_y).
#include "slbm_stream.cuh"

namespace slbm {
template <>
cudaError_t launch_stream_collide_wrap<fx16, float>(const Params<float>& p, int P, const fx16* fin0,
                                             const fx16* fin1, fx16* fout0, fx16* fout1,
                                             const uint8_t* flag_cur, uint8_t* flag_nxt,
                                             const uint8_t* tile_mask, uint8_t* mask_next,
                                             cudaStream_t st) {
  return launch_stream_collide_impl<fx16, float, true>(p, P, fin0, fin1, fout0, fout1, flag_cur,
                                                  flag_nxt, tile_mask, mask_next, st);
}
}  // namespace slbm
