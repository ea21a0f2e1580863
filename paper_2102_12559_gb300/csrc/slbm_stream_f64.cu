// Double-precision instantiation of the fused stream-collide kernel.
#include "slbm_stream.cuh"

namespace slbm {
template <>
cudaError_t launch_stream_collide<double, double>(const Params<double>& p, int P, const double* fin0,
                                        const double* fin1, double* fout0, double* fout1,
                                        const uint8_t* flag_cur, uint8_t* flag_nxt,
                                        const uint8_t* tile_mask, uint8_t* mask_next,
                                        cudaStream_t st) {
  if (p.wrap_y)
    return launch_stream_collide_wrap<double, double>(p, P, fin0, fin1, fout0, fout1, flag_cur, flag_nxt,
                                               tile_mask, mask_next, st);
  return launch_stream_collide_impl<double, double, false>(p, P, fin0, fin1, fout0, fout1, flag_cur,
                                                   flag_nxt, tile_mask, mask_next, st);
}
}  // namespace slbm
