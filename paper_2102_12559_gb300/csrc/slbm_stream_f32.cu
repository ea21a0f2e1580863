// Single-precision instantiation of the fused stream-collide kernel.
#include "slbm_stream.cuh"

namespace slbm {
template <>
cudaError_t launch_stream_collide<float, float>(const Params<float>& p, int P, const void* tm0,
                                          const void* tm1, float* fout0, float* fout1,
                                          const uint8_t* flag_cur, uint8_t* flag_nxt,
                                          const uint8_t* tile_mask, uint8_t* mask_next,
                                          const BcDev& bc, int* err, cudaStream_t st) {
  return launch_stream_collide_impl<float, float>(p, P, static_cast<const CUtensorMap*>(tm0),
                                            static_cast<const CUtensorMap*>(tm1), fout0, fout1,
                                            flag_cur, flag_nxt, tile_mask, mask_next, bc, err,
                                            st);
}

static int staged_row(int elem_size) {
  return elem_size == 2 ? StageGeom<__half>::txp : StageGeom<float>::txp;
}

size_t stream_stage_bytes(int elem_size, int nh, int G) {
  return (size_t)nh * nh * (kTY + 2 * G) * staged_row(elem_size) * elem_size;
}

void stream_box(int elem_size, int G, int Q, unsigned box[3]) {
  box[0] = staged_row(elem_size);
  box[1] = kTY + 2 * G;
  box[2] = Q;
}
}  // namespace slbm
