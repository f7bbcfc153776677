// dtw_inst_b.cu -- instantiation of the FP32 DTW kernels for tile list TC_TILES_B.
#include "dtw_core.cuh"

namespace tc {
TC_TILES_B(TC_TILE_DEF)
}  // namespace tc
