// dtw_inst_d.cu -- instantiation of the FP32 DTW kernels for tile list TC_TILES_D.
#include "dtw_core.cuh"

namespace tc {
TC_TILES_D(TC_TILE_DEF)
}  // namespace tc
