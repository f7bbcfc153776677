// dtw_inst_a.cu -- instantiation of the FP32 DTW kernels for tile list TC_TILES_A.
#include "dtw_core.cuh"

namespace tc {
TC_TILES_A(TC_TILE_DEF)
}  // namespace tc
