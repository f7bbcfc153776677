// dtw_inst_c.cu -- instantiation of the FP32 DTW kernels for tile list TC_TILES_C.
#include "dtw_core.cuh"

namespace tc {
TC_TILES_C(TC_TILE_DEF)
}  // namespace tc
