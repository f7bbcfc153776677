// batch_dtw_r16.cu -- the batched search's band DTW with 16 rows per lane, one kernel
// per point width DM (exact width, 1..8); a unit of its own so that the
// tile instantiations compile in parallel.
#include "batch_internal.cuh"

namespace tc {

#define TC_DMS_R16(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8)

cudaError_t batch_dtw_launch_r16(int dm, int grid, cudaStream_t s, const BatchSet *sets, const int *order, int nsets,
                                 int phase, BatchCtl *ctl) {
    switch (dm) {
#define X(DMV)                                                                                             \
    case DMV:                                                                                              \
        k_batch_dtw<16, DMV><<<grid, kBatchThreads, batch_dtw_smem(16, DMV), s>>>(sets, order, nsets, phase, ctl); \
        return cudaGetLastError();
        TC_DMS_R16(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

cudaError_t batch_dtw_grid_r16(int dm, int *grid) {
    switch (dm) {
#define X(DMV) \
    case DMV: return kernel_grid((const void *)k_batch_dtw<16, DMV>, batch_dtw_smem(16, DMV), grid);
        TC_DMS_R16(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

}  // namespace tc
