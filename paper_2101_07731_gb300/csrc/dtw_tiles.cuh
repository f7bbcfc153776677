// dtw_tiles.cuh -- compiled band tiles of the DTW kernels and their launch records.
// A tile fixes R (rows per lane, i.e. reuse of each loaded candidate point) and
// DMAX (dimensions held in registers; D <= DMAX, the rest zero-padded).  The
// group width G (lanes per pair) is a run-time choice with G*(R+1) >= 2W+R.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// X(id, R, DMAX)
#define TC_TILES(X)                                   \
    X(0, 4, 4) X(1, 8, 4) X(2, 16, 4)                 \
    X(3, 4, 6) X(4, 8, 6) X(5, 16, 6)                 \
    X(6, 4, 8) X(7, 8, 8)                             \
    X(8, 4, 12) X(9, 8, 12)                           \
    X(10, 4, 16) X(11, 8, 16)                         \
    X(12, 2, 32) X(13, 4, 32) X(14, 6, 32)            \
    X(15, 2, 64)

namespace tc {

struct TileInfo {
    int R, DMAX;
};
#define TC_TILE_INFO(id, R, DMAX) {R, DMAX},
static const TileInfo kTiles[] = {TC_TILES(TC_TILE_INFO)};
#undef TC_TILE_INFO
constexpr int kNumTiles = (int)(sizeof(kTiles) / sizeof(kTiles[0]));

struct DtwNnArgs {
    const float *Q;        // block of queries [Mb][L][D]
    const float *C;        // candidates [N][L][D]
    int L, D, W, G;
    int64_t N;
    const uint32_t *pairs; // entry -> m*N + n
    const float *lb;       // entry -> best lower bound (+inf = pruned)
    const int32_t *count;  // number of entries (device), or null: n_static
    int n_static;
    int *cursor;           // work counter (zeroed before launch)
    unsigned long long *bsf;  // [Mb] packed best-so-far
    float rho;
    float *dtw;            // entry -> FP32 DTW or +inf
    unsigned long long *counters;  // started, abandoned, cells, pruned
};

struct DtwRefineArgs {
    const float *Q;
    const float *C;
    int L, D, W, G;
    int64_t N;
    const uint32_t *pairs;
    const int32_t *count;
    double *d64;
    unsigned long long *best64;
};

cudaError_t dtw_pairs_launch(int tile, int G, int blocks, cudaStream_t s, const float *A, const float *B, int64_t P,
                             int L, int D, int W, float *dist, float *ck, int C);
cudaError_t dtw_nn_launch(int tile, int blocks, cudaStream_t s, const DtwNnArgs &x);
cudaError_t dtw_refine_launch(int tile, int blocks, cudaStream_t s, const DtwRefineArgs &x);
cudaError_t dtw_backward_launch(int tile, int G, int blocks, size_t smem, cudaStream_t s, const float *A,
                                const float *B, const float *ck, int C, const float *gd, int64_t P, int L, int D,
                                int W, float *gA, float *gB, int threads);
int dtw_occupancy(int tile, int which);

}  // namespace tc
