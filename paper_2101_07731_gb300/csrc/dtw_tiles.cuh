// dtw_tiles.cuh -- compiled band tiles of the FP32 DTW kernels and their launch
// records.  A tile fixes R (rows per lane: each loaded candidate point serves R
// cells) and DM (dimensions held in registers; D <= DM, the rest zero-padded; for
// D <= 8 there is a tile with DM == D).  The group width G (lanes per pair) is a
// run-time choice with G*(R+1) >= 2W+R.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// X(id, R, DM), split over four translation units compiled in parallel
#define TC_TILES_A(X)                                                                                      \
    X(0, 4, 1) X(1, 8, 1) X(2, 16, 1) X(3, 4, 2) X(4, 8, 2) X(5, 16, 2) X(6, 4, 3) X(7, 8, 3) X(8, 16, 3) \
    X(9, 4, 4) X(10, 8, 4) X(11, 16, 4)
#define TC_TILES_B(X)                                                                                           \
    X(12, 4, 5) X(13, 8, 5) X(14, 16, 5) X(15, 4, 6) X(16, 8, 6) X(17, 16, 6) X(18, 4, 7) X(19, 8, 7) X(20, 16, 7) \
    X(21, 4, 8) X(22, 8, 8) X(23, 16, 8)
#define TC_TILES_C(X) \
    X(24, 4, 12) X(25, 8, 12) X(26, 4, 16) X(27, 8, 16) X(28, 2, 32) X(29, 4, 32) X(30, 6, 32) X(31, 2, 64)
#define TC_TILES_D(X) X(32, 4, 9) X(33, 8, 9) X(34, 4, 10) X(35, 8, 10) X(36, 4, 11) X(37, 8, 11)
#define TC_TILES(X) TC_TILES_A(X) TC_TILES_B(X) TC_TILES_C(X) TC_TILES_D(X)

// FP64 refine: rows per lane (one warp per pair, G = 32)
#define TC_REFINE_RS(X) X(1) X(2) X(4) X(6) X(8) X(16)

namespace tc {

struct TileInfo {
    int R, DMAX;
};
#define TC_TILE_INFO(id, R, DM) {R, DM},
static const TileInfo kTiles[] = {TC_TILES(TC_TILE_INFO)};
#undef TC_TILE_INFO
constexpr int kNumTiles = (int)(sizeof(kTiles) / sizeof(kTiles[0]));

struct DtwNnArgs {
    const float *Q;        // block of queries [Mb][L][D]
    const float *C;        // candidates [N][L][D]
    int L, D, W, G;
    int64_t N;
    const uint32_t *pairs; // entry -> m*N + n
    const float *lb;       // entry -> best lower bound (+inf = pruned), or null
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
    int L, D, W;
    int64_t N;
    const uint32_t *pairs;
    const int32_t *count;
    double *d64;
    unsigned long long *best64;
};

cudaError_t dtw_pairs_launch(int tile, int G, int blocks, cudaStream_t s, const float *A, const float *B, int64_t P,
                             int L, int D, int W, float *dist, float *ck, int C);
cudaError_t dtw_nn_launch(int tile, int blocks, cudaStream_t s, const DtwNnArgs &x);
// FP64 refine with R rows per lane (R in TC_REFINE_RS, one warp per pair)
cudaError_t dtw_refine_launch(int R, int blocks, cudaStream_t s, const DtwRefineArgs &x);
// double-float pass: d64 receives the double-float values, best64 the per-query minimum
cudaError_t dtw_refine_df_launch(int R, int blocks, cudaStream_t s, const DtwRefineArgs &x);
// whether dtw_refine_df_launch keeps the band's cost table in shared memory
bool refine_df_table_fits_smem(int L, int D, int W);
// the same pass with the cost table in global memory: `slots` blocks, tab holding
// slots * refine_gtab_slot_bytes(L, W) bytes
size_t refine_gtab_slot_bytes(int L, int W);
cudaError_t dtw_refine_df_gtab_launch(int R, int slots, cudaStream_t s, const DtwRefineArgs &x, float2 *tab);
int refine_rows_for(int W);  // smallest compiled R with 32*(R+1) >= 2W+R, or 0
cudaError_t dtw_backward_launch(int tile, int G, int blocks, size_t smem, cudaStream_t s, const float *A,
                                const float *B, const float *ck, int C, const float *gd, int64_t P, int L, int D,
                                int W, float *gA, float *gB, int threads);
// resident blocks per SM of a launch of the tile with G lanes per pair (which: 0 pairs,
// 1 search)
int dtw_occupancy(int tile, int which, int G);

}  // namespace tc
