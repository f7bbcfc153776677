// dtw_dispatch.cu -- tile dispatch of the FP32 DTW kernels, and the FP64 refine.
//
// FP64 refine.  The candidates whose FP32 DTW cannot be told apart from the best
// one are recomputed in FP64, in exactly the operation order of a sequential
// evaluation of Eq. (1): per cell t_p = a_p - b_p, s = ((t_0*t_0) + t_1*t_1) + ...
// (separate multiply and add, no fusion), R(i,j) = s + min(up, left, diag).  The
// result is therefore bit-identical to a plain FP64 evaluation.  FP64 issues at a
// small fraction of the FP32 rate on this GPU, so a pair gets a whole warp (G = 32)
// and the fewest rows per lane R the band allows, to spread its cells over lanes.
#include "dtw_core.cuh"

namespace tc {

TC_TILES(TC_TILE_DECL)

// Entries e < *count: pair id m*N + n; stores the FP64 DTW in d64[e] and lowers
// best64[m] (bit pattern of a non-negative double orders like its value).
template <int R>
__global__ void __launch_bounds__(128) k_dtw_refine(const float *__restrict__ Q, const float *__restrict__ Cand, int L,
                                                     int D, int W, int64_t N, const uint32_t *__restrict__ pairs,
                                                     const int32_t *__restrict__ count, double *__restrict__ d64,
                                                     unsigned long long *__restrict__ best64) {
    Grp g = make_grp(32);
    const int warps_per_block = blockDim.x / 32;
    const int gid = blockIdx.x * warps_per_block + threadIdx.x / 32;
    const int stride = gridDim.x * warps_per_block;
    const int n_entries = *count;
    for (int e = gid; e < n_entries; e += stride) {
        const uint32_t pid = pairs[e];
        const int m = (int)(pid / (uint32_t)N);
        const int64_t n = (int64_t)(pid - (uint32_t)m * (uint32_t)N);
        double r = band_pass64<R>(Q + (size_t)m * L * D, Cand + (size_t)n * L * D, L, D, W, g);
        r = grp_min(r, g);
        if (g.lig == 0) {
            d64[e] = r;
            atomicMin(best64 + m, (unsigned long long)__double_as_longlong(r));
        }
    }
}

int refine_rows_for(int W) {
#define TC_RR(R) \
    if (32 * ((R) + 1) >= 2 * W + (R)) return R;
    TC_REFINE_RS(TC_RR)
#undef TC_RR
    return 0;
}

cudaError_t dtw_refine_launch(int R, int blocks, cudaStream_t s, const DtwRefineArgs &x) {
    switch (R) {
#define TC_RL(RV)                                                                                                \
    case RV:                                                                                                     \
        k_dtw_refine<RV><<<blocks, 128, 0, s>>>(x.Q, x.C, x.L, x.D, x.W, x.N, x.pairs, x.count, x.d64, x.best64); \
        note_launch();                                                                                           \
        return cudaGetLastError();
        TC_REFINE_RS(TC_RL)
#undef TC_RL
    }
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ FP32 tile dispatch
cudaError_t dtw_pairs_launch(int tile, int G, int blocks, cudaStream_t s, const float *A, const float *B, int64_t P,
                             int L, int D, int W, float *dist, float *ck, int C) {
    switch (tile) {
#define X(id, R, DM) \
    case id:         \
        return tile##id##_pairs(G, blocks, s, A, B, P, L, D, W, dist, ck, C);
        TC_TILES(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

cudaError_t dtw_nn_launch(int tile, int blocks, cudaStream_t s, const DtwNnArgs &x) {
    switch (tile) {
#define X(id, R, DM) \
    case id:         \
        return tile##id##_nn(blocks, s, x);
        TC_TILES(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

cudaError_t dtw_backward_launch(int tile, int G, int blocks, size_t smem, cudaStream_t s, const float *A,
                                const float *B, const float *ck, int C, const float *gd, int64_t P, int L, int D,
                                int W, float *gA, float *gB, int threads) {
    switch (tile) {
#define X(id, R, DM) \
    case id:         \
        return tile##id##_backward(G, blocks, threads, smem, s, A, B, ck, C, gd, P, L, D, W, gA, gB);
        TC_TILES(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

int dtw_occupancy(int tile, int which) {
    switch (tile) {
#define X(id, R, DM) \
    case id:         \
        return tile##id##_occupancy(which);
        TC_TILES(X)
#undef X
    }
    return 0;
}

}  // namespace tc
