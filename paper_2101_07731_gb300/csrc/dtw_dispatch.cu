// dtw_dispatch.cu -- tile dispatch of the FP32 DTW kernels, and the FP64 refine.
//
// FP64 refine.  The candidates whose FP32 DTW cannot be told apart from the best
// one are recomputed in FP64, in exactly the operation order of a sequential
// evaluation of Eq. (1): per cell t_p = a_p - b_p, s = ((t_0*t_0) + t_1*t_1) + ...
// (separate multiply and add, no fusion), R(i,j) = s + min(up, left, diag).  The
// result is therefore bit-identical to a plain FP64 evaluation.  FP64 issues at a
// small fraction of the FP32 rate on this GPU, so a pair gets a whole warp (G = 32)
// and the fewest rows per lane R the band allows, to spread its cells over lanes.
#include "df.cuh"
#include "dtw_core.cuh"

namespace tc {

TC_TILES(TC_TILE_DECL)

// Entries e < *count: pair id m*N + n; stores the FP64 DTW in d64[e] and lowers
// best64[m] (bit pattern of a non-negative double orders like its value).  One warp
// per block, so that a handful of entries spreads over as many SMs (the FP64 pipe
// of each SM is the bound); ad_per_lane > 0: the lanes' rows widened in shared memory.
template <int R>
__global__ void __launch_bounds__(32) k_dtw_refine(const float *__restrict__ Q, const float *__restrict__ Cand, int L,
                                                    int D, int W, int64_t N, const uint32_t *__restrict__ pairs,
                                                    const int32_t *__restrict__ count, double *__restrict__ d64,
                                                    unsigned long long *__restrict__ best64, int ad_per_lane) {
    extern __shared__ double ad_smem[];
    double *ad = ad_per_lane ? ad_smem + (size_t)threadIdx.x * ad_per_lane : nullptr;
    Grp g = make_grp(32);
    const int n_entries = *count;
    for (int e = blockIdx.x; e < n_entries; e += gridDim.x) {
        const uint32_t pid = pairs[e];
        const int m = (int)(pid / (uint32_t)N);
        const int64_t n = (int64_t)(pid - (uint32_t)m * (uint32_t)N);
        double r = band_pass64<R>(Q + (size_t)m * L * D, Cand + (size_t)n * L * D, L, D, W, g, ad);
        r = grp_min(r, g);
        if (g.lig == 0) {
            d64[e] = r;
            atomicMin(best64 + m, (unsigned long long)__double_as_longlong(r));
        }
    }
}

// Double-float refine: entries e < *count get v[e] = their double-float DTW (rounded
// to double) and lower bestdf[m] (double bits); one warp per block, as above.
template <int R>
__global__ void __launch_bounds__(32) k_dtw_refine_df(const float *__restrict__ Q, const float *__restrict__ Cand,
                                                       int L, int D, int W, int64_t N,
                                                       const uint32_t *__restrict__ pairs,
                                                       const int32_t *__restrict__ count, double *__restrict__ v,
                                                       unsigned long long *__restrict__ bestdf) {
    Grp g = make_grp(32);
    const int n_entries = *count;
    for (int e = blockIdx.x; e < n_entries; e += gridDim.x) {
        const uint32_t pid = pairs[e];
        const int m = (int)(pid / (uint32_t)N);
        const int64_t n = (int64_t)(pid - (uint32_t)m * (uint32_t)N);
        double r = band_pass_df<R>(Q + (size_t)m * L * D, Cand + (size_t)n * L * D, L, D, W, g);
        r = grp_min(r, g);
        if (g.lig == 0) {
            v[e] = r;
            atomicMin(bestdf + m, (unsigned long long)__double_as_longlong(r));
        }
    }
}

// The same with the band's cell costs tabulated first: the block (kDfBandThreads
// threads) computes every in-band cell's double-float cost into a shared-memory table
// in parallel (two cells per thread at a time: each cost is a long serial chain), and
// one warp then runs the band DP from the table (band_pass_df_table).  The series are
// read through L1 (a pair is a few KB); the table alone fits twice per SM for the
// benchmark shape (108 KB at L = 256, W = 26).  Bit-identical to k_dtw_refine_df; used
// when the table fits in shared memory.
constexpr int kDfBandThreads = 128;

template <int R, int DM>
__global__ void __launch_bounds__(kDfBandThreads) k_dtw_refine_df_band(const float *__restrict__ Q,
                                                                       const float *__restrict__ Cand, int L, int D,
                                                                       int W, int64_t N,
                                                                       const uint32_t *__restrict__ pairs,
                                                                       const int32_t *__restrict__ count,
                                                                       double *__restrict__ v,
                                                                       unsigned long long *__restrict__ bestdf) {
    extern __shared__ __align__(16) float2 cost[];
    const int E = L * D, BW = 2 * W + 1, cells = L * BW;
    const int n_entries = *count;
    for (int e = blockIdx.x; e < n_entries; e += gridDim.x) {
        const uint32_t pid = pairs[e];
        const int m = (int)(pid / (uint32_t)N);
        const int64_t n = (int64_t)(pid - (uint32_t)m * (uint32_t)N);
        const float *qa = Q + (size_t)m * E, *cb = Cand + (size_t)n * E;
        __syncthreads();  // the previous entry's sweep is done with the table
        for (int k0 = threadIdx.x; k0 < cells; k0 += 2 * kDfBandThreads) {
            float ch[2], cl[2];
            bool in[2];
            int kk[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                kk[u] = k0 + u * kDfBandThreads;
                const int k = kk[u] < cells ? kk[u] : cells - 1;
                const int i = k / BW, j = i + (k - i * BW) - W;
                in[u] = kk[u] < cells && j >= 0 && j < L;
                const int jj = in[u] ? j : i;
                df_cell_cost<DM>(qa + (size_t)i * D, cb + (size_t)jj * D, D, ch[u], cl[u]);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u)
                if (in[u]) cost[kk[u]] = make_float2(ch[u], cl[u]);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            Grp g = make_grp(32);
            double r = band_pass_df_table<R>(cost, L, W, g);
            r = grp_min(r, g);
            if (g.lig == 0) {
                v[e] = r;
                atomicMin(bestdf + m, (unsigned long long)__double_as_longlong(r));
            }
        }
    }
}

namespace {
constexpr size_t kDfBandSmemMax = 200 * 1024;

size_t df_band_smem(int L, int, int W) { return (size_t)L * (2 * W + 1) * sizeof(float2); }

template <int R, int DM>
cudaError_t launch_refine_df_band(int blocks, cudaStream_t s, const DtwRefineArgs &x, size_t smem) {
    static bool attr = false;  // idempotent
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_dtw_refine_df_band<R, DM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDfBandSmemMax);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_dtw_refine_df_band<R, DM><<<blocks, kDfBandThreads, smem, s>>>(x.Q, x.C, x.L, x.D, x.W, x.N, x.pairs, x.count,
                                                                     x.d64, x.best64);
    note_launch();
    return cudaGetLastError();
}
}  // namespace

bool refine_df_table_fits_smem(int L, int D, int W) {
    return refine_rows_for(W) <= 2 && D <= 32 && df_band_smem(L, D, W) <= kDfBandSmemMax;
}

cudaError_t dtw_refine_df_launch(int R, int blocks, cudaStream_t s, const DtwRefineArgs &x) {
    const size_t smem = df_band_smem(x.L, x.D, x.W);
    if ((R == 1 || R == 2) && x.D <= 32 && smem <= kDfBandSmemMax) {
        if (R == 1) {
            if (x.D <= 8) return launch_refine_df_band<1, 8>(blocks, s, x, smem);
            if (x.D <= 16) return launch_refine_df_band<1, 16>(blocks, s, x, smem);
            return launch_refine_df_band<1, 32>(blocks, s, x, smem);
        }
        if (x.D <= 8) return launch_refine_df_band<2, 8>(blocks, s, x, smem);
        if (x.D <= 16) return launch_refine_df_band<2, 16>(blocks, s, x, smem);
        return launch_refine_df_band<2, 32>(blocks, s, x, smem);
    }
    switch (R) {
#define TC_RD(RV)                                                                                                  \
    case RV:                                                                                                       \
        k_dtw_refine_df<RV><<<blocks, 32, 0, s>>>(x.Q, x.C, x.L, x.D, x.W, x.N, x.pairs, x.count, x.d64, x.best64); \
        note_launch();                                                                                             \
        return cudaGetLastError();
        TC_REFINE_RS(TC_RD)
#undef TC_RD
    }
    return cudaErrorInvalidValue;
}

int refine_rows_for(int W) {
#define TC_RR(R) \
    if (32 * ((R) + 1) >= 2 * W + (R)) return R;
    TC_REFINE_RS(TC_RR)
#undef TC_RR
    return 0;
}

// Rows widened in shared memory when a warp's slots fit in 64 KB.
int refine_ad_per_lane(int R, int D) { return R * D <= 256 ? R * D : 0; }

cudaError_t dtw_refine_launch(int R, int blocks, cudaStream_t s, const DtwRefineArgs &x) {
    const int ad = refine_ad_per_lane(R, x.D);
    const size_t smem = (size_t)32 * ad * sizeof(double);
    switch (R) {
#define TC_RL(RV)                                                                                                 \
    case RV: {                                                                                                    \
        static bool attr = false;                                                                                 \
        if (!attr) {                                                                                              \
            cudaError_t e = cudaFuncSetAttribute(k_dtw_refine<RV>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                                 64 * 1024);                                                      \
            if (e != cudaSuccess) return e;                                                                       \
            attr = true;                                                                                          \
        }                                                                                                         \
        k_dtw_refine<RV><<<blocks, 32, smem, s>>>(x.Q, x.C, x.L, x.D, x.W, x.N, x.pairs, x.count, x.d64, x.best64, \
                                                  ad);                                                            \
        note_launch();                                                                                            \
        return cudaGetLastError();                                                                                \
    }
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

int dtw_occupancy(int tile, int which, int G) {
    switch (tile) {
#define X(id, R, DM) \
    case id:         \
        return tile##id##_occupancy(which, G);
        TC_TILES(X)
#undef X
    }
    return 0;
}

}  // namespace tc
