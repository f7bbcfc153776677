// dtw_refine_gtab.cu -- double-float refine of long bands with the cell-cost table in
// global memory.
//
// The tabulated refine (k_dtw_refine_df_band, dtw_dispatch.cu) takes the double-float
// cost arithmetic off the sequential DP path: a block computes every in-band cell's
// cost in parallel into a table, then one warp sweeps the band reading the table.  Its
// table lives in shared memory, L*(2W+1)*8 bytes, so long bands (L = 2,048, W = 102:
// 3.4 MB) fell back to one warp doing both, with the cost of 32 dimensions in
// double-float as one long serial chain per cell (~26 ms for one pair).  Here each
// block owns a slot of a global-memory table instead: it writes its entry's costs with
// all threads, in the order the sweep reads them (per step, the 32 lanes' R costs
// contiguous: table_dp_pos), synchronises, and its first warp runs
// band_pass_df_table_dp, which streams each lane's costs through a shared-memory ring
// of cp.async copies a few steps ahead (a sweep that loaded its costs from the
// row-major table step by step waited ~3 us per step on L2/HBM).  Same operations in
// the same order, so the value is bit-identical to k_dtw_refine_df and to the
// shared-memory table kernel.
#include "df.cuh"
#include "dtw_core.cuh"

namespace tc {

constexpr int kGtabThreads = 128;  // two blocks (table slots) per SM at up to 255 registers
// consecutive band columns of one row per thread and item (registers: the query point and
// the columns' candidate points, DM floats each)
template <int DM>
__host__ __device__ constexpr int gtab_cols() { return DM <= 32 ? 4 : 2; }

// Steps of the band sweep with R rows per lane: tau in [0, tau_end].
__host__ __device__ inline int sweep_steps(int L, int W, int R) {
    const int nv = (L + R - 1) / R;
    const int jhi = min(L - 1, (nv - 1) * R + R - 1 + W);
    return jhi + nv;  // tau_end + 1
}

template <int R, int DM>
__global__ void __launch_bounds__(kGtabThreads) k_dtw_refine_df_gtab(const float *__restrict__ Q,
                                                                     const float *__restrict__ Cand, int L, int D,
                                                                     int W, int64_t N,
                                                                     const uint32_t *__restrict__ pairs,
                                                                     const int32_t *__restrict__ count,
                                                                     float2 *__restrict__ tab,
                                                                     double *__restrict__ v,
                                                                     unsigned long long *__restrict__ bestdf) {
    extern __shared__ __align__(16) float2 dring[];  // the sweep warp's ring, 32 * R * kDfRing
    const int E = L * D, BW = 2 * W + 1, cells = L * BW;
    float2 *cost = tab + (size_t)blockIdx.x * sweep_steps(L, W, R) * 32 * R;
    const int n_entries = *count;
    for (int e = blockIdx.x; e < n_entries; e += gridDim.x) {
        const uint32_t pid = pairs[e];
        const int m = (int)(pid / (uint32_t)N);
        const int64_t n = (int64_t)(pid - (uint32_t)m * (uint32_t)N);
        const float *qa = Q + (size_t)m * E, *cb = Cand + (size_t)n * E;
        __syncthreads();  // the previous entry's sweep is done with the slot
        // items (row i, kGtabCols consecutive band offsets): the query point once, the
        // candidate points of the columns next (their loads in flight together), then
        // the costs; 16-byte loads where the rows allow
        const bool vec = (D % 4) == 0 && ((((uintptr_t)qa) | ((uintptr_t)cb)) & 15) == 0;
        constexpr int kGtabCols = gtab_cols<DM>();
        const int ngrp = (BW + kGtabCols - 1) / kGtabCols;
        for (int it = threadIdx.x; it < L * ngrp; it += kGtabThreads) {
            const int i = it / ngrp, o0 = (it - i * ngrp) * kGtabCols;
            float a[DM];
            df_load_point<DM>(qa + (size_t)i * D, D, vec, a);
            float b[kGtabCols][DM];
            bool in[kGtabCols];
            int jj[kGtabCols];
#pragma unroll
            for (int u = 0; u < kGtabCols; ++u) {
                const int j = i + o0 + u - W;
                in[u] = o0 + u < BW && j >= 0 && j < L;
                jj[u] = in[u] ? j : i;
                df_load_point<DM>(cb + (size_t)jj[u] * D, D, vec, b[u]);
            }
            // cell (i, j) is row r of virtual lane vv = i / R, read by lane vv % 32 at step j + vv
            const int vv = i / R, r = i - vv * R;
#pragma unroll
            for (int u = 0; u < kGtabCols; ++u) {
                float ch, cl;
                df_cell_cost_regs<DM>(a, b[u], D, ch, cl);
                if (in[u]) cost[table_dp_pos(jj[u] + vv, vv & 31, R, r)] = make_float2(ch, cl);
            }
        }
        __syncthreads();  // the block's table writes are visible to its first warp
        if (threadIdx.x < 32) {
            Grp g = make_grp(32);
            double r = band_pass_df_table_dp<R>(cost, L, W, g, dring);
            r = grp_min(r, g);
            if (g.lig == 0) {
                v[e] = r;
                atomicMin(bestdf + m, (unsigned long long)__double_as_longlong(r));
            }
        }
    }
}

size_t refine_gtab_slot_bytes(int L, int W) {
    const int R = refine_rows_for(W);
    return (size_t)sweep_steps(L, W, R) * 32 * (R > 0 ? R : 1) * sizeof(float2);
}

// Launch with `slots` blocks (one table slot each; tab holds slots * L*(2W+1) float2).
cudaError_t dtw_refine_df_gtab_launch(int R, int slots, cudaStream_t s, const DtwRefineArgs &x, float2 *tab) {
    const int dm = x.D <= 8 ? 8 : x.D <= 32 ? 32 : 64;
#define TC_GT(RV, DMV)                                                                                         \
    if (R == RV && dm == DMV) {                                                                                \
        k_dtw_refine_df_gtab<RV, DMV><<<slots, kGtabThreads, (size_t)32 * RV * kDfRing * sizeof(float2), s>>>( \
            x.Q, x.C, x.L, x.D, x.W, x.N, x.pairs, x.count, tab, x.d64, x.best64);                                 \
        note_launch();                                                                                         \
        return cudaGetLastError();                                                                             \
    }
#define TC_GT_R(RV) TC_GT(RV, 8) TC_GT(RV, 32) TC_GT(RV, 64)
    TC_REFINE_RS(TC_GT_R)
#undef TC_GT_R
#undef TC_GT
    return cudaErrorInvalidValue;
}

}  // namespace tc
