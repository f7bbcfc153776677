// dtw.cu -- banded DTW dynamic programme (Eq. 1 with the Sakoe-Chiba window,
// Section 2) on sm_103a.
//
// Work decomposition ("row-block systolic sweep").  A group of G lanes (G = 4, 8,
// 16 or 32, several groups per warp) computes one pair.  The L rows are cut into
// "virtual lanes" of R consecutive rows; virtual lane v (rows vR .. vR+R-1) visits
// the columns of its band, j in [vR-W, vR+R-1+W] clipped to [0, L-1], one column
// per time step, and computes all R cells of that column from R query points held
// in registers and one candidate point loaded per step (so a candidate load is
// reused R times).  Virtual lane v processes column j at time t = j + v, exactly one
// step after virtual lane v-1 did, so the only value crossing lanes per step is the
// bottom cell of the lane above, passed with one shuffle.  Physical lane l of the
// group runs virtual lanes l, l+G, l+2G, ...; they never overlap in time when
// G*(R+1) >= 2W+R, which the host checks when it picks a tile.
//
// Early abandoning (Section 7.1).  Define tau(i,j) = floor(i/R) + j.  Along any
// warping path tau grows by 0, 1 or 2 per step, so every path from (0,0) to
// (L-1,L-1) has a cell with tau in {t-1, t}; along the backtracked argmin path the
// computed values never decrease.  Hence if every cell computed at times t-1 and t
// exceeds the threshold, so does the final value, and the pair can be dropped.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "dtw_tiles.cuh"

namespace tc {

template <typename T>
__device__ __forceinline__ T tinf();
template <>
__device__ __forceinline__ float tinf<float>() { return __int_as_float(0x7f800000); }
template <>
__device__ __forceinline__ double tinf<double>() { return __longlong_as_double(0x7ff0000000000000LL); }

// Squared Euclidean cell cost.  FP32: fused multiply-add chain (its rounding is
// covered by the error bound used for pruning).  FP64: separate multiply and add
// in dimension order, so the value is bit-identical to a plain sequential sum.
// Padded dimensions hold 0 in both operands and add exactly 0.
template <int DMAX>
__device__ __forceinline__ float cell_cost(const float (&a)[DMAX], const float (&b)[DMAX]) {
    float s = 0.f;
#pragma unroll
    for (int p = 0; p < DMAX; ++p) {
        float t = a[p] - b[p];
        s = fmaf(t, t, s);
    }
    return s;
}
template <int DMAX>
__device__ __forceinline__ double cell_cost(const double (&a)[DMAX], const double (&b)[DMAX]) {
    double s = 0.0;
#pragma unroll
    for (int p = 0; p < DMAX; ++p) {
        double t = __dsub_rn(a[p], b[p]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}
__device__ __forceinline__ float add_rn(float x, float y) { return __fadd_rn(x, y); }
__device__ __forceinline__ double add_rn(double x, double y) { return __dadd_rn(x, y); }
__device__ __forceinline__ float tmin3(float a, float b, float c) { return fminf(fminf(a, b), c); }
__device__ __forceinline__ double tmin3(double a, double b, double c) { return fmin(fmin(a, b), c); }

// Lane-group geometry inside a warp.
struct Grp {
    int G;          // lanes per group
    int lig;        // lane index in group
    unsigned mask;  // lanes of this group
    int src;        // warp lane of the predecessor (cyclic) in the group
};
__device__ __forceinline__ Grp make_grp(int G) {
    Grp g;
    int lane = threadIdx.x & 31;
    g.G = G;
    g.lig = lane & (G - 1);
    int base = lane - g.lig;
    g.mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << base);
    g.src = base + ((g.lig + G - 1) & (G - 1));
    return g;
}
template <typename T>
__device__ __forceinline__ T grp_min(T v, const Grp &g) {
    for (int o = g.G >> 1; o > 0; o >>= 1) {
        T w = __shfl_xor_sync(g.mask, v, o);
        v = v < w ? v : w;
    }
    return v;
}

// Columns visited by virtual lane v: [jlo, jhi].
__device__ __forceinline__ int v_jlo(int v, int R, int W) { return max(0, v * R - W); }
__device__ __forceinline__ int v_jhi(int v, int R, int W, int L) { return min(L - 1, v * R + R - 1 + W); }

// No-op hook set: the default for a plain forward pass.
struct NoHooks {
    __device__ __forceinline__ void cell_row(int, int, int, float) {}
    __device__ __forceinline__ void cell_row(int, int, int, double) {}
    template <typename T>
    __device__ __forceinline__ T top(int) const { return tinf<T>(); }
    // called every kAbandonEvery steps with the group-wide frontier minimum
    template <typename T>
    __device__ __forceinline__ bool abandon(T) { return false; }
    template <typename T>
    __device__ __forceinline__ void after_col(int, int, T) {}
    static constexpr bool kAbandon = false;
    static constexpr bool kCells = false;
};

constexpr int kAbandonEvery = 8;

// One pass of the band DP over virtual lanes [v0, v1) of one pair.
//   A: rows series [L][D] (float32), B: columns series.
//   v0 > 0: the row above (v0*R-1) comes from hooks.top(j); v0 == 0: the DP origin.
//   Hooks::cell_row(i, j, r, val) sees every cell of row-offset r (if kCells).
// Returns R(L-1, L-1) on the lane that computed it (other lanes: +inf), or +inf
// everywhere if the hooks abandoned the pass.  *cells counts computed cells.
template <typename T, int R, int DMAX, class Hooks>
__device__ __forceinline__ T band_pass(const float *__restrict__ A, const float *__restrict__ B,
                                       int L, int D, int W, int v0, int v1, const Grp &g,
                                       Hooks &hooks, bool *abandoned, long long *cells) {
    const T INF = tinf<T>();
    T a[R][DMAX];
    T col[R];
    T bottom = INF, prev_in = INF, result = INF;
    T mn_prev = INF;
    int v = v0 + g.lig;
    const int vlast = (L - 1) / R;
    const int tau0 = v_jlo(v0, R, W) + v0;
    const int tau_end = v_jhi(v1 - 1, R, W, L) + (v1 - 1);
    bool loaded = false;
    long long ncell = 0;
    *abandoned = false;
    for (int tau = tau0; tau <= tau_end; ++tau) {
        T in = __shfl_sync(g.mask, bottom, g.src);
        if (v < v1 && tau > v_jhi(v, R, W, L) + v) {
            v += g.G;
            loaded = false;
        }
        int j = tau - v;
        bool active = v < v1 && j >= v_jlo(v, R, W) && j <= v_jhi(v, R, W, L);
        T step_min = INF;
        if (active) {
            if (!loaded) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    int i = v * R + r;
#pragma unroll
                    for (int p = 0; p < DMAX; ++p)
                        a[r][p] = (i < L && p < D) ? (T)__ldg(A + (size_t)i * D + p) : (T)0;
                    col[r] = INF;
                }
                loaded = true;
            }
            T b[DMAX];
#pragma unroll
            for (int p = 0; p < DMAX; ++p) b[p] = (p < D) ? (T)__ldg(B + (size_t)j * D + p) : (T)0;
            const int i0 = v * R;
            T up, diag;
            if (v == v0) {
                if (v0 == 0) {
                    up = INF;
                    diag = (j == 0) ? (T)0 : INF;
                } else {
                    up = (j <= i0 - 1 + W) ? hooks.template top<T>(j) : INF;
                    diag = (j >= 1 && j <= i0 + W) ? hooks.template top<T>(j - 1) : INF;
                }
            } else {
                up = (j <= i0 - 1 + W) ? in : INF;
                diag = (j >= 1 && j <= i0 + W) ? prev_in : INF;
            }
            // rows of this column inside the band: r in [j-W-i0, j+W-i0] and i < L
            const int rlo = j - W - i0, rhi = min(j + W - i0, L - 1 - i0);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                T left = col[r];
                T c = cell_cost<DMAX>(a[r], b);
                T m = tmin3(up, left, diag);
                bool valid = (r >= rlo) && (r <= rhi);
                T val = valid ? add_rn(c, m) : INF;
                diag = left;
                up = val;
                col[r] = val;
                if (Hooks::kCells && valid) hooks.cell_row(i0 + r, j, r, val);
                if (Hooks::kAbandon) step_min = step_min < val ? step_min : val;
            }
            bottom = col[R - 1];
            hooks.after_col(i0, j, bottom);
            ncell += max(0, min(rhi, R - 1) - max(rlo, 0) + 1);
            if (v == vlast && j == L - 1) {
                const int rl = (L - 1) - i0;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (r == rl) result = col[r];
            }
        }
        prev_in = in;
        if (Hooks::kAbandon) {
            T fm = mn_prev < step_min ? mn_prev : step_min;
            mn_prev = step_min;
            if (((tau - tau0) % kAbandonEvery) == kAbandonEvery - 1) {
                fm = grp_min(fm, g);
                if (hooks.abandon(fm)) {
                    *abandoned = true;
                    *cells = ncell;
                    return INF;
                }
            }
        }
    }
    *cells = ncell;
    return result;
}

// ============================================================= pairs forward
// Checkpoint layout: for pair p, nck = ceil(L/C)-1 rows; row k holds R(C*(k+1)-1, j)
// for j = i-W .. i+W at index j-i+W (2W+1 floats; entries outside [0,L) unused).
template <int R>
struct CkptHooks {
    float *ck;   // this pair's checkpoint rows, or null
    int C, W, L;
    static constexpr bool kAbandon = false;
    static constexpr bool kCells = false;
    template <typename T>
    __device__ __forceinline__ T top(int) const { return tinf<T>(); }
    template <typename T>
    __device__ __forceinline__ bool abandon(T) { return false; }
    __device__ __forceinline__ void cell_row(int, int, int, float) {}
    __device__ __forceinline__ void cell_row(int, int, int, double) {}
    // the bottom row i0+R-1 of a virtual lane is a checkpoint row when C | i0+R
    __device__ __forceinline__ void after_col(int i0, int j, float bottom) {
        const int i = i0 + R - 1;
        if (ck && ((i + 1) % C) == 0 && i + 1 < L && j >= i - W && j <= i + W)
            ck[(size_t)((i + 1) / C - 1) * (2 * W + 1) + (j - i + W)] = bottom;
    }
};

template <int R, int DMAX>
__global__ void __launch_bounds__(128) k_dtw_pairs(const float *__restrict__ A, const float *__restrict__ B,
                                                    int64_t P, int L, int D, int W, int G,
                                                    float *__restrict__ dist, float *__restrict__ ckpt,
                                                    int C) {
    Grp g = make_grp(G);
    const int groups_per_block = blockDim.x / G;
    const int64_t gid = (int64_t)blockIdx.x * groups_per_block + threadIdx.x / G;
    const int64_t stride = (int64_t)gridDim.x * groups_per_block;
    const int nv = (L + R - 1) / R;
    const int nck = (L + C - 1) / C - 1;
    for (int64_t p = gid; p < P; p += stride) {
        CkptHooks<R> h;
        h.ck = ckpt ? ckpt + (size_t)p * nck * (2 * W + 1) : nullptr;
        h.C = C; h.W = W; h.L = L;
        bool ab;
        long long cells;
        float r = band_pass<float, R, DMAX>(A + (size_t)p * L * D, B + (size_t)p * L * D, L, D, W, 0, nv,
                                            g, h, &ab, &cells);
        r = grp_min(r, g);
        if (g.lig == 0) dist[p] = r;
    }
}

// ============================================================= NN search (FP32)
struct NnHooks {
    const unsigned long long *bsf;  // this query's packed best-so-far
    float rho;
    static constexpr bool kAbandon = true;
    static constexpr bool kCells = false;
    template <typename T>
    __device__ __forceinline__ T top(int) const { return tinf<T>(); }
    __device__ __forceinline__ bool abandon(float fm) {
        return fm > prune_threshold(ld_volatile_u64(bsf), rho);
    }
    __device__ __forceinline__ bool abandon(double) { return false; }
    __device__ __forceinline__ void cell_row(int, int, int, float) {}
    __device__ __forceinline__ void cell_row(int, int, int, double) {}
    template <typename T>
    __device__ __forceinline__ void after_col(int, int, T) {}
};

// Entries e in [0, *count): pair (m = pairs[e] / N, n = pairs[e] % N); lb[e] is the
// entry's best lower bound (+inf = already pruned).  Writes dtw[e] (FP32 DTW, or
// +inf when pruned / abandoned) and lowers bsf[m].
template <int R, int DMAX>
__global__ void __launch_bounds__(128) k_dtw_nn(const float *__restrict__ Q, const float *__restrict__ Cand,
                                                 int L, int D, int W, int G, int64_t N,
                                                 const uint32_t *__restrict__ pairs, const float *__restrict__ lb,
                                                 const int32_t *__restrict__ count, int n_static, int *__restrict__ cursor,
                                                 unsigned long long *bsf, float rho, float *__restrict__ dtw,
                                                 unsigned long long *__restrict__ counters /* started, abandoned, cells, pruned */) {
    Grp g = make_grp(G);
    const int nv = (L + R - 1) / R;
    const int n_entries = count ? *count : n_static;
    unsigned long long started = 0, aband = 0, ncells = 0, pruned = 0;
    for (;;) {
        int e = 0;
        if (g.lig == 0) e = atomicAdd(cursor, 1);
        e = __shfl_sync(g.mask, e, (threadIdx.x & 31) & ~(G - 1));  // from the group's first lane
        if (e >= n_entries) break;
        const uint32_t pid = pairs[e];
        if (pid == 0xffffffffu) {
            if (g.lig == 0) dtw[e] = TC_INF;
            continue;
        }
        const int m = (int)(pid / (uint32_t)N);
        const int64_t n = (int64_t)(pid - (uint32_t)m * (uint32_t)N);
        const float lbe = lb ? lb[e] : 0.f;
        const float thr = prune_threshold(ld_volatile_u64(bsf + m), rho);
        if (!(lbe <= thr) || lbe == TC_INF) {
            if (g.lig == 0) { dtw[e] = TC_INF; if (lbe != TC_INF) ++pruned; }
            continue;
        }
        NnHooks h;
        h.bsf = bsf + m;
        h.rho = rho;
        bool ab;
        long long cells;
        float r = band_pass<float, R, DMAX>(Q + (size_t)m * L * D, Cand + (size_t)n * L * D, L, D, W, 0, nv, g, h,
                                            &ab, &cells);
        r = grp_min(r, g);
        long long cs = cells;
        for (int o = G >> 1; o > 0; o >>= 1) cs += __shfl_xor_sync(g.mask, cs, o);
        if (g.lig == 0) {
            ++started;
            ncells += (unsigned long long)cs;
            if (ab) {
                ++aband;
                dtw[e] = TC_INF;
            } else {
                dtw[e] = r;
                atomicMin(bsf + m, pack_best(r, (uint32_t)n));
            }
        }
    }
    if (g.lig == 0 && counters && (started | pruned)) {
        atomicAdd(counters + 0, started);
        atomicAdd(counters + 1, aband);
        atomicAdd(counters + 2, ncells);
        atomicAdd(counters + 3, pruned);
    }
}

// ============================================================= FP64 refine
// Entries e < *count: pair id as above; computes the FP64 DTW (bit-identical to a
// sequential FP64 evaluation of Eq. 1), stores it in d64[e] and lowers best64[m].
template <int R, int DMAX>
__global__ void __launch_bounds__(128) k_dtw_refine(const float *__restrict__ Q, const float *__restrict__ Cand,
                                                     int L, int D, int W, int G, int64_t N,
                                                     const uint32_t *__restrict__ pairs,
                                                     const int32_t *__restrict__ count, double *__restrict__ d64,
                                                     unsigned long long *__restrict__ best64) {
    Grp g = make_grp(G);
    const int nv = (L + R - 1) / R;
    const int groups_per_block = blockDim.x / G;
    const int gid = blockIdx.x * groups_per_block + threadIdx.x / G;
    const int stride = gridDim.x * groups_per_block;
    const int n_entries = *count;
    for (int e = gid; e < n_entries; e += stride) {
        const uint32_t pid = pairs[e];
        const int m = (int)(pid / (uint32_t)N);
        const int64_t n = (int64_t)(pid - (uint32_t)m * (uint32_t)N);
        NoHooks h;
        bool ab;
        long long cells;
        double r = band_pass<double, R, DMAX>(Q + (size_t)m * L * D, Cand + (size_t)n * L * D, L, D, W, 0, nv,
                                              g, h, &ab, &cells);
        r = grp_min(r, g);
        if (g.lig == 0) {
            d64[e] = r;
            atomicMin(best64 + m, (unsigned long long)__double_as_longlong(r));
        }
    }
}

// ============================================================= backward (adjoint)
// Segment hooks: store every computed cell of rows [row0, row0+C) into shared
// memory S[(i-row0+1)*(2W+1) + (j-i+W)]; the row above the segment comes from
// the checkpoint row, copied into S row 0.
struct SegHooks {
    float *S;
    int row0, W;
    static constexpr bool kAbandon = false;
    static constexpr bool kCells = true;
    template <typename T>
    __device__ __forceinline__ T top(int j) const {
        int i = row0 - 1;
        return S[(j - i + W)];
    }
    template <typename T>
    __device__ __forceinline__ bool abandon(T) { return false; }
    __device__ __forceinline__ void cell_row(int i, int j, int, float val) {
        S[(size_t)(i - row0 + 1) * (2 * W + 1) + (j - i + W)] = val;
    }
    __device__ __forceinline__ void cell_row(int, int, int, double) {}
    template <typename T>
    __device__ __forceinline__ void after_col(int, int, T) {}
};

// One group per pair.  Shared memory per group: (C+1) * (2W+1) floats.
template <int R, int DMAX>
__global__ void __launch_bounds__(128) k_dtw_backward(const float *__restrict__ A, const float *__restrict__ B,
                                                       const float *__restrict__ ckpt, int C,
                                                       const float *__restrict__ gdist, int64_t P, int L, int D,
                                                       int W, int G, float *__restrict__ gA, float *__restrict__ gB) {
    extern __shared__ float smem[];
    Grp g = make_grp(G);
    const int groups_per_block = blockDim.x / G;
    const int grp_in_block = threadIdx.x / G;
    const int BW = 2 * W + 1;
    float *S = smem + (size_t)grp_in_block * (C + 1) * BW;
    const int64_t gid = (int64_t)blockIdx.x * groups_per_block + grp_in_block;
    const int64_t stride = (int64_t)gridDim.x * groups_per_block;
    const int nseg = (L + C - 1) / C;
    const int nck = nseg - 1;
    constexpr int KD = (DMAX + 3) / 4;  // dims per lane (G >= 4)
    const float INF = TC_INF;
    for (int64_t p = gid; p < P; p += stride) {
        const float *a = A + (size_t)p * L * D;
        const float *b = B + (size_t)p * L * D;
        const float *ck = ckpt + (size_t)p * nck * BW;
        float *ga = gA + (size_t)p * L * D;
        float *gb = gB + (size_t)p * L * D;
        const float gscale = gdist[p];
        float acc_a[KD], acc_b[KD];
#pragma unroll
        for (int k = 0; k < KD; ++k) { acc_a[k] = 0.f; acc_b[k] = 0.f; }
        int ci = L - 1, cj = L - 1;  // path cursor
        bool done = false;
        for (int s = nseg - 1; s >= 0 && !done; --s) {
            const int row0 = s * C;
            const int row1 = min(L, row0 + C);
            // row above the segment
            for (int k = g.lig; k < BW; k += G) S[k] = (s == 0) ? INF : ck[(size_t)(s - 1) * BW + k];
            __syncwarp(g.mask);
            SegHooks h;
            h.S = S; h.row0 = row0; h.W = W;
            bool ab;
            long long cells;
            band_pass<float, R, DMAX>(a, b, L, D, W, row0 / R, (row1 + R - 1) / R, g, h, &ab, &cells);
            __syncwarp(g.mask);
            // backtrack through this segment
            while (ci >= row0) {
                // accumulate d/da_ci, d/db_cj
#pragma unroll
                for (int k = 0; k < KD; ++k) {
                    int pp = g.lig + k * G;
                    if (pp < D) {
                        float diff = a[(size_t)ci * D + pp] - b[(size_t)cj * D + pp];
                        acc_a[k] += 2.f * diff;
                        acc_b[k] -= 2.f * diff;
                    }
                }
                if (ci == 0 && cj == 0) { done = true; break; }
                // predecessor values (row ci-1 may be the checkpoint row in S row 0)
                auto Rv = [&](int i, int j) -> float {
                    if (i < 0 || j < 0 || abs(i - j) > W) return INF;
                    return S[(size_t)(i - row0 + 1) * BW + (j - i + W)];
                };
                float vd = Rv(ci - 1, cj - 1), vu = Rv(ci - 1, cj), vl = Rv(ci, cj - 1);
                int ni = ci - 1, nj = cj - 1;
                float best = vd;
                if (vu < best) { best = vu; ni = ci - 1; nj = cj; }
                if (vl < best) { best = vl; ni = ci; nj = cj - 1; }
                if (ni != ci) {  // leaving row ci
#pragma unroll
                    for (int k = 0; k < KD; ++k) {
                        int pp = g.lig + k * G;
                        if (pp < D) ga[(size_t)ci * D + pp] = gscale * acc_a[k];
                        acc_a[k] = 0.f;
                    }
                }
                if (nj != cj) {  // leaving column cj
#pragma unroll
                    for (int k = 0; k < KD; ++k) {
                        int pp = g.lig + k * G;
                        if (pp < D) gb[(size_t)cj * D + pp] = gscale * acc_b[k];
                        acc_b[k] = 0.f;
                    }
                }
                ci = ni;
                cj = nj;
            }
            __syncwarp(g.mask);
        }
        // flush row 0 / column 0
#pragma unroll
        for (int k = 0; k < KD; ++k) {
            int pp = g.lig + k * G;
            if (pp < D) {
                ga[pp] = gscale * acc_a[k];
                gb[pp] = gscale * acc_b[k];
            }
        }
        __syncwarp(g.mask);
    }
}

// ============================================================= host dispatch
namespace {
template <int R, int DMAX>
struct TileKernels {
    static cudaError_t pairs(dim3 grid, dim3 block, cudaStream_t s, const float *A, const float *B, int64_t P, int L,
                             int D, int W, int G, float *dist, float *ck, int C) {
        k_dtw_pairs<R, DMAX><<<grid, block, 0, s>>>(A, B, P, L, D, W, G, dist, ck, C);
        return cudaGetLastError();
    }
    static cudaError_t nn(dim3 grid, dim3 block, cudaStream_t s, const DtwNnArgs &x) {
        k_dtw_nn<R, DMAX><<<grid, block, 0, s>>>(x.Q, x.C, x.L, x.D, x.W, x.G, x.N, x.pairs, x.lb, x.count, x.n_static, x.cursor,
                                                 x.bsf, x.rho, x.dtw, x.counters);
        return cudaGetLastError();
    }
    static cudaError_t refine(dim3 grid, dim3 block, cudaStream_t s, const DtwRefineArgs &x) {
        k_dtw_refine<R, DMAX><<<grid, block, 0, s>>>(x.Q, x.C, x.L, x.D, x.W, x.G, x.N, x.pairs, x.count, x.d64,
                                                     x.best64);
        return cudaGetLastError();
    }
    static cudaError_t backward(dim3 grid, dim3 block, size_t smem, cudaStream_t s, const float *A, const float *B,
                                const float *ck, int C, const float *gd, int64_t P, int L, int D, int W, int G,
                                float *gA, float *gB) {
        if (smem > 227 * 1024) return cudaErrorInvalidValue;
        auto k = k_dtw_backward<R, DMAX>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k<<<grid, block, smem, s>>>(A, B, ck, C, gd, P, L, D, W, G, gA, gB);
        return cudaGetLastError();
    }
    static int occupancy_pairs() {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_dtw_pairs<R, DMAX>, 128, 0);
        return n;
    }
    static int occupancy_nn() {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_dtw_nn<R, DMAX>, 128, 0);
        return n;
    }
};
}  // namespace

#define TC_TILE_CASE(id, R, DMAX) \
    case id:                      \
        return TileKernels<R, DMAX>::

cudaError_t dtw_pairs_launch(int tile, int G, int blocks, cudaStream_t s, const float *A, const float *B, int64_t P,
                             int L, int D, int W, float *dist, float *ck, int C) {
    dim3 grid(blocks), block(128);
    switch (tile) {
#define X(id, R, DMAX) TC_TILE_CASE(id, R, DMAX) pairs(grid, block, s, A, B, P, L, D, W, G, dist, ck, C);
        TC_TILES(X)
#undef X
    }
    return cudaErrorInvalidValue;
}
cudaError_t dtw_nn_launch(int tile, int blocks, cudaStream_t s, const DtwNnArgs &x) {
    dim3 grid(blocks), block(128);
    switch (tile) {
#define X(id, R, DMAX) TC_TILE_CASE(id, R, DMAX) nn(grid, block, s, x);
        TC_TILES(X)
#undef X
    }
    return cudaErrorInvalidValue;
}
cudaError_t dtw_refine_launch(int tile, int blocks, cudaStream_t s, const DtwRefineArgs &x) {
    dim3 grid(blocks), block(128);
    switch (tile) {
#define X(id, R, DMAX) TC_TILE_CASE(id, R, DMAX) refine(grid, block, s, x);
        TC_TILES(X)
#undef X
    }
    return cudaErrorInvalidValue;
}
cudaError_t dtw_backward_launch(int tile, int G, int blocks, size_t smem, cudaStream_t s, const float *A,
                                const float *B, const float *ck, int C, const float *gd, int64_t P, int L, int D,
                                int W, float *gA, float *gB, int threads) {
    dim3 grid(blocks), block(threads);
    switch (tile) {
#define X(id, R, DMAX) TC_TILE_CASE(id, R, DMAX) backward(grid, block, smem, s, A, B, ck, C, gd, P, L, D, W, G, gA, gB);
        TC_TILES(X)
#undef X
    }
    return cudaErrorInvalidValue;
}
int dtw_occupancy(int tile, int which) {
    switch (tile) {
#define X(id, R, DMAX) \
    case id:           \
        return which == 0 ? TileKernels<R, DMAX>::occupancy_pairs() : TileKernels<R, DMAX>::occupancy_nn();
        TC_TILES(X)
#undef X
    }
    return 0;
}

}  // namespace tc
