// dtw_core.cuh -- banded DTW dynamic programme (Eq. 1 with the Sakoe-Chiba window,
// Section 2) on sm_103a: device code and kernel templates, instantiated per band
// tile by dtw_inst_*.cu.
//
// Work decomposition ("row-block systolic sweep").  A group of G lanes (G = 4, 8,
// 16 or 32, several groups per warp) computes one pair.  The L rows are cut into
// "virtual lanes" of R consecutive rows; virtual lane v (rows vR .. vR+R-1) visits
// the columns of its band, j in [vR-W, vR+R-1+W] clipped to [0, L-1], one column
// per time step, and computes all R cells of that column from R query points held
// in registers and one candidate point loaded per step (so each loaded candidate
// point serves R cells).  Virtual lane v processes column j at time t = j + v,
// exactly one step after virtual lane v-1 did, so the only value crossing lanes per
// step is the bottom cell of the lane above, passed with one shuffle.  Physical lane
// l of the group runs virtual lanes l, l+G, l+2G, ...; they never overlap in time
// when G*(R+1) >= 2W+R, which the host checks when it picks a tile.
//
// The squared-Euclidean cell costs of two adjacent rows are computed together with
// packed f32x2 subtract / fused multiply-add (two cells per instruction, each cell
// rounded exactly as a scalar fmaf chain); the recurrence uses the three-input min.
//
// Early abandoning (Section 7.1).  Define tau(i,j) = floor(i/R) + j.  Along any
// warping path tau grows by 0, 1 or 2 per step, so every path from (0,0) to
// (L-1,L-1) has a cell with tau in {t-1, t}; along the backtracked argmin path the
// computed values never decrease.  Hence if every cell computed at times t-1 and t
// exceeds the threshold, so does the final value, and the pair can be dropped.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "dtw_tiles.cuh"

namespace tc {

// ------------------------------------------------------------------ packed FP32 pairs
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// max that returns NaN when either operand is NaN (a NaN cost stays NaN, as with a select)
__device__ __forceinline__ float max_nan(float a, float b) {
    float r;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// ------------------------------------------------------------------ cp.async staging
__device__ __forceinline__ void cp_async_4(float *smem, const float *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_16(float *smem, const float *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// 0, computed from v in a way the compiler cannot see through: a copy whose
// destination depends on it cannot be issued before v (a shared-memory read) is in.
__device__ __forceinline__ unsigned opaque_zero(float v) {
    unsigned z;
    asm volatile("and.b32 %0, %1, 0;" : "=r"(z) : "r"(__float_as_uint(v)));
    return z;
}
// Copy rows [i0, i0+nrows) of a [L][D] series (contiguous nrows*D floats) to dst.
// vec4: the block starts 16-byte aligned and nrows*D is a multiple of 4 when
// nrows == R; a shorter last block falls back to 4-byte copies.
__device__ __forceinline__ void stage_rows(float *dst, const float *A, int i0, int nrows, int D, bool vec4) {
    const float *src = A + (size_t)i0 * D;
    const int n = nrows * D;
    if (vec4 && (n % 4) == 0 && ((((uintptr_t)src) & 15) == 0)) {
        for (int k = 0; k < n; k += 4) cp_async_16(dst + k, src + k);
    } else {
        for (int k = 0; k < n; ++k) cp_async_4(dst + k, src + k);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Lane-group geometry inside a warp.
struct Grp {
    int G;          // lanes per group
    int lig;        // lane index in group
    unsigned mask;  // lanes of this group
    int src;        // warp lane of the predecessor (cyclic) in the group
    int first;      // warp lane of the group's first lane
};
__device__ __forceinline__ Grp make_grp(int G) {
    Grp g;
    const int lane = threadIdx.x & 31;
    g.G = G;
    g.lig = lane & (G - 1);
    g.first = lane - g.lig;
    g.mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << g.first);
    g.src = g.first + ((g.lig + G - 1) & (G - 1));
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

// Rows r in [lo, hi] of [0, R) as a bit mask (empty if lo > hi after clipping).
__device__ __forceinline__ unsigned row_mask(int lo, int hi, int R) {
    lo = max(lo, 0);
    hi = min(hi, R - 1);
    if (lo > hi) return 0u;
    return (0xffffffffu >> (31 - hi)) & (0xffffffffu << lo);
}

// Steps between two abandon checks (a power of two).  Each check costs a group-wide
// minimum and a read of the best-so-far; a pair is dropped at most that many steps later
// than it could be.  Measured on GB300: 16 for narrow points, 32 for wide ones (whose
// steps are longer) beat 8 by 1% and 4% of the search's DTW stage.
__host__ __device__ constexpr int abandon_every(int DM) { return DM >= 16 ? 32 : 16; }

// ------------------------------------------------------------------ column / row rings
// Wide points (DM >= 16) are costly to fetch per lane and step: each lane
// of a group reads a different candidate point, so a warp-wide load touches 32
// different cache lines.  In the ring variant (kRing) every lane group keeps in shared
// memory a ring of the candidate columns its lanes are about to read (RC slots of
// ring_stride(DM) floats) and a ring of the query rows of its next virtual lanes
// (kRingRows slots of R*DM floats).  Every kRingFill steps the group fills both with
// coalesced cp.async copies for the steps of the next kRingAhead periods (a prologue
// covers the first periods), then waits for the fills of kRingAhead periods ago (the
// candidates stream from HBM: the lookahead covers its latency, and the fill
// bookkeeping, commit, wait and warp barriers run once per period).  Reads then hit
// shared memory: a float4 per four dimensions, conflict-free across consecutive columns
// because the slot stride is an odd number of 16-byte units.
// Sizes (checked against the exact schedule for every small (L, W, R, G)): at most G
// virtual lanes are active at a time, so the columns in use at step t and those filled
// at t for up to kRingFill*(kRingAhead+1) - 1 steps ahead span fewer than
// kRingFill*(kRingAhead+1) + G slots; virtual lanes start at most one per step, so
// kRingFill*(kRingAhead+1) row slots suffice.
constexpr int kRingFill = 8;
constexpr int kRingAhead = 1;
constexpr int kRingRows = 16;
static_assert(kRingRows >= kRingFill * (kRingAhead + 1), "row ring too small");
__host__ __device__ constexpr int ring_stride(int DM) { return ((DM / 4) & 1) ? DM + 8 : DM + 4; }
// The (R = 6, DM = 32) tile keeps the last ring_smem_rows(R, DM) of its 6 rows in a
// lane-private shared-memory slot (G*DM floats per row and group, [row][DM/4][G] float4 so
// a quarter warp reads 128 contiguous bytes) instead of 32 registers per row: at 192
// registers of rows the search kernel ran at the 255-register cap with dependent
// instructions issued back to back, and with the slot the scheduler has room to overlap
// them (one more float4 load per row and 4 dimensions; ncu on GB300: issue 42 -> 49%
// active, FMA pipe 46 -> 55%, the search's DTW stage 408 -> 364 ms per 256 queries at
// L = 2,048, W = 102).
__host__ __device__ constexpr int ring_smem_rows(int R, int DM) { return (DM == 32 && R == 6) ? 1 : 0; }
__host__ __device__ constexpr int ring_cols(int G) {
    return (kRingFill * (kRingAhead + 1) + G) <= 16   ? 16
           : (kRingFill * (kRingAhead + 1) + G) <= 32 ? 32
                                                       : 64;
}
__host__ __device__ constexpr int ring_group_floats(int R, int DM, int G) {
    return ring_cols(G) * ring_stride(DM) + kRingRows * R * DM + ring_smem_rows(R, DM) * G * DM;
}
// Band table of the row-slot tile (one per block, after the groups' rings): whether row r
// of a virtual lane is inside the band at column j depends only on dj = j - i0, so entry
// dj + W (0 <= dj + W < 2W + R) holds the cost floor of each row (0 inside the band, +inf
// outside: a max of cost and floor replaces a bit test and a select per row) and the number of
// rows inside, read with two float4 loads per step.  Rows past the end of the series
// (the last virtual lane when R does not divide L) take the exact row mask instead.
// Space is kept for G(R+1) >= 2W+R entries, the most a valid (tile, G) can need.
__host__ __device__ constexpr bool ring_band_table(int R, int DM) { return ring_smem_rows(R, DM) > 0 && R <= 7; }
constexpr int kBandEntry = 8;  // floats per entry: R floors, the row count (int bits), padding
__host__ __device__ constexpr size_t band_table_bytes(int R, int DM, int G) {
    return ring_band_table(R, DM) ? (size_t)G * (R + 1) * kBandEntry * sizeof(float) : 0;
}
// shared memory of a 128-thread block of the ring variant: the groups' rings, then the
// band table
__host__ __device__ constexpr size_t ring_block_bytes(int R, int DM, int G) {
    return (size_t)(128 / G) * ring_group_floats(R, DM, G) * sizeof(float) + band_table_bytes(R, DM, G);
}
__device__ __forceinline__ void cp_async_wait_ahead() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kRingAhead) : "memory");
}
// smallest virtual lane still active at step T (v0 = 0), and largest started by T
__device__ __forceinline__ int ring_vmin(int T, int R, int W, int L) {
    const int x = T - R + 1 - W;
    const int a = x <= 0 ? 0 : (x + R) / (R + 1);
    return max(a, T - L + 1);
}
__device__ __forceinline__ int ring_vmax(int T, int R, int W, int v1) {
    return min(v1 - 1, min(T, (T + W) / (R + 1)));
}
// Copy n floats from src (global) to dst (shared) with the lanes of a group.
__device__ __forceinline__ void ring_copy(float *dst, const float *src, int n, bool vec, const Grp &g) {
    if (vec) {
        for (int p = g.lig * 4; p < n; p += 4 * g.G) cp_async_16(dst + p, src + p);
    } else {
        for (int p = g.lig; p < n; p += g.G) cp_async_4(dst + p, src + p);
    }
}
// Issue the fills needed up to step T: columns [*col_hi, c_end) and the rows of virtual
// lanes [*v_hi, v_end).
template <int R, int DM>
__device__ __forceinline__ void ring_fill(float *rcols, float *rrows, int RC, const float *A, const float *B, int L,
                                          int D, int W, int v1, int T, int *col_hi, int *v_hi, bool vec,
                                          const Grp &g) {
    constexpr int DMS = ring_stride(DM);
    constexpr int SEG = DM / 4;  // 16-byte segments of a slot row (a power of two)
    const int c_end = min(L, T - ring_vmin(T, R, W, L) + 1);
    const int v_end = min(v1, ring_vmax(T, R, W, v1) + 1);
    if (vec) {
        // one (point, 16-byte segment) item per lane and pass, over all the points of
        // the fill: the new columns, then the rows of the new virtual lanes (consecutive
        // query rows), so that every lane copies rather than one point per pass
        const int segs = D >> 2, c0 = *col_hi, nc = c_end > c0 ? c_end - c0 : 0;
        for (int k = g.lig; k < nc * SEG; k += g.G) {
            const int c = c0 + k / SEG, s = k % SEG;
            if (s < segs) cp_async_16(rcols + (c & (RC - 1)) * DMS + 4 * s, B + (size_t)c * D + 4 * s);
        }
        const int r0 = *v_hi * R, r1 = min(v_end * R, L), nr = r1 > r0 ? r1 - r0 : 0;
        for (int k = g.lig; k < nr * SEG; k += g.G) {
            const int row = r0 + k / SEG, s = k % SEG;
            if (s < segs)
                cp_async_16(rrows + ((row / R) & (kRingRows - 1)) * R * DM + (row % R) * DM + 4 * s,
                            A + (size_t)row * D + 4 * s);
        }
    } else {
        for (int c = *col_hi; c < c_end; ++c)
            ring_copy(rcols + (c & (RC - 1)) * DMS, B + (size_t)c * D, D, vec, g);
        for (int vv = *v_hi; vv < v_end; ++vv) {
            float *dst = rrows + (vv & (kRingRows - 1)) * R * DM;
            const int nr = min(R, L - vv * R);
            for (int r = 0; r < nr; ++r) ring_copy(dst + r * DM, A + (size_t)(vv * R + r) * D, D, vec, g);
        }
    }
    if (c_end > *col_hi) *col_hi = c_end;
    if (v_end > *v_hi) *v_hi = v_end;
}

// Hook sets.  top(j): row above the first virtual lane of a pass (v0 > 0).
// cell(i, j, val): every in-band cell (kCells).  after_col(i0, j, bottom): once per
// computed column of a virtual lane.  abandon(m): every abandon_every(DM) steps with the
// group-wide frontier minimum (kAbandon).
struct NoHooks {
    static constexpr bool kAbandon = false;
    static constexpr bool kCells = false;
    __device__ __forceinline__ float top(int) const { return TC_INF; }
    __device__ __forceinline__ bool abandon(float) { return false; }
    __device__ __forceinline__ void cell(int, int, float) {}
    __device__ __forceinline__ void after_col(int, int, float) {}
};

// One pass of the band DP over virtual lanes [v0, v1) of one pair.
//   A: rows series [L][D] (float32), B: columns series.
//   v0 > 0: the row above (v0*R-1) comes from hooks.top(j); v0 == 0: the DP origin.
// Returns R(L-1, L-1) on the lane that computed it (other lanes: +inf), or +inf
// on every lane of a group whose hooks abandoned the pass.  *cells counts cells.
// All lanes of g.mask must call band_pass together: with g.mask covering the whole
// warp (lockstep kernels) every group of the warp runs the same time loop; a group
// with live == false only takes part in the shuffles.  An abandoned group turns
// idle; the loop ends early once no lane under g.mask has work left.
// stage (may be null): this lane's shared-memory slot of R*D floats, used to copy
// the rows of the lane's next virtual lane with cp.async while it works on the
// current one (a virtual-lane start then reads shared memory, not global memory).
// kRing (wide points only, v0 == 0): candidate columns and query rows come from the
// group's rings at `ring` (ring_group_floats(R, DM, G) floats, RC = ring_cols(G) column
// slots, the dimensions D..DM-1 of every slot zero); all lanes of the warp call it.  The
// last ring_smem_rows(R, DM) rows of a lane's virtual lane are copied from the row ring to
// the lane's private slot after the rings (read there every step), the other rows to
// registers.
template <int R, int DM, class Hooks, bool kRing = false>
__device__ __forceinline__ float band_pass(const float *__restrict__ A, const float *__restrict__ B, int L, int D,
                                           int W, int v0, int v1, const Grp &g, Hooks &hooks, bool live,
                                           bool *abandoned, long long *cells, float *stage = nullptr,
                                           float *ring = nullptr, int RC = 0, const float *band = nullptr) {
    const bool stage_vec4 = (((uintptr_t)A) & 15) == 0;
    static_assert(R % 2 == 0, "rows are processed in pairs");
    static_assert(!kRing || (DM >= 16 && DM % 4 == 0), "rings hold float4-aligned wide points");
    constexpr int RP = R / 2;
    const float INF = TC_INF;
    constexpr bool kDimPack = DM >= 16;
    constexpr int DH = (DM + 1) / 2;
    f2 a2[kDimPack ? 1 : RP][kDimPack ? 1 : DM];     // rows (2k, 2k+1) of the virtual lane, dimension p
    constexpr int RSM = kRing ? ring_smem_rows(R, DM) : 0;
    constexpr int RREG = R - RSM;
    f2 ad[kDimPack ? RREG : 1][kDimPack ? DH : 1];      // wide points: row r, dimensions (2h, 2h+1)
    float col[R];      // R(i0 + r, j-1) -> R(i0 + r, j)
    float b[DM];
    float bottom = INF, prev_in = INF, result = INF, mn_prev = INF;
    int v = live ? v0 + g.lig : v1;
    const int vlast = (L - 1) / R;
    const int tau0 = v_jlo(v0, R, W) + v0;
    const int tau_end = v_jhi(v1 - 1, R, W, L) + (v1 - 1);
    bool dead = !live;
    // current virtual lane: active for tau in [tlo, thi]
    int tlo = v < v1 ? v_jlo(v, R, W) + v : 1 << 30;
    int thi = v < v1 ? v_jhi(v, R, W, L) + v : -1;
    bool loaded = false, staged = false;
    int ncell = 0;  // statistics only; 32 bits hold a lane's cells for L < 10^8
    *abandoned = false;
    float *rcols = ring, *rrows = ring + (kRing ? RC * ring_stride(DM) : 0);
    float *rpriv = RSM ? rrows + kRingRows * R * DM + 4 * g.lig : nullptr;
    int col_hi = 0, v_hi = 0;
    const bool ring_vec = ((D & 3) == 0) && (((((uintptr_t)A) | ((uintptr_t)B)) & 15) == 0);
    if (kRing) {
        // prologue: everything the first kRingAhead periods read, complete before the loop
        if (!dead)
            ring_fill<R, DM>(rcols, rrows, RC, A, B, L, D, W, v1, tau0 + kRingFill * kRingAhead - 1, &col_hi, &v_hi,
                             ring_vec, g);
        cp_async_wait_all();
        __syncwarp();
    }
    for (int tau = tau0; tau <= tau_end; ++tau) {
        if (kRing && ((tau - tau0) & (kRingFill - 1)) == 0) {
            __syncwarp();  // the earlier steps' reads of the slots refilled below are done
            if (!dead)
                ring_fill<R, DM>(rcols, rrows, RC, A, B, L, D, W, v1, tau + kRingFill * (kRingAhead + 1) - 1, &col_hi,
                                 &v_hi, ring_vec, g);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            cp_async_wait_ahead();  // the fills of kRingAhead periods ago cover this period
            __syncwarp();
        }
        const float in = __shfl_sync(g.mask, bottom, g.src);
        if (tau > thi && v < v1) {
            v += g.G;
            loaded = false;
            tlo = v < v1 ? v_jlo(v, R, W) + v : 1 << 30;
            thi = v < v1 ? v_jhi(v, R, W, L) + v : -1;
        }
        float step_min = INF;
        if (tau >= tlo && tau <= thi) {
            const int j = tau - v;
            const int i0 = v * R;
            if (!loaded) {
                if (staged && !kDimPack) {
                    // rows were copied to this lane's shared slot one virtual lane ago
                    cp_async_wait_all();
#pragma unroll
                    for (int k = 0; k < RP; ++k) {
                        const int i = i0 + 2 * k;
#pragma unroll
                        for (int p = 0; p < DM; ++p) {
                            const float lo = (i < L && p < D) ? stage[(2 * k) * D + p] : 0.f;
                            const float hi = (i + 1 < L && p < D) ? stage[(2 * k + 1) * D + p] : 0.f;
                            a2[k][p] = pk(lo, hi);
                        }
                    }
                } else if (!kDimPack) {
#pragma unroll
                    for (int k = 0; k < RP; ++k) {
                        const int i = i0 + 2 * k;
#pragma unroll
                        for (int p = 0; p < DM; ++p) {
                            const float lo = (i < L && p < D) ? __ldg(A + (size_t)i * D + p) : 0.f;
                            const float hi = (i + 1 < L && p < D) ? __ldg(A + (size_t)(i + 1) * D + p) : 0.f;
                            a2[k][p] = pk(lo, hi);
                        }
                    }
                }
                if (kDimPack && kRing) {
                    const float *rr = rrows + (v & (kRingRows - 1)) * R * DM;
#pragma unroll
                    for (int r = 0; r < RREG; ++r) {
#pragma unroll
                        for (int k = 0; k < DM / 4; ++k) {
                            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (i0 + r < L) x = *reinterpret_cast<const float4 *>(rr + r * DM + 4 * k);
                            ad[kDimPack ? r : 0][kDimPack ? 2 * k : 0] = pk(x.x, x.y);
                            ad[kDimPack ? r : 0][kDimPack ? 2 * k + 1 : 0] = pk(x.z, x.w);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < RSM; ++q) {
#pragma unroll
                        for (int k = 0; k < DM / 4; ++k) {
                            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (i0 + RREG + q < L)
                                x = *reinterpret_cast<const float4 *>(rr + (RREG + q) * DM + 4 * k);
                            *reinterpret_cast<float4 *>(rpriv + (q * (DM / 4) + k) * 4 * g.G) = x;
                        }
                    }
                } else if (kDimPack) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int i = i0 + r;
#pragma unroll
                        for (int h = 0; h < DH; ++h) {
                            const float x0 = (i < L && 2 * h < D) ? __ldg(A + (size_t)i * D + 2 * h) : 0.f;
                            const float x1 = (i < L && 2 * h + 1 < D) ? __ldg(A + (size_t)i * D + 2 * h + 1) : 0.f;
                            ad[kDimPack ? r : 0][kDimPack ? h : 0] = pk(x0, x1);
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < R; ++r) col[r] = INF;
                loaded = true;
                // start copying the rows of this lane's next virtual lane (after the
                // reads of the slot above have completed: opaque data dependency)
                const bool had = staged;
                staged = false;
                if (!kDimPack && stage && v + g.G < v1) {
                    float last_lo, last_hi;
                    upk(a2[RP - 1][DM - 1], last_lo, last_hi);
                    const unsigned z = had ? opaque_zero(last_hi) : 0u;
                    stage_rows(stage + z, A, (v + g.G) * R, min(R, L - (v + g.G) * R), D, stage_vec4);
                    staged = true;
                }
            }
            f2 cs[kDimPack ? R : 1];
            if (kDimPack && kRing) {
                // the column from the ring, four dimensions per shared-memory load
                const float *bc = rcols + (j & (RC - 1)) * ring_stride(DM);
#pragma unroll
                for (int r = 0; r < R; ++r) cs[kDimPack ? r : 0] = 0ull;
#pragma unroll
                for (int k = 0; k < DM / 4; ++k) {
                    const float4 x = *reinterpret_cast<const float4 *>(bc + 4 * k);
                    const f2 b0 = pk(x.x, x.y), b1 = pk(x.z, x.w);
#pragma unroll
                    for (int r = 0; r < RREG; ++r) {
                        const f2 t0 = sub2(ad[kDimPack ? r : 0][kDimPack ? 2 * k : 0], b0);
                        cs[kDimPack ? r : 0] = fma2(t0, t0, cs[kDimPack ? r : 0]);
                        const f2 t1 = sub2(ad[kDimPack ? r : 0][kDimPack ? 2 * k + 1 : 0], b1);
                        cs[kDimPack ? r : 0] = fma2(t1, t1, cs[kDimPack ? r : 0]);
                    }
#pragma unroll
                    for (int q = 0; q < RSM; ++q) {
                        const float4 y = *reinterpret_cast<const float4 *>(rpriv + (q * (DM / 4) + k) * 4 * g.G);
                        const f2 t0 = sub2(pk(y.x, y.y), b0);
                        cs[kDimPack ? RREG + q : 0] = fma2(t0, t0, cs[kDimPack ? RREG + q : 0]);
                        const f2 t1 = sub2(pk(y.z, y.w), b1);
                        cs[kDimPack ? RREG + q : 0] = fma2(t1, t1, cs[kDimPack ? RREG + q : 0]);
                    }
                }
            } else if (kDimPack) {
                // the column two dimensions at a time, each pair used by all R rows
#pragma unroll
                for (int r = 0; r < R; ++r) cs[kDimPack ? r : 0] = 0ull;
#pragma unroll
                for (int h = 0; h < DH; ++h) {
                    const float x0 = (2 * h < D) ? __ldg(B + (size_t)j * D + 2 * h) : 0.f;
                    const float x1 = (2 * h + 1 < D) ? __ldg(B + (size_t)j * D + 2 * h + 1) : 0.f;
                    const f2 bh = pk(x0, x1);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const f2 t = sub2(ad[kDimPack ? r : 0][kDimPack ? h : 0], bh);
                        cs[kDimPack ? r : 0] = fma2(t, t, cs[kDimPack ? r : 0]);
                    }
                }
            } else {
#pragma unroll
                for (int p = 0; p < DM; ++p) b[p] = (p < D) ? __ldg(B + (size_t)j * D + p) : 0.f;
            }
            float up, diag;
            if (v == v0) {
                if (v0 == 0) {
                    up = INF;
                    diag = (j == 0) ? 0.f : INF;
                } else {
                    up = (j <= i0 - 1 + W) ? hooks.top(j) : INF;
                    diag = (j >= 1 && j <= i0 + W) ? hooks.top(j - 1) : INF;
                }
            } else {
                up = (j <= i0 - 1 + W) ? in : INF;
                diag = (j >= 1 && j <= i0 + W) ? prev_in : INF;
            }
            // rows of this column inside the band: r in [j-W-i0, j+W-i0] and i < L
            // (the search kernel keeps the row mask: with its abandoning state the table's
            // floors took it from 248 to 255 registers and 4% longer; the pairs kernel runs
            // 7% faster with the table)
            constexpr bool kTable = kRing && ring_band_table(R, DM) && !Hooks::kCells && !Hooks::kAbandon;
            unsigned vm = 0u;
            float floor_r[kTable ? R : 1];
            int nin = 0;
            if (kTable && i0 + R <= L) {
                const float *be = band + (j - i0 + W) * kBandEntry;
                const float4 ba = *reinterpret_cast<const float4 *>(be);
                const float4 bb4 = *reinterpret_cast<const float4 *>(be + 4);
                const float fl[8] = {ba.x, ba.y, ba.z, ba.w, bb4.x, bb4.y, bb4.z, bb4.w};
#pragma unroll
                for (int r = 0; r < (kTable ? R : 1); ++r) floor_r[r] = fl[r];
                nin = __float_as_int(fl[kTable ? R : 1]);
            } else {
                vm = row_mask(j - W - i0, min(j + W - i0, L - 1 - i0), R);
                if (kTable) {
#pragma unroll
                    for (int r = 0; r < (kTable ? R : 1); ++r) floor_r[r] = ((vm >> r) & 1u) ? 0.f : INF;
                }
                nin = __popc(vm);
            }
            f2 bb[kDimPack ? 1 : DM];
            if (!kDimPack) {
#pragma unroll
                for (int p = 0; p < DM; ++p) bb[kDimPack ? 0 : p] = pk(b[p], b[p]);
            }
#pragma unroll
            for (int k = 0; k < RP; ++k) {
                float c0, c1;
                if (kDimPack) {
                    float x, y;
                    upk(cs[kDimPack ? 2 * k : 0], x, y);
                    c0 = __fadd_rn(x, y);
                    upk(cs[kDimPack ? 2 * k + 1 : 0], x, y);
                    c1 = __fadd_rn(x, y);
                } else {
                    f2 s = 0ull;
#pragma unroll
                    for (int p = 0; p < DM; ++p) {
                        const f2 t = sub2(a2[k][p], bb[p]);
                        s = fma2(t, t, s);
                    }
                    upk(s, c0, c1);
                }
                // row 2k
                // cells outside the band get cost +inf (so the value is +inf), which keeps
                // the masking off the row-to-row dependency chain
                if (kTable) {
                    c0 = max_nan(c0, floor_r[kTable ? 2 * k : 0]);
                    c1 = max_nan(c1, floor_r[kTable ? 2 * k + 1 : 0]);
                } else {
                    c0 = ((vm >> (2 * k)) & 1u) ? c0 : INF;
                    c1 = ((vm >> (2 * k + 1)) & 1u) ? c1 : INF;
                }
                float left = col[2 * k];
                float val = __fadd_rn(c0, min3f(up, left, diag));
                diag = left;
                up = val;
                col[2 * k] = val;
                if (Hooks::kCells && ((vm >> (2 * k)) & 1u)) hooks.cell(i0 + 2 * k, j, val);
                // row 2k+1
                float left1 = col[2 * k + 1];
                float val1 = __fadd_rn(c1, min3f(up, left1, diag));
                diag = left1;
                up = val1;
                col[2 * k + 1] = val1;
                if (Hooks::kCells && ((vm >> (2 * k + 1)) & 1u)) hooks.cell(i0 + 2 * k + 1, j, val1);
                if (Hooks::kAbandon) step_min = min3f(step_min, val, val1);
            }
            bottom = col[R - 1];
            hooks.after_col(i0, j, bottom);
            ncell += nin;
        }
        prev_in = in;
        if (Hooks::kAbandon) {
            float fm = fminf(mn_prev, step_min);
            mn_prev = step_min;
            if (((tau - tau0) & (abandon_every(DM) - 1)) == abandon_every(DM) - 1) {
                fm = grp_min(fm, g);
                if (!dead && hooks.abandon(fm)) {
                    dead = true;
                    *abandoned = true;
                    v = v1;  // no more work for this group
                    tlo = 1 << 30;
                    thi = -1;
                }
                if (__all_sync(g.mask, dead)) break;
            }
        }
    }
    *cells = ncell;
    if (kRing) {
        // no fill of this pair may land after the next pair's fills of the same slots
        cp_async_wait_all();
        __syncwarp();
    }
    // R(L-1, L-1): the last cell of the last virtual lane, still in its lane's column
    // registers (the lane computes nothing after that virtual lane's last column)
    if (!*abandoned && live && ((vlast - v0) % g.G) == g.lig && vlast >= v0 && vlast < v1) {
        const int rl = (L - 1) - vlast * R;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (r == rl) result = col[r];
    }
    return *abandoned ? INF : result;
}

// ============================================================= pairs forward
// Checkpoint layout: for pair p, nck = ceil(L/C)-1 rows; row k holds R(C*(k+1)-1, j)
// for j = i-W .. i+W at index j-i+W (2W+1 floats; entries outside [0,L) unused).
template <int R>
struct CkptHooks {
    float *ck;  // this pair's checkpoint rows, or null
    int C, W, L;
    static constexpr bool kAbandon = false;
    static constexpr bool kCells = false;
    __device__ __forceinline__ float top(int) const { return TC_INF; }
    __device__ __forceinline__ bool abandon(float) { return false; }
    __device__ __forceinline__ void cell(int, int, float) {}
    // the bottom row i0+R-1 of a virtual lane is a checkpoint row when C | i0+R
    __device__ __forceinline__ void after_col(int i0, int j, float bottom) {
        const int i = i0 + R - 1;
        if (ck && ((i + 1) % C) == 0 && i + 1 < L && j >= i - W && j <= i + W)
            ck[(size_t)((i + 1) / C - 1) * (2 * W + 1) + (j - i + W)] = bottom;
    }
};

// Shared memory of the pairs and search kernels: one staging slot of R*DM floats per
// thread (rows of the next virtual lane).
template <int R, int DM>
constexpr size_t stage_bytes() { return (size_t)128 * R * DM * sizeof(float); }

// Block rings of the ring variant: the group's slice of the dynamic shared memory,
// zeroed once (the dimensions D..DM-1 of every slot are never written afterwards).
template <int R, int DM, bool kRing, bool kBand>
__device__ __forceinline__ float *block_ring(float *smem, int G, int W, const float **band) {
    *band = nullptr;
    if (!kRing) return nullptr;
    const int gf = ring_group_floats(R, DM, G);
    for (int k = threadIdx.x; k < (128 / G) * gf; k += blockDim.x) smem[k] = 0.f;
    if (kBand && ring_band_table(R, DM)) {
        float *tab = smem + (size_t)(128 / G) * gf;
        const int nt = min(2 * W + R, G * (R + 1));  // valid (tile, G, W): 2W + R <= G(R+1)
        for (int t = threadIdx.x; t < nt; t += blockDim.x) {
            const int dj = t - W;
            int nin = 0;
            for (int r = 0; r < R; ++r) {
                const bool in = dj - r <= W && r - dj <= W;
                tab[t * kBandEntry + r] = in ? 0.f : TC_INF;
                nin += in;
            }
            tab[t * kBandEntry + R] = __int_as_float(nin);
            for (int r = R + 1; r < kBandEntry; ++r) tab[t * kBandEntry + r] = 0.f;
        }
        *band = tab;
    }
    __syncthreads();
    return smem + (size_t)(threadIdx.x / G) * gf;
}

template <int R, int DM, bool kRing>
__global__ void __launch_bounds__(128) k_dtw_pairs(const float *__restrict__ A, const float *__restrict__ B, int64_t P,
                                                    int L, int D, int W, int G, float *__restrict__ dist,
                                                    float *__restrict__ ckpt, int C) {
    extern __shared__ __align__(16) float stage_smem[];
    float *stage = kRing ? nullptr : stage_smem + (size_t)threadIdx.x * R * DM;
    const float *band = nullptr;
    float *ring = block_ring<R, DM, kRing, true>(stage_smem, G, W, &band);
    const int RC = ring_cols(G);
    Grp g = make_grp(G);
    g.mask = 0xffffffffu;  // lockstep: every group of the warp runs the same schedule
    const int gpw = 32 / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nv = (L + R - 1) / R;
    const int nck = (L + C - 1) / C - 1;
    for (int64_t base = warp * gpw; base < P; base += nwarps * gpw) {
        const int64_t p = base + (threadIdx.x & 31) / G;
        const bool live = p < P;
        CkptHooks<R> h;
        h.ck = (ckpt && live) ? ckpt + (size_t)p * nck * (2 * W + 1) : nullptr;
        h.C = C;
        h.W = W;
        h.L = L;
        bool ab = false;
        long long cells;
        const int64_t pp = live ? p : 0;
        float r = band_pass<R, DM, CkptHooks<R>, kRing>(A + (size_t)pp * L * D, B + (size_t)pp * L * D, L, D, W, 0,
                                                       nv, g, h, live, &ab, &cells, stage, ring, RC, band);
        r = grp_min(r, g);
        if (live && g.lig == 0) dist[p] = r;
    }
}

// ============================================================= NN search (FP32)
struct NnHooks {
    const unsigned long long *bsf;  // this query's packed best-so-far
    float rho;
    static constexpr bool kAbandon = true;
    static constexpr bool kCells = false;
    __device__ __forceinline__ float top(int) const { return TC_INF; }
    __device__ __forceinline__ bool abandon(float fm) { return fm > prune_threshold(ld_volatile_u64(bsf), rho); }
    __device__ __forceinline__ void cell(int, int, float) {}
    __device__ __forceinline__ void after_col(int, int, float) {}
};

// Entries e in [0, count): pair (m = pairs[e] / N, n = pairs[e] % N); lb[e] is the
// entry's best lower bound (+inf = already dropped; lb == null: 0).  Writes dtw[e]
// (FP32 DTW, or +inf when pruned / abandoned) and lowers bsf[m].
// R = 16 with up to 5 dimensions: capped at 128 registers (4 CTAs, 16 warps per SM)
template <int R, int DM, bool kRing>
__global__ void __launch_bounds__(128, (R >= 16 && DM <= 5) ? 4 : 1) k_dtw_nn(const float *__restrict__ Q, const float *__restrict__ Cand, int L,
                                                 int D, int W, int G, int64_t N, const uint32_t *__restrict__ pairs,
                                                 const float *__restrict__ lb, const int32_t *__restrict__ count,
                                                 int n_static, int *__restrict__ cursor, unsigned long long *bsf,
                                                 float rho, float *__restrict__ dtw,
                                                 unsigned long long *__restrict__ counters) {
    extern __shared__ __align__(16) float stage_smem[];
    float *stage = kRing ? nullptr : stage_smem + (size_t)threadIdx.x * R * DM;
    const float *band = nullptr;
    float *ring = block_ring<R, DM, kRing, false>(stage_smem, G, W, &band);
    const int RC = ring_cols(G);
    Grp g = make_grp(G);
    g.mask = 0xffffffffu;  // lockstep: every group of the warp runs the same schedule
    const int gpw = 32 / G;
    const int nv = (L + R - 1) / R;
    const int n_entries = count ? *count : n_static;
    unsigned long long started = 0, aband = 0, ncells = 0, pruned = 0;
    for (;;) {
        // the warp takes gpw consecutive entries, one per group, and runs them together
        int base = 0;
        if ((threadIdx.x & 31) == 0) base = atomicAdd(cursor, gpw);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_entries) break;
        const int e = base + (threadIdx.x & 31) / G;
        bool live = e < n_entries;
        const uint32_t pid = live ? pairs[e] : 0xffffffffu;
        live = live && pid != 0xffffffffu;
        int m = 0;
        int64_t n = 0;
        if (live) {
            m = (int)(pid / (uint32_t)N);
            n = (int64_t)(pid - (uint32_t)m * (uint32_t)N);
            const float lbe = lb ? lb[e] : 0.f;
            const float thr = prune_threshold(ld_volatile_u64(bsf + m), rho);
            if (!(lbe <= thr) || lbe == TC_INF) {
                if (g.lig == 0 && lbe != TC_INF) ++pruned;
                live = false;
            }
        }
        NnHooks h;
        h.bsf = bsf + m;
        h.rho = rho;
        bool ab = false;
        long long cells = 0;
        float r = band_pass<R, DM, NnHooks, kRing>(Q + (size_t)m * L * D, Cand + (size_t)n * L * D, L, D, W, 0, nv, g,
                                                   h, live, &ab, &cells, stage, ring, RC, band);
        r = grp_min(r, g);
        long long cs = cells;
        for (int o = G >> 1; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
        if (e < n_entries && g.lig == 0) {
            if (!live) {
                dtw[e] = TC_INF;
            } else {
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
    }
    if (g.lig == 0 && counters && (started | pruned)) {
        atomicAdd(counters + 0, started);
        atomicAdd(counters + 1, aband);
        atomicAdd(counters + 2, ncells);
        atomicAdd(counters + 3, pruned);
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
    __device__ __forceinline__ float top(int j) const { return S[j - (row0 - 1) + W]; }
    __device__ __forceinline__ bool abandon(float) { return false; }
    __device__ __forceinline__ void cell(int i, int j, float val) {
        S[(size_t)(i - row0 + 1) * (2 * W + 1) + (j - i + W)] = val;
    }
    __device__ __forceinline__ void after_col(int, int, float) {}
};

// One group per pair.  Shared memory per group: (C+1) * (2W+1) floats.
template <int R, int DM>
__global__ void __launch_bounds__(128) k_dtw_backward(const float *__restrict__ A, const float *__restrict__ B,
                                                       const float *__restrict__ ckpt, int C,
                                                       const float *__restrict__ gdist, int64_t P, int L, int D, int W,
                                                       int G, float *__restrict__ gA, float *__restrict__ gB) {
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
    constexpr int KD = (DM + 3) / 4;  // dims per lane (G >= 4)
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
        for (int k = 0; k < KD; ++k) {
            acc_a[k] = 0.f;
            acc_b[k] = 0.f;
        }
        int ci = L - 1, cj = L - 1;  // path cursor
        bool done = false;
        for (int s = nseg - 1; s >= 0 && !done; --s) {
            const int row0 = s * C;
            const int row1 = min(L, row0 + C);
            for (int k = g.lig; k < BW; k += G) S[k] = (s == 0) ? INF : ck[(size_t)(s - 1) * BW + k];
            __syncwarp(g.mask);
            SegHooks h;
            h.S = S;
            h.row0 = row0;
            h.W = W;
            bool ab;
            long long cells;
            band_pass<R, DM>(a, b, L, D, W, row0 / R, (row1 + R - 1) / R, g, h, true, &ab, &cells);
            __syncwarp(g.mask);
            while (ci >= row0) {
#pragma unroll
                for (int k = 0; k < KD; ++k) {
                    const int pp = g.lig + k * G;
                    if (pp < D) {
                        const float diff = a[(size_t)ci * D + pp] - b[(size_t)cj * D + pp];
                        acc_a[k] += 2.f * diff;
                        acc_b[k] -= 2.f * diff;
                    }
                }
                if (ci == 0 && cj == 0) {
                    done = true;
                    break;
                }
                auto Rv = [&](int i, int j) -> float {
                    if (i < 0 || j < 0 || abs(i - j) > W) return INF;
                    return S[(size_t)(i - row0 + 1) * BW + (j - i + W)];
                };
                const float vd = Rv(ci - 1, cj - 1), vu = Rv(ci - 1, cj), vl = Rv(ci, cj - 1);
                int ni = ci - 1, nj = cj - 1;
                float best = vd;
                if (vu < best) { best = vu; ni = ci - 1; nj = cj; }
                if (vl < best) { best = vl; ni = ci; nj = cj - 1; }
                if (ni != ci) {  // leaving row ci
#pragma unroll
                    for (int k = 0; k < KD; ++k) {
                        const int pp = g.lig + k * G;
                        if (pp < D) ga[(size_t)ci * D + pp] = gscale * acc_a[k];
                        acc_a[k] = 0.f;
                    }
                }
                if (nj != cj) {  // leaving column cj
#pragma unroll
                    for (int k = 0; k < KD; ++k) {
                        const int pp = g.lig + k * G;
                        if (pp < D) gb[(size_t)cj * D + pp] = gscale * acc_b[k];
                        acc_b[k] = 0.f;
                    }
                }
                ci = ni;
                cj = nj;
            }
            __syncwarp(g.mask);
        }
#pragma unroll
        for (int k = 0; k < KD; ++k) {
            const int pp = g.lig + k * G;
            if (pp < D) {
                ga[pp] = gscale * acc_a[k];
                gb[pp] = gscale * acc_b[k];
            }
        }
        __syncwarp(g.mask);
    }
}

// ============================================================= FP64 band pass
// The FP64 recompute of Eq. (1) in the oracle's operation order (per cell
// t_p = a_p - b_p, s = ((t_0*t_0) + t_1*t_1) + ... without fusion, R = s + min),
// so the value is bit-identical to a plain sequential FP64 evaluation.  One warp
// (g.G = 32) per pair, R rows per lane, D at run time.
//
// FP64 issues at a small fraction of the FP32 rate on this GPU, so the pass keeps
// FP64 work to the 3D operations per cell the definition needs: a column's D
// values are widened once per column (not once per cell), the lane's R rows once
// per virtual lane into its shared-memory slot ad (R*D doubles; null: widened per
// cell), the first term is not added to 0, and the three-way minimum compares the
// bit patterns as integers (the DP values are non-negative doubles or +inf, whose
// bit patterns order like their values).
__device__ __forceinline__ double min_nonneg(double a, double b) {
    const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
    return __longlong_as_double(x < y ? x : y);
}

template <int R>
__device__ double band_pass64(const float *__restrict__ A, const float *__restrict__ B, int L, int D, int W,
                              const Grp &g, double *ad = nullptr) {
    const double INF = __longlong_as_double(0x7ff0000000000000LL);
    double col[R];
    double bottom = INF, prev_in = INF, result = INF;
    const int nv = (L + R - 1) / R;
    const int vlast = (L - 1) / R;
    int v = g.lig;
    const int tau0 = 0;
    const int tau_end = v_jhi(nv - 1, R, W, L) + (nv - 1);
    int tlo = v < nv ? v_jlo(v, R, W) + v : 1 << 30;
    int thi = v < nv ? v_jhi(v, R, W, L) + v : -1;
    bool fresh = true;
    for (int tau = tau0; tau <= tau_end; ++tau) {
        const double in = __shfl_sync(g.mask, bottom, g.src);
        if (tau > thi && v < nv) {
            v += g.G;
            fresh = true;
            tlo = v < nv ? v_jlo(v, R, W) + v : 1 << 30;
            thi = v < nv ? v_jhi(v, R, W, L) + v : -1;
        }
        if (tau >= tlo && tau <= thi) {
            const int j = tau - v;
            const int i0 = v * R;
            if (fresh) {
#pragma unroll
                for (int r = 0; r < R; ++r) col[r] = INF;
                if (ad) {
                    for (int r = 0; r < R; ++r)
                        for (int p = 0; p < D; ++p)
                            ad[r * D + p] = i0 + r < L ? (double)__ldg(A + (size_t)(i0 + r) * D + p) : 0.0;
                }
                fresh = false;
            }
            double up = (v == 0) ? INF : ((j <= i0 - 1 + W) ? in : INF);
            double diag = (v == 0) ? ((j == 0) ? 0.0 : INF) : ((j >= 1 && j <= i0 + W) ? prev_in : INF);
            const unsigned vm = row_mask(j - W - i0, min(j + W - i0, L - 1 - i0), R);
            const float *bj = B + (size_t)j * D;
            // cell costs of the lane's R rows at column j (rows past the end read row
            // L-1 and are masked below)
            double s[R];
            for (int p = 0; p < D; ++p) {
                const double bp = (double)__ldg(bj + p);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const double ap = ad ? ad[r * D + p] : (double)__ldg(A + (size_t)min(i0 + r, L - 1) * D + p);
                    const double t = __dsub_rn(ap, bp);
                    const double t2 = __dmul_rn(t, t);
                    s[r] = p == 0 ? t2 : __dadd_rn(s[r], t2);
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const double left = col[r];
                const double val = ((vm >> r) & 1u) ? __dadd_rn(s[r], min_nonneg(min_nonneg(up, left), diag)) : INF;
                diag = left;
                up = val;
                col[r] = val;
            }
            bottom = col[R - 1];
            if (v == vlast && j == L - 1) {
                const int rl = (L - 1) - i0;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (r == rl) result = col[r];
            }
        }
        prev_in = in;
    }
    return result;
}

// ============================================================= per-tile launchers
// The ring variant is compiled for the wide-point tiles (DM >= 16, a multiple of 4) and
// used when its shared memory for the launch's G stays within kRingSmemMax (two blocks
// per SM); otherwise, and for narrow points, the plain variant runs.
constexpr size_t kRingSmemMax = 112 * 1024;

template <int R, int DM>
struct TileKernels {
    static constexpr bool kHasRing = DM >= 16 && DM % 4 == 0;
    static constexpr bool kDimPack = DM >= 16;
    // the plain variant's staging slots (narrow points only; wide points read rows directly)
    static constexpr size_t plain_bytes() { return kDimPack ? 0 : stage_bytes<R, DM>(); }
    static bool use_ring(int G) { return kHasRing && ring_block_bytes(R, DM, G) <= kRingSmemMax; }
    static cudaError_t prepare() {  // allow dynamic shared memory above 48 KB (once)
        static bool done = false;
        if (done) return cudaSuccess;
        const int sb = (int)(plain_bytes() > 0 ? plain_bytes() : 1024);
        cudaError_t e = cudaFuncSetAttribute(k_dtw_pairs<R, DM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_dtw_nn<R, DM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb);
        if constexpr (kHasRing) {
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_dtw_pairs<R, DM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kRingSmemMax);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_dtw_nn<R, DM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kRingSmemMax);
        }
        done = e == cudaSuccess;
        return e;
    }
    static cudaError_t pairs(int G, int blocks, cudaStream_t s, const float *A, const float *B, int64_t P, int L,
                             int D, int W, float *dist, float *ck, int C) {
        cudaError_t e = prepare();
        if (e != cudaSuccess) return e;
        if constexpr (kHasRing) {
            if (use_ring(G)) {
                k_dtw_pairs<R, DM, true><<<blocks, 128, ring_block_bytes(R, DM, G), s>>>(A, B, P, L, D, W, G, dist,
                                                                                          ck, C);
                note_launch();
                return cudaGetLastError();
            }
        }
        k_dtw_pairs<R, DM, false><<<blocks, 128, plain_bytes(), s>>>(A, B, P, L, D, W, G, dist, ck, C);
        note_launch();
        return cudaGetLastError();
    }
    static cudaError_t nn(int blocks, cudaStream_t s, const DtwNnArgs &x) {
        cudaError_t e = prepare();
        if (e != cudaSuccess) return e;
        if constexpr (kHasRing) {
            if (use_ring(x.G)) {
                k_dtw_nn<R, DM, true><<<blocks, 128, ring_block_bytes(R, DM, x.G), s>>>(
                    x.Q, x.C, x.L, x.D, x.W, x.G, x.N, x.pairs, x.lb, x.count, x.n_static, x.cursor, x.bsf, x.rho,
                    x.dtw, x.counters);
                note_launch();
                return cudaGetLastError();
            }
        }
        k_dtw_nn<R, DM, false><<<blocks, 128, plain_bytes(), s>>>(x.Q, x.C, x.L, x.D, x.W, x.G, x.N, x.pairs, x.lb,
                                                                   x.count, x.n_static, x.cursor, x.bsf, x.rho, x.dtw,
                                                                   x.counters);
        note_launch();
        return cudaGetLastError();
    }
    static cudaError_t backward(int G, int blocks, int threads, size_t smem, cudaStream_t s, const float *A,
                                const float *B, const float *ck, int C, const float *gd, int64_t P, int L, int D,
                                int W, float *gA, float *gB) {
        if (smem > 227 * 1024) return cudaErrorInvalidValue;
        auto k = k_dtw_backward<R, DM>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k<<<blocks, threads, smem, s>>>(A, B, ck, C, gd, P, L, D, W, G, gA, gB);
        note_launch();
        return cudaGetLastError();
    }
    // resident blocks per SM of the variant a launch with G runs (which: 0 pairs, 1 search)
    static int occupancy(int which, int G) {
        int n = 0;
        if (prepare() != cudaSuccess) return 0;
        if constexpr (kHasRing) {
            if (use_ring(G)) {
                const size_t sb = ring_block_bytes(R, DM, G);
                if (which == 0)
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_dtw_pairs<R, DM, true>, 128, sb);
                else
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_dtw_nn<R, DM, true>, 128, sb);
                return n;
            }
        }
        if (which == 0)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_dtw_pairs<R, DM, false>, 128, plain_bytes());
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_dtw_nn<R, DM, false>, 128, plain_bytes());
        return n;
    }
};

// Per-tile entry points (defined in the instantiation units).
#define TC_TILE_DECL(id, R, DM)                                                                                     \
    cudaError_t tile##id##_pairs(int G, int blocks, cudaStream_t s, const float *A, const float *B, int64_t P,     \
                                 int L, int D, int W, float *dist, float *ck, int C);                              \
    cudaError_t tile##id##_nn(int blocks, cudaStream_t s, const DtwNnArgs &x);                                     \
    cudaError_t tile##id##_backward(int G, int blocks, int threads, size_t smem, cudaStream_t s, const float *A,   \
                                    const float *B, const float *ck, int C, const float *gd, int64_t P, int L,     \
                                    int D, int W, float *gA, float *gB);                                           \
    int tile##id##_occupancy(int which, int G);

#define TC_TILE_DEF(id, R, DM)                                                                                      \
    cudaError_t tile##id##_pairs(int G, int blocks, cudaStream_t s, const float *A, const float *B, int64_t P,     \
                                 int L, int D, int W, float *dist, float *ck, int C) {                             \
        return TileKernels<R, DM>::pairs(G, blocks, s, A, B, P, L, D, W, dist, ck, C);                              \
    }                                                                                                               \
    cudaError_t tile##id##_nn(int blocks, cudaStream_t s, const DtwNnArgs &x) {                                    \
        return TileKernels<R, DM>::nn(blocks, s, x);                                                                \
    }                                                                                                               \
    cudaError_t tile##id##_backward(int G, int blocks, int threads, size_t smem, cudaStream_t s, const float *A,   \
                                    const float *B, const float *ck, int C, const float *gd, int64_t P, int L,     \
                                    int D, int W, float *gA, float *gB) {                                          \
        return TileKernels<R, DM>::backward(G, blocks, threads, smem, s, A, B, ck, C, gd, P, L, D, W, gA, gB);      \
    }                                                                                                               \
    int tile##id##_occupancy(int which, int G) { return TileKernels<R, DM>::occupancy(which, G); }

}  // namespace tc
