// batch_internal.cuh -- definitions shared by the batched search (batch.cu) and the
// instantiation units of its band DTW (batch_dtw_r*.cu): the per-set descriptor, the
// launch control block, and the DTW work loop, templated on the band tile (R rows per
// lane, DM dimensions) that the tuner chose for each set.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "dtw_core.cuh"

namespace tc {


constexpr int kBatchMaxD = 12;      // dimensions of the batched path (one exact-width tile per D)
constexpr int kBatchThreads = 128;  // 4 warps per CTA
constexpr int kBatchQB = 32;        // queries per LB_MV tile
constexpr int kSeedSlots = 8;       // seed slots per query
constexpr long long kSpinLimit = 4000000;  // ~1 s of 256 ns sleeps
constexpr size_t kBatchSmem = 48 * 1024;   // LB_MV double buffers / box scratch / FP64 row slots

// Per-set counters (ints, zeroed before every run).
enum : int { kCntPrep = 0, kCntMv, kCntList, kCntSeedCursor, kCntSurvCursor, kCntSeed2Cursor, kCntPerSet };
// seed_dtw of a second-round seed whose DTW is still to run
constexpr float kSeedPending = -1.f;

struct BatchSet {
    const float *cand, *q;
    int64_t *idx;
    double *dist;
    int64_t N;
    int L, D, W, K, M;
    int G, R, dcase, Rref, S;  // DTW lanes per pair, rows per lane and tile DM; FP64 rows per lane;
                               // seeds per query
    int S2;                    // second-round seeds per query (abandoning LB_MV)
    int use_pc, use_ti, Lq, w, P, Gpc, np2, vec4, check_finite;
    float e_pc, e_ti, rho, rho_ref;
    double kappa;
    int64_t ldE;
    int n_qtiles, n_ctiles;
    int samp, sstride;                   // LB_MV sample of the abandoning form (samp 0: whole rows)
    float *U, *Lo, *dq_lo, *dq_hi, *boxes;
    float *Up, *Lp;                      // [M][ldE] envelope, one query per row (samp > 0)
    int32_t *box_counts;
    float *lbm;                          // [M][N] LB_MV
    uint32_t *surv;                      // [M][N] survivor candidate ids, per query
    float *surv_lb, *surv_dtw;           // [M][N]
    uint32_t *list;                      // [M*N] DTW work list: q*N + position in the query's survivors
    uint32_t *seeds;                     // [M][8] (UINT32_MAX: empty slot)
    float *seed_dtw;                     // [M][8]
    double *d64;                         // [M][N+8] refine values
    unsigned long long *bsf;             // [M] packed best-so-far
    int *nseed, *ncnt;                   // [M]
    int *cnt;                            // kCntPerSet counters
};

enum : int { kItemPrep = 0, kItemMv, kItemSeed, kItemMid, kItemRefine, kItemStall, kItemRest, kItemSeed2 };
constexpr int kRefinePerItem = 4;  // queries per refine item (one per warp)
struct BatchItem {
    int kind, set, a, b;
};

struct BatchCtl {
    int next[4];  // cursors of the front, mid, refine and LB_MV completion item ranges
    int abort;
    int never;    // stays 0: the self-test waits on it
    DevStatus status;
    unsigned long long counters[10];  // started, abandoned, cells, pruned at DTW, pruned MV, PC, TI, refined,
                                      // refined in FP64, LB_MV terms of the completion pass
};


// ------------------------------------------------------------------ DTW launches
// Phase 0: the seed entries i < M*8 (query i/8, slot i%8); phase 1: the work list;
// phase 2: the second-round seed entries (slots whose seed_dtw is kSeedPending).
// A warp takes 32/G consecutive entries of one set (one per lane group) and runs
// them in lockstep, as the single-set kernel does; the sets follow each other in
// the order given, each with its own cursor, so warps move on as a set runs dry.
// Every set of one launch has the launch's tile (R, DM); G is the set's own.
template <int R, int DM>
__device__ __forceinline__ void dtw_set(const BatchSet &S, int phase, float *stage, BatchCtl *ctl) {
    Grp g = make_grp(S.G);
    g.mask = 0xffffffffu;
    const int G = S.G, gpw = 32 / G;
    const int L = S.L, D = S.D, W = S.W;
    const int64_t N = S.N;
    const int nv = (L + R - 1) / R;
    const int n_entries = phase == 1 ? S.cnt[kCntList] : S.M * kSeedSlots;
    int *cursor = S.cnt + (phase == 0 ? kCntSeedCursor : phase == 1 ? kCntSurvCursor : kCntSeed2Cursor);
    unsigned long long started = 0, aband = 0, ncells = 0, pruned = 0;
    for (;;) {
        int base = 0;
        if ((threadIdx.x & 31) == 0) base = atomicAdd(cursor, gpw);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_entries) break;
        const int e = base + (threadIdx.x & 31) / G;
        bool live = e < n_entries;
        int q = 0;
        uint32_t cn = 0;
        float lbe = 0.f;
        float *out = nullptr;
        if (live) {
            if (phase != 1) {
                q = e / kSeedSlots;
                cn = S.seeds[e];
                out = S.seed_dtw + e;
                live = cn != 0xffffffffu && (phase == 0 || *out == kSeedPending);
            } else {
                const uint32_t pid = S.list[e];
                q = (int)(pid / (uint64_t)N);
                cn = S.surv[pid];
                lbe = S.surv_lb[pid];
                out = S.surv_dtw + pid;
            }
        }
        if (live) {
            const float thr = prune_threshold(ld_volatile_u64(S.bsf + q), S.rho);
            if (!(lbe <= thr) || lbe == TC_INF) {
                if (g.lig == 0 && lbe != TC_INF) ++pruned;
                if (g.lig == 0) *out = TC_INF;
                live = false;
            }
        }
        NnHooks h;
        h.bsf = S.bsf + q;
        h.rho = S.rho;
        bool ab = false;
        long long cells = 0;
        float r = band_pass<R, DM>(S.q + (size_t)q * L * D, S.cand + (size_t)cn * L * D, L, D, W, 0, nv, g, h, live,
                                   &ab, &cells, stage);
        r = grp_min(r, g);
        long long cs = cells;
        for (int o = G >> 1; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
        if (live && g.lig == 0) {
            ++started;
            ncells += (unsigned long long)cs;
            if (ab) {
                ++aband;
                *out = TC_INF;
            } else {
                *out = r;
                atomicMin(S.bsf + q, pack_best(r, cn));
            }
        }
    }
    if (g.lig == 0 && (started | pruned)) {
        atomicAdd(&ctl->counters[0], started);
        atomicAdd(&ctl->counters[1], aband);
        atomicAdd(&ctl->counters[2], ncells);
        atomicAdd(&ctl->counters[3], pruned);
    }
}

// One launch per tile class (R, DM) and phase: the sets order[0..nsets) of the class.
// (One kernel holding every DM variant does not reuse registers across them and
// spills inside the DP loop.)
// (Register caps: 3 blocks per SM (168 registers), 2 for 16 rows of 6..8 dimensions;
// a few dozen bytes of spills remain outside the cell loop for R = 16.)
template <int R, int DM>
__global__ void __launch_bounds__(kBatchThreads, R >= 16 && DM > 5 ? 2 : 3) k_batch_dtw(const BatchSet *__restrict__ sets,
                                                                const int *__restrict__ order, int nsets, int phase,
                                                                BatchCtl *ctl) {
    extern __shared__ __align__(16) float stage_smem[];
    float *stage = stage_smem + (size_t)threadIdx.x * R * DM;
    for (int oi = 0; oi < nsets; ++oi) dtw_set<R, DM>(sets[order[oi]], phase, stage, ctl);
}

// Staging slots of the DTW launch (one R x DM slot per thread).
constexpr size_t batch_dtw_smem(int R, int DM) { return (size_t)kBatchThreads * R * DM * sizeof(float); }

// Opt the kernel in to `smem` bytes of dynamic shared memory and return its resident
// grid (blocks per SM x SMs).
cudaError_t kernel_grid(const void *fn, size_t smem, int *grid);

// The compiled batched tiles: R in {4, 8, 16} for D <= 8 (exact-width DM = D), R in
// {4, 8} for D = 9..12.
inline bool batch_tile_compiled(int R, int D) { return D >= 1 && D <= 12 && (R == 4 || R == 8 || (R == 16 && D <= 8)); }

// Per rows-per-lane instantiation unit (batch_dtw_r{4,8,16}.cu): launch / grid of tile (R, dm).
cudaError_t batch_dtw_launch_r4(int dm, int grid, cudaStream_t s, const BatchSet *sets, const int *order, int nsets,
                                int phase, BatchCtl *ctl);
cudaError_t batch_dtw_launch_r8(int dm, int grid, cudaStream_t s, const BatchSet *sets, const int *order, int nsets,
                                int phase, BatchCtl *ctl);
cudaError_t batch_dtw_launch_r16(int dm, int grid, cudaStream_t s, const BatchSet *sets, const int *order, int nsets,
                                 int phase, BatchCtl *ctl);
cudaError_t batch_dtw_grid_r4(int dm, int *grid);
cudaError_t batch_dtw_grid_r8(int dm, int *grid);
cudaError_t batch_dtw_grid_r16(int dm, int *grid);

}  // namespace tc
