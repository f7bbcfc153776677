// lb.cu -- lower bounds, compaction and selection on sm_103a.
//
// Every bound is computed in FP32 with directed rounding so that the stored value
// never exceeds the exact bound (hence never exceeds the exact DTW):
//   |c - clamp(c, lo, hi)| is rounded toward zero, squares and sums are rounded
//   down (LB_MV Section 3, LB_PC Section 5); LB_TI (Section 4) carries a lower bound
//   rounded down and an upper bound rounded up through Eqs. (bt_lb), (bt_ub).
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "lb_device.cuh"
#include "lb_kernels.cuh"

namespace tc {

// ============================================================== LB_MV stream
// CTA tile: 128 candidates (one per thread) x QB queries.  LB_MV is a sum over the
// flat (point, dimension) elements e = 0 .. E-1 (E = L*D), each candidate element
// against the query envelope at the same element, so the elements are streamed in
// chunks of 32: the candidate chunk [128][32] and the envelope chunk of the tile's
// queries are copied to shared memory with cp.async (16-byte copies when aligned),
// double buffered.  A candidate row is 128 bytes; its eight 16-byte segments are
// stored XOR-swizzled by (row & 7) so the per-thread 16-byte reads are free of bank
// conflicts.  The envelope is stored query-pair interleaved, [q/2][e][q%2], so one
// 16-byte broadcast read gives two elements of two queries.
// Per element and query:  m = max(c -rd U, Lo -rd c, 0)  (one three-input max),
// acc += m*m rounded down; the subtractions and the multiply-adds of two queries go
// in one packed f32x2 instruction each.  Sums are two-level (32 elements of a chunk,
// then the chunk sums), so a round-down chain is at most 32 + E/32 long.
template <int QB>
__global__ void __launch_bounds__(128) k_lb_mv(const float *__restrict__ cand, int64_t N, int nchunks, int cstride,
                                               int Erow, int64_t ldC, int vec4,
                                               const float *__restrict__ UI, const float *__restrict__ LI,
                                               int64_t ldE, int Mb, float *__restrict__ lb, int64_t ldLb,
                                               int n_ctiles, int n_qtiles) {
    __shared__ __align__(16) float sc[2][kMvRows * kMvChunk];
    __shared__ __align__(16) float su[2][QB * kMvChunk];
    __shared__ __align__(16) float sl[2][QB * kMvChunk];
    const int ntiles = n_ctiles * n_qtiles;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int ct = tile / n_qtiles, qt = tile % n_qtiles;
        lb_mv_tile<QB>(cand, N, nchunks, cstride, Erow, ldC, vec4, UI, LI, ldE, Mb, lb, ldLb, (int64_t)ct * kMvRows,
                       qt * QB, sc, su, sl);
    }
}

bool lb_mv_vec4(const float *cand, int E) { return (E % 4) == 0 && (((uintptr_t)cand) & 15) == 0; }
static int64_t row_stride(const LbMvArgs &a) { return a.ldC > 0 ? a.ldC : a.E; }
static int row_elems(const LbMvArgs &a) { return a.Erow > 0 ? a.Erow : a.E; }

cudaError_t launch_lb_mv(const LbMvArgs &a, cudaStream_t s) {
    if (a.N <= 0 || a.Mb <= 0) return cudaSuccess;
    if (a.status) {  // the TMA-fed stream where it applies (lb_tma.cu)
        cudaError_t e = launch_lb_mv_tma(a, s);
        if (e != cudaErrorNotSupported) return e;
    }
    const int64_t ldC = row_stride(a);
    const int Erow = row_elems(a), cstride = a.cstride > 0 ? a.cstride : 1;
    const int nchunks = (a.E + kMvChunk - 1) / kMvChunk;
    const int vec4 = lb_mv_vec4(a.cand, Erow) && (ldC % 4) == 0;
    const int n_ctiles = (int)((a.N + kMvRows - 1) / kMvRows);
    int QB = 32;
    if (a.Mb <= 8) QB = 8;
    else if (a.Mb <= 16) QB = 16;
    const int n_qtiles = (a.Mb + QB - 1) / QB;
    int occ = 0;
#define TC_MV_LAUNCH(QBV)                                                                                       \
    do {                                                                                                        \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lb_mv<QBV>, 128, 0);                              \
        int64_t tiles = (int64_t)n_ctiles * n_qtiles;                                                           \
        int64_t grid = (int64_t)(occ > 0 ? occ : 1) * a.sms;                                                    \
        if (grid > tiles) grid = tiles;                                                                         \
        k_lb_mv<QBV><<<(int)grid, 128, 0, s>>>(a.cand, a.N, nchunks, cstride, Erow, ldC, vec4, a.U, a.Lo, a.ldE, \
                                               a.Mb, a.lb, a.ldLb,                                              \
                                               n_ctiles, n_qtiles);                                             \
        note_launch();                                                                                          \
    } while (0)
    if (QB == 8) TC_MV_LAUNCH(8);
    else if (QB == 16) TC_MV_LAUNCH(16);
    else TC_MV_LAUNCH(32);
#undef TC_MV_LAUNCH
    return cudaGetLastError();
}

// ============================================================== compaction
// Survivors of row m: lb[m][n] <= thr(m), where thr(m) = thresh[m] if given, else
// the pruning threshold of the packed best-so-far bsf[m].
__device__ __forceinline__ float row_thr(const float *thresh, const unsigned long long *bsf, float rho, int64_t m) {
    return thresh ? thresh[m] : prune_threshold(bsf[m], rho);
}

// The per-row passes run one CTA of kRowThreads threads per row; a row of N bounds
// was just written by the LB_MV stream and sits in L2, so the passes are bound by load
// latency: every thread keeps four loads (count, seeds) or kRowEpt loads (write) in
// flight instead of walking the row one coalesced load at a time.
constexpr int kRowThreads = 1024;
constexpr int kRowEpt = 16;  // write pass: contiguous bounds per thread per chunk

__device__ __forceinline__ int block_sum(int c, int *red) {
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    int t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

// count pass: one CTA per row
__global__ void __launch_bounds__(kRowThreads) k_count_rows(const float *__restrict__ lb, int64_t N, int64_t ldLb,
                                                            const float *thresh, const unsigned long long *bsf,
                                                            float rho, int32_t *__restrict__ counts,
                                                            unsigned long long *pruned) {
    __shared__ int red[32];
    const int64_t m = blockIdx.x;
    const float thr = row_thr(thresh, bsf, rho, m);
    const float *row = lb + (size_t)m * ldLb;
    const int64_t bd = blockDim.x;
    int c = 0;
    for (int64_t n0 = threadIdx.x; n0 < N; n0 += 4 * bd) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = n0 + u * bd < N ? row[n0 + u * bd] : TC_INF;
#pragma unroll
        for (int u = 0; u < 4; ++u) c += (n0 + u * bd < N && v[u] <= thr);
    }
    const int t = block_sum(c, red);
    if (threadIdx.x == 0) {
        counts[m] = t;
        if (pruned) atomicAdd(pruned, (unsigned long long)(N - t));
    }
}

// exclusive scan of counts[0..M) -> offsets, total (single CTA of 1024 threads)
__global__ void k_scan_counts(const int32_t *__restrict__ counts, int64_t M, int32_t *__restrict__ offsets,
                              int32_t *__restrict__ total) {
    __shared__ int32_t part[1024];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < M; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const int32_t v = i < M ? counts[i] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int32_t t = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < M) offsets[i] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// write pass: one CTA per row, survivors in increasing n.  The row is taken in chunks
// of kRowThreads * kRowEpt bounds; thread t owns the kRowEpt consecutive bounds
// [t*kRowEpt, (t+1)*kRowEpt) of a chunk, so one exclusive scan of the per-thread
// survivor counts gives every survivor its place.  Output position of row m's k-th
// survivor: base(m) + k with base(m) = offsets[m] (flat list) or m * ldOut (per-row
// lists).  pairs (flat) receive m*N + n and lbs the bound; idx_out (per-row) receives n.
__global__ void __launch_bounds__(kRowThreads) k_write_rows(const float *__restrict__ lb, int64_t N, int64_t ldLb,
                                                            const float *thresh, const unsigned long long *bsf,
                                                            float rho, const int32_t *__restrict__ offsets,
                                                            int64_t ldOut, uint32_t *__restrict__ pairs,
                                                            float *__restrict__ lbs, int32_t *__restrict__ idx_out) {
    __shared__ int wsum[32];
    __shared__ int chunk_total;
    const int64_t m = blockIdx.x;
    const float thr = row_thr(thresh, bsf, rho, m);
    const float *row = lb + (size_t)m * ldLb;
    const int64_t base = offsets ? (int64_t)offsets[m] : m * ldOut;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t chunk = (int64_t)blockDim.x * kRowEpt;
    int64_t running = 0;
    for (int64_t c0 = 0; c0 < N; c0 += chunk) {
        const int64_t s = c0 + (int64_t)threadIdx.x * kRowEpt;
        float v[kRowEpt];
#pragma unroll
        for (int k = 0; k < kRowEpt; ++k) v[k] = s + k < N ? row[s + k] : TC_INF;
        unsigned keep = 0;
#pragma unroll
        for (int k = 0; k < kRowEpt; ++k) keep |= (unsigned)(s + k < N && v[k] <= thr) << k;
        const int cnt = __popc(keep);
        // exclusive scan of cnt over the CTA
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = lane < nw ? wsum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            if (lane < nw) wsum[lane] = w;  // inclusive over warps
            if (lane == 31) chunk_total = w;
        }
        __syncthreads();
        int64_t pos = base + running + (warp > 0 ? wsum[warp - 1] : 0) + incl - cnt;
#pragma unroll
        for (int k = 0; k < kRowEpt; ++k) {
            if ((keep >> k) & 1u) {
                if (pairs) {
                    pairs[pos] = (uint32_t)(m * N + s + k);
                    lbs[pos] = v[k];
                } else {
                    idx_out[pos] = (int32_t)(s + k);
                }
                ++pos;
            }
        }
        running += chunk_total;
        __syncthreads();  // wsum and chunk_total are rewritten by the next chunk
    }
}

cudaError_t launch_compact(const CompactArgs &a, cudaStream_t s) {
    if (a.M <= 0) return cudaSuccess;
    k_count_rows<<<(unsigned)a.M, kRowThreads, 0, s>>>(a.lb, a.N, a.ldLb, a.thresh, a.bsf, a.rho, a.counts,
                                                        a.pruned);
    note_launch();
    if (a.offsets) {
        k_scan_counts<<<1, 1024, 0, s>>>(a.counts, a.M, a.offsets, a.total);
        note_launch();
    }
    k_write_rows<<<(unsigned)a.M, kRowThreads, 0, s>>>(a.lb, a.N, a.ldLb, a.thresh, a.bsf, a.rho, a.offsets, a.ldOut,
                                                        a.pairs, a.lbs, a.idx_out);
    note_launch();
    return cudaGetLastError();
}

// ============================================================== seeds
// Per row m (one CTA of kRowThreads threads): the S candidates with the smallest bound
// (ties: smaller n) become seed entries m*N + n (empty slots: UINT32_MAX), and
// their bound in the row is replaced by +inf so they do not survive compaction.
// Per row m (one CTA): seed entries m*N + n (empty slots: UINT32_MAX).
__global__ void __launch_bounds__(kRowThreads) k_seed_topk(float *__restrict__ lb, int64_t N, int64_t ldLb, int S,
                                                          uint32_t *__restrict__ seeds) {
    __shared__ uint32_t picked[kMaxSeeds];
    const int64_t m = blockIdx.x;
    seed_topk_row(lb + (size_t)m * ldLb, N, S, picked);
    if (threadIdx.x < (unsigned)S) {
        const uint32_t n = picked[threadIdx.x];
        seeds[m * S + threadIdx.x] = (n == 0xffffffffu) ? 0xffffffffu : (uint32_t)(m * N + n);
    }
}

cudaError_t launch_seed_topk(float *lb, int64_t M, int64_t N, int64_t ldLb, int S, uint32_t *seeds, cudaStream_t s) {
    if (M <= 0 || S <= 0) return cudaSuccess;
    if (S > kMaxSeeds) S = kMaxSeeds;
    k_seed_topk<<<(unsigned)M, kRowThreads, 0, s>>>(lb, N, ldLb, S, seeds);
    note_launch();
    return cudaGetLastError();
}

// ============================================================== LB_PC / LB_TI on listed pairs
// One warp per entry.  Entry e (e < *count): pair id pairs[e] = m*N + n and its
// current bound lbv[e] (+inf: already dropped).  The gate of selective deployment
// (Section 6): the tight bound runs only if e_gate * bsf < lbv[e] <= threshold.
// A pair whose tight bound exceeds the threshold gets lbv[e] = +inf.
template <int DMAX>
__global__ void __launch_bounds__(128) k_lb_pc_list(PairListArgs a, const float *__restrict__ boxes,
                                                    const int32_t *__restrict__ counts, int K, int w,
                                                    const unsigned long long *bsf, float rho, float e_gate,
                                                    unsigned long long *stat_pruned) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n_entries = a.count ? (int64_t)*a.count : a.n_static;
    const int G = (a.L + w - 1) / w;
    unsigned long long pruned = 0;
    for (int64_t e = warp; e < n_entries; e += nwarps) {
        const uint32_t pid = a.pairs[e];
        if (pid == 0xffffffffu) continue;
        const float cur = a.lb[e];
        if (!(cur < TC_INF)) continue;
        const int64_t m = pid / (uint64_t)a.N, n = pid - m * a.N;
        const unsigned long long key = ld_volatile_u64(bsf + m);
        if (cur > prune_threshold(key, rho)) continue;  // dropped (and counted) by the DTW stage
        if (!(cur > e_gate * best_dist(key))) continue;
        float bound;
        const bool dropped = lb_pc_pair<DMAX>(a.C + (size_t)n * a.L * a.D, boxes + (size_t)m * G * K * 2 * a.D,
                                              counts + (size_t)m * G, a.L, a.D, K, w, bsf + m, rho, &bound);
        if (lane == 0) {
            if (dropped) { a.lb[e] = TC_INF; ++pruned; }
            else a.lb[e] = fmaxf(cur, bound);
        }
    }
    if (lane == 0 && pruned && stat_pruned) atomicAdd(stat_pruned, pruned);
}

// LB_TI of the listed pairs, one warp per pair.  The block takes runs of kTiChunk
// consecutive entries (the survivor lists are ordered by query, so a run rarely spans
// two queries) and stages the query of the run's first entry -- its points and the
// [dq_lo, dq_hi] interval of its neighbour distances -- in shared memory when it fits;
// entries of another query read theirs from global memory.
constexpr int kTiChunk = 64;

template <int DMAX>
__global__ void __launch_bounds__(128) k_lb_ti_list(PairListArgs a, const float *__restrict__ dq_lo,
                                                    const float *__restrict__ dq_hi, int P,
                                                    const unsigned long long *bsf, float rho, float e_gate,
                                                    unsigned long long *stat_pruned, int stage) {
    extern __shared__ float sq[];  // [L][D] query points, [L] dq_lo, [L] dq_hi
    __shared__ int64_t s_m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n_entries = a.count ? (int64_t)*a.count : a.n_static;
    const int L = a.L, D = a.D;
    unsigned long long pruned = 0;
    for (int64_t c0 = (int64_t)blockIdx.x * kTiChunk; c0 < n_entries; c0 += (int64_t)gridDim.x * kTiChunk) {
        const int64_t c1 = min(c0 + kTiChunk, n_entries);
        if (stage) {
            __syncthreads();  // the previous run is done with the staged query
            if (threadIdx.x == 0) {
                const uint32_t pid = a.pairs[c0];
                s_m = pid == 0xffffffffu ? -1 : (int64_t)(pid / (uint64_t)a.N);
            }
            __syncthreads();
            if (s_m >= 0) {
                const float *qm = a.Q + (size_t)s_m * L * D;
                for (int k = threadIdx.x; k < L * D; k += blockDim.x) sq[k] = __ldg(qm + k);
                for (int k = threadIdx.x; k < L; k += blockDim.x) {
                    sq[L * D + k] = __ldg(dq_lo + (size_t)s_m * L + k);
                    sq[L * D + L + k] = __ldg(dq_hi + (size_t)s_m * L + k);
                }
            }
            __syncthreads();
        }
        for (int64_t e = c0 + warp; e < c1; e += 4) {
            const uint32_t pid = a.pairs[e];
            if (pid == 0xffffffffu) continue;
            const float cur = a.lb[e];
            if (!(cur < TC_INF)) continue;
            const int64_t m = pid / (uint64_t)a.N, n = pid - m * a.N;
            const unsigned long long key = ld_volatile_u64(bsf + m);
            if (cur > prune_threshold(key, rho)) continue;  // dropped (and counted) by the DTW stage
            if (!(cur > e_gate * best_dist(key))) continue;
            const bool staged = stage && m == s_m;
            const float *qp = staged ? sq : a.Q + (size_t)m * L * D;
            const float *dl = staged ? sq + L * D : dq_lo + (size_t)m * L;
            const float *dh = staged ? sq + L * D + L : dq_hi + (size_t)m * L;
            float bound;
            const bool dropped = lb_ti_pair<DMAX>(a.C + (size_t)n * L * D, qp, dl, dh, L, D, a.W, P, bsf + m, rho,
                                                  &bound);
            if (lane == 0) {
                if (dropped) { a.lb[e] = TC_INF; ++pruned; }
                else a.lb[e] = fmaxf(cur, bound);
            }
        }
    }
    if (lane == 0 && pruned && stat_pruned) atomicAdd(stat_pruned, pruned);
}

// LB_TI without the exact window top (basic / TIP variants; lb_ti_rows_pair), one warp
// per listed pair, same gate and bookkeeping as k_lb_ti_list.
template <int DMAX, int NS>
__global__ void __launch_bounds__(128) k_lb_ti_rows_list(PairListArgs a, const float *__restrict__ dq_lo,
                                                         const float *__restrict__ dq_hi, int P,
                                                         const unsigned long long *bsf, float rho, float e_gate,
                                                         unsigned long long *stat_pruned) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n_entries = a.count ? (int64_t)*a.count : a.n_static;
    unsigned long long pruned = 0;
    for (int64_t e = warp; e < n_entries; e += nwarps) {
        const uint32_t pid = a.pairs[e];
        if (pid == 0xffffffffu) continue;
        const float cur = a.lb[e];
        if (!(cur < TC_INF)) continue;
        const int64_t m = pid / (uint64_t)a.N, n = pid - m * a.N;
        const unsigned long long key = ld_volatile_u64(bsf + m);
        if (cur > prune_threshold(key, rho)) continue;  // dropped (and counted) by the DTW stage
        if (!(cur > e_gate * best_dist(key))) continue;
        const float bound = lb_ti_rows_pair<DMAX, NS>(a.C + (size_t)n * a.L * a.D, a.Q + (size_t)m * a.L * a.D,
                                                      dq_lo + (size_t)m * a.L, dq_hi + (size_t)m * a.L, a.L, a.D,
                                                      a.W, P);
        const bool dropped = __shfl_sync(0xffffffffu, bound > prune_threshold(ld_volatile_u64(bsf + m), rho), 0);
        if (lane == 0) {
            if (dropped) { a.lb[e] = TC_INF; ++pruned; }
            else a.lb[e] = fmaxf(cur, bound);
        }
    }
    if (lane == 0 && pruned && stat_pruned) atomicAdd(stat_pruned, pruned);
}

#define TC_DMAX_DISPATCH(D, CALL) \
    do {                          \
        if ((D) <= 8) { CALL(8); }        \
        else if ((D) <= 16) { CALL(16); } \
        else if ((D) <= 32) { CALL(32); } \
        else { CALL(64); }                \
    } while (0)

static int list_blocks(int64_t n_entries_hint, int sms) {
    int64_t b = (n_entries_hint + 3) / 4;  // 4 warps per block
    const int64_t cap = (int64_t)sms * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_lb_pc_list(const PairListArgs &a, const float *boxes, const int32_t *counts, int K, int w,
                              const unsigned long long *bsf, float rho, float e_gate, unsigned long long *stat_pruned,
                              int64_t n_hint, int sms, cudaStream_t s) {
    const int blocks = list_blocks(n_hint, sms);
#define TC_PC_CALL(DM) k_lb_pc_list<DM><<<blocks, 128, 0, s>>>(a, boxes, counts, K, w, bsf, rho, e_gate, stat_pruned)
    TC_DMAX_DISPATCH(a.D, TC_PC_CALL); note_launch();
#undef TC_PC_CALL
    return cudaGetLastError();
}

cudaError_t launch_lb_ti_list(const PairListArgs &a, const float *dq_lo, const float *dq_hi, int P,
                              const unsigned long long *bsf, float rho, float e_gate, unsigned long long *stat_pruned,
                              int64_t n_hint, int sms, cudaStream_t s) {
    // the entry count is on the device (the hint is a guess): a full grid, runs taken
    // by striding
    (void)n_hint;
    const int blocks = sms * 16;
    const size_t sq = (size_t)a.L * (a.D + 2) * sizeof(float);
    const int stage = sq <= 32 * 1024;  // the staged query in shared memory (else global memory)
#define TC_TI_CALL(DM) \
    k_lb_ti_list<DM><<<blocks, 128, stage ? sq : 0, s>>>(a, dq_lo, dq_hi, P, bsf, rho, e_gate, stat_pruned, stage)
    TC_DMAX_DISPATCH(a.D, TC_TI_CALL); note_launch();
#undef TC_TI_CALL
    return cudaGetLastError();
}

bool lb_ti_rows_supported(int W) { return W <= 127; }

cudaError_t launch_lb_ti_rows_list(const PairListArgs &a, const float *dq_lo, const float *dq_hi, int P,
                                   const unsigned long long *bsf, float rho, float e_gate,
                                   unsigned long long *stat_pruned, int64_t n_hint, int sms, cudaStream_t s) {
    if (!lb_ti_rows_supported(a.W)) return cudaErrorInvalidValue;
    const int blocks = list_blocks(n_hint, sms);
    const int w2 = 2 * a.W + 1;
#define TC_TIR_NS(DM, NSV) \
    k_lb_ti_rows_list<DM, NSV><<<blocks, 128, 0, s>>>(a, dq_lo, dq_hi, P, bsf, rho, e_gate, stat_pruned)
#define TC_TIR_CALL(DM)                          \
    do {                                         \
        if (w2 <= 32) TC_TIR_NS(DM, 1);          \
        else if (w2 <= 64) TC_TIR_NS(DM, 2);     \
        else if (w2 <= 128) TC_TIR_NS(DM, 4);    \
        else TC_TIR_NS(DM, 8);                   \
    } while (0)
    TC_DMAX_DISPATCH(a.D, TC_TIR_CALL);
    note_launch();
#undef TC_TIR_CALL
#undef TC_TIR_NS
    return cudaGetLastError();
}

// ============================================================== reverse LB_MV on listed pairs
// Candidate-side LB_MV (the bound with the roles of query and candidate exchanged:
// Section 3's envelope is taken around the candidate and the query's points are
// measured against it).  One warp per entry; the candidate envelopes Uc, Lc [N][L*D]
// are computed once per index.  Per element m = max(q -rd Uc, Lc -rd q, 0), m*m added
// rounded down; every 512 elements the warp's partial sum (rounded down) is compared
// with the live threshold and the pair is dropped as soon as it exceeds it.  A kept
// pair's bound becomes max(its bound, reverse bound): both are lower bounds of DTW.
__global__ void __launch_bounds__(128) k_lb_rev_list(PairListArgs a, const float *__restrict__ Uc,
                                                     const float *__restrict__ Lc, const unsigned long long *bsf,
                                                     float rho, unsigned long long *stat_pruned) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n_entries = a.count ? (int64_t)*a.count : a.n_static;
    const int64_t E = (int64_t)a.L * a.D;
    unsigned long long pruned = 0;
    for (int64_t e = warp; e < n_entries; e += nwarps) {
        const uint32_t pid = a.pairs[e];
        if (pid == 0xffffffffu) continue;
        const float cur = a.lb[e];
        if (!(cur < TC_INF)) continue;
        const int64_t m = pid / (uint64_t)a.N, n = pid - m * a.N;
        const float *q = a.Q + (size_t)m * E;
        const float *hi = Uc + (size_t)n * E, *lo = Lc + (size_t)n * E;
        float thr = bsf ? prune_threshold(ld_volatile_u64(bsf + m), rho) : TC_INF;
        if (cur > thr) continue;  // dropped (and counted) by the DTW stage
        float acc = 0.f, total = 0.f;
        bool dropped = false;
        for (int64_t c0 = 0; c0 < E && !dropped; c0 += 512) {
            const int64_t c1 = c0 + 512 < E ? c0 + 512 : E;
            for (int64_t k = c0 + lane; k < c1; k += 32) acc = acc_box(__ldg(q + k), __ldg(lo + k), __ldg(hi + k), acc);
            float t = acc;
            for (int o = 16; o > 0; o >>= 1) t = __fadd_rd(t, __shfl_xor_sync(0xffffffffu, t, o));
            total = t;
            if (bsf) thr = prune_threshold(ld_volatile_u64(bsf + m), rho);
            dropped = __shfl_sync(0xffffffffu, total > thr, 0);
        }
        if (lane == 0) {
            if (dropped) { a.lb[e] = TC_INF; ++pruned; }
            else a.lb[e] = fmaxf(cur, total);
        }
    }
    if (lane == 0 && pruned && stat_pruned) atomicAdd(stat_pruned, pruned);
}

cudaError_t launch_lb_rev_list(const PairListArgs &a, const float *Uc, const float *Lc, const unsigned long long *bsf,
                               float rho, unsigned long long *stat_pruned, int64_t n_hint, int sms, cudaStream_t s) {
    const int blocks = list_blocks(n_hint, sms);
    k_lb_rev_list<<<blocks, 128, 0, s>>>(a, Uc, Lc, bsf, rho, stat_pruned);
    note_launch();
    return cudaGetLastError();
}

// ============================================================== refine and select
// Entries of a list whose FP32 DTW is within the final threshold join the refine
// list (their FP64 DTW decides the winner).
__global__ void k_refine_select(const uint32_t *__restrict__ pairs, const float *__restrict__ dtw,
                                const int32_t *count, int64_t n_static, int64_t N, const unsigned long long *bsf,
                                float rho, uint32_t *__restrict__ out, int32_t *__restrict__ out_count,
                                int64_t cap) {
    const int64_t n_entries = count ? (int64_t)*count : n_static;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_entries;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t pid = pairs[e];
        if (pid == 0xffffffffu) continue;
        const float d = dtw[e];
        if (!(d < TC_INF)) continue;
        const int64_t m = pid / (uint64_t)N;
        if (d <= prune_threshold(bsf[m], rho)) {
            const int pos = atomicAdd(out_count, 1);
            if (pos < cap) out[pos] = pid;
        }
    }
}

// best index among refine entries whose FP64 DTW equals the row's minimum
__global__ void k_refine_pick(const uint32_t *__restrict__ pairs, const double *__restrict__ d64,
                              const int32_t *count, int64_t N, const unsigned long long *__restrict__ best64,
                              unsigned long long *__restrict__ best_idx) {
    const int64_t n_entries = *count;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_entries;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t pid = pairs[e];
        const int64_t m = pid / (uint64_t)N, n = pid - m * N;
        if ((unsigned long long)__double_as_longlong(d64[e]) == best64[m]) atomicMin(best_idx + m, (unsigned long long)n);
    }
}

// The double-float values of a query's refine entries cannot order the entries
// whose values lie within kappa of the best one (or any entry, when no value is
// finite): those queries take the FP64 recompute.
__device__ __forceinline__ bool needs_fp64(int amb, unsigned long long bestdf) {
    return amb >= 2 || !(__longlong_as_double((long long)bestdf) < __longlong_as_double(0x7ff0000000000000LL));
}

// Per refine entry: count the entries that the double-float values cannot separate
// from the best one (v <= bestdf * kappa, rounded up), and take the smallest
// index among the entries at the best value.
__global__ void k_refine_amb(const uint32_t *__restrict__ pairs, const double *__restrict__ v, const int32_t *count,
                             int64_t N, const unsigned long long *__restrict__ bestdf, double kappa,
                             int32_t *__restrict__ amb, unsigned long long *__restrict__ best_idx_df) {
    const int64_t n_entries = *count;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_entries;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t pid = pairs[e];
        const int64_t m = pid / (uint64_t)N, n = pid - m * N;
        const unsigned long long b = bestdf[m];
        const double x = v[e];
        if (!(x > __dmul_ru(__longlong_as_double((long long)b), kappa))) atomicAdd(amb + m, 1);
        if ((unsigned long long)__double_as_longlong(x) == b) atomicMin(best_idx_df + m, (unsigned long long)n);
    }
}

// Refine entries of the queries that need FP64 and lie within kappa of the best
// double-float value join the FP64 list.
__global__ void k_refine_need64(const uint32_t *__restrict__ pairs, const double *__restrict__ v,
                                const int32_t *count, int64_t N, const unsigned long long *__restrict__ bestdf,
                                double kappa, const int32_t *__restrict__ amb, uint32_t *__restrict__ out,
                                int32_t *__restrict__ out_count, int64_t cap) {
    const int64_t n_entries = *count;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_entries;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t pid = pairs[e];
        const int64_t m = pid / (uint64_t)N;
        const unsigned long long b = bestdf[m];
        if (!needs_fp64(amb[m], b)) continue;
        if (!(v[e] > __dmul_ru(__longlong_as_double((long long)b), kappa))) {
            const int pos = atomicAdd(out_count, 1);
            if (pos < cap) out[pos] = pid;
        }
    }
}

__global__ void k_finalize(int64_t Mb, const unsigned long long *__restrict__ bestdf,
                           const unsigned long long *__restrict__ best_idx_df, const int32_t *__restrict__ amb,
                           const unsigned long long *__restrict__ best64,
                           const unsigned long long *__restrict__ best_idx, int64_t *__restrict__ idx,
                           double *__restrict__ dist) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Mb) return;
    if (needs_fp64(amb[m], bestdf[m])) {
        idx[m] = (int64_t)best_idx[m];
        dist[m] = __longlong_as_double((long long)best64[m]);
    } else {
        idx[m] = (int64_t)best_idx_df[m];
        dist[m] = __longlong_as_double((long long)bestdf[m]);
    }
}

__global__ void k_init_block(int64_t Mb, unsigned long long *bsf, unsigned long long *best64,
                             unsigned long long *best_idx, unsigned long long *bestdf,
                             unsigned long long *best_idx_df, int32_t *amb) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Mb) return;
    bsf[m] = pack_best(TC_INF, 0xffffffffu);  // +inf: every finite distance is smaller
    if (best64) best64[m] = 0x7ff0000000000000ull;
    if (best_idx) best_idx[m] = ~0ull;
    if (bestdf) bestdf[m] = 0x7ff0000000000000ull;
    if (best_idx_df) best_idx_df[m] = ~0ull;
    if (amb) amb[m] = 0;
}

__global__ void k_count_add(unsigned long long *acc, const int32_t *v) { *acc += (unsigned long long)*v; }

__global__ void k_iota_pairs(uint32_t *p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (uint32_t)i;
}

cudaError_t launch_count_add(unsigned long long *acc, const int32_t *v, cudaStream_t s) {
    k_count_add<<<1, 1, 0, s>>>(acc, v); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_iota_pairs(uint32_t *p, int64_t n, cudaStream_t s) {
    int64_t b = (n + 255) / 256;
    if (b > 65535) b = 65535;
    k_iota_pairs<<<(unsigned)b, 256, 0, s>>>(p, n); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_refine_select(const uint32_t *pairs, const float *dtw, const int32_t *count, int64_t n_static,
                                 int64_t N, const unsigned long long *bsf, float rho, uint32_t *out,
                                 int32_t *out_count, int64_t cap, int sms, cudaStream_t s) {
    k_refine_select<<<sms * 4, 256, 0, s>>>(pairs, dtw, count, n_static, N, bsf, rho, out, out_count, cap); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_refine_pick(const uint32_t *pairs, const double *d64, const int32_t *count, int64_t N,
                               const unsigned long long *best64, unsigned long long *best_idx, int sms,
                               cudaStream_t s) {
    k_refine_pick<<<sms, 256, 0, s>>>(pairs, d64, count, N, best64, best_idx); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_refine_amb(const uint32_t *pairs, const double *v, const int32_t *count, int64_t N,
                              const unsigned long long *bestdf, double kappa, int32_t *amb,
                              unsigned long long *best_idx_df, int sms, cudaStream_t s) {
    k_refine_amb<<<sms, 256, 0, s>>>(pairs, v, count, N, bestdf, kappa, amb, best_idx_df); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_refine_need64(const uint32_t *pairs, const double *v, const int32_t *count, int64_t N,
                                 const unsigned long long *bestdf, double kappa, const int32_t *amb, uint32_t *out,
                                 int32_t *out_count, int64_t cap, int sms, cudaStream_t s) {
    k_refine_need64<<<sms, 256, 0, s>>>(pairs, v, count, N, bestdf, kappa, amb, out, out_count, cap); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_finalize(int64_t Mb, const unsigned long long *bestdf, const unsigned long long *best_idx_df,
                            const int32_t *amb, const unsigned long long *best64, const unsigned long long *best_idx,
                            int64_t *idx, double *dist, cudaStream_t s) {
    k_finalize<<<(unsigned)((Mb + 255) / 256), 256, 0, s>>>(Mb, bestdf, best_idx_df, amb, best64, best_idx, idx,
                                                            dist); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_init_block(int64_t Mb, unsigned long long *bsf, unsigned long long *best64,
                              unsigned long long *best_idx, unsigned long long *bestdf,
                              unsigned long long *best_idx_df, int32_t *amb, cudaStream_t s) {
    k_init_block<<<(unsigned)((Mb + 255) / 256), 256, 0, s>>>(Mb, bsf, best64, best_idx, bestdf, best_idx_df, amb);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tc
