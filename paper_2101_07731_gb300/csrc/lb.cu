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
constexpr int kMvRows = 128;
constexpr int kMvChunk = 32;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem, int src_bytes) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

typedef unsigned long long f2;
__device__ __forceinline__ f2 pk(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 sub2_rd(f2 a, f2 b) {
    f2 r;
    asm("sub.rm.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 fma2_rd(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rm.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f2 add2_rd(f2 a, f2 b) {
    f2 r;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// squared distance of x to [lo, hi], rounded down, accumulated into acc
__device__ __forceinline__ float acc_box(float x, float lo, float hi, float acc) {
    const float m = max3f(__fsub_rd(x, hi), __fsub_rd(lo, x), 0.f);
    return __fmaf_rd(m, m, acc);
}

// one packed step: element value c2 = {x, x} against two queries' (U, Lo)
__device__ __forceinline__ f2 mv_step(f2 c2, float u0, float u1, float l0, float l1, f2 part) {
    float a0, a1, b0, b1;
    upk(sub2_rd(c2, pk(u0, u1)), a0, a1);
    upk(sub2_rd(pk(l0, l1), c2), b0, b1);
    const float m0 = max3f(a0, b0, 0.f), m1 = max3f(a1, b1, 0.f);
    const f2 m2 = pk(m0, m1);
    return fma2_rd(m2, m2, part);
}

template <int QB>
__device__ __forceinline__ void mv_issue(const float *__restrict__ cand, int64_t N, int E, bool vec4,
                                         const float *UI, const float *LI, int64_t ldE, int n_qp, int64_t n0, int q0,
                                         int e0, float *sc, float *su, float *sl) {
    const int tid = threadIdx.x;
    if (vec4) {
#pragma unroll
        for (int k = 0; k < (kMvRows * 8) / 128; ++k) {
            const int idx = tid + 128 * k;
            const int row = idx >> 3, seg = idx & 7;
            const int64_t n = n0 + row;
            const int e = e0 + seg * 4;
            const bool ok = n < N && e < E;
            const float *src = ok ? cand + (size_t)n * E + e : cand;
            cp_async16(sc + row * kMvChunk + ((seg ^ (row & 7)) << 2), src, ok ? 16 : 0);
        }
    } else {
        for (int k = 0; k < kMvRows * kMvChunk / 128; ++k) {
            const int idx = tid + 128 * k;
            const int row = idx >> 5, el = idx & 31;
            const int64_t n = n0 + row;
            const int e = e0 + el;
            const bool ok = n < N && e < E;
            const float *src = ok ? cand + (size_t)n * E + e : cand;
            const int seg = el >> 2;
            cp_async4(sc + row * kMvChunk + ((seg ^ (row & 7)) << 2) + (el & 3), src, ok ? 4 : 0);
        }
    }
    // envelope chunk: QB/2 query pairs x 32 elements x 2 floats (256 bytes), U and Lo
    for (int idx = tid; idx < (QB / 2) * 16 * 2; idx += 128) {
        const int which = idx / ((QB / 2) * 16);
        const int r = idx % ((QB / 2) * 16);
        const int qp = r >> 4, seg = r & 15;
        const int qpg = min(q0 / 2 + qp, n_qp - 1);
        const float *src = (which ? LI : UI) + ((size_t)qpg * ldE + e0) * 2 + seg * 4;
        cp_async16((which ? sl : su) + qp * 2 * kMvChunk + seg * 4, src, 16);
    }
}

template <int QB>
__global__ void __launch_bounds__(128) k_lb_mv(const float *__restrict__ cand, int64_t N, int E, int vec4,
                                               const float *__restrict__ UI, const float *__restrict__ LI,
                                               int64_t ldE, int Mb, float *__restrict__ lb, int64_t ldLb,
                                               int n_ctiles, int n_qtiles) {
    __shared__ __align__(16) float sc[2][kMvRows * kMvChunk];
    __shared__ __align__(16) float su[2][QB * kMvChunk];
    __shared__ __align__(16) float sl[2][QB * kMvChunk];
    const int tid = threadIdx.x;
    const int nchunks = (E + kMvChunk - 1) / kMvChunk;
    const int ntiles = n_ctiles * n_qtiles;
    const int n_qp = (Mb + 1) / 2;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int ct = tile / n_qtiles, qt = tile % n_qtiles;
        const int64_t n0 = (int64_t)ct * kMvRows;
        const int q0 = qt * QB;
        f2 acc[QB / 2];
#pragma unroll
        for (int k = 0; k < QB / 2; ++k) acc[k] = 0ull;
        mv_issue<QB>(cand, N, E, vec4, UI, LI, ldE, n_qp, n0, q0, 0, sc[0], su[0], sl[0]);
        cp_async_commit();
        for (int c = 0; c < nchunks; ++c) {
            const int buf = c & 1;
            if (c + 1 < nchunks) {
                mv_issue<QB>(cand, N, E, vec4, UI, LI, ldE, n_qp, n0, q0, (c + 1) * kMvChunk, sc[buf ^ 1],
                             su[buf ^ 1], sl[buf ^ 1]);
                cp_async_commit();
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            f2 c2[kMvChunk];
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const float4 v = *reinterpret_cast<const float4 *>(&sc[buf][tid * kMvChunk + ((s ^ (tid & 7)) << 2)]);
                c2[4 * s] = pk(v.x, v.x);
                c2[4 * s + 1] = pk(v.y, v.y);
                c2[4 * s + 2] = pk(v.z, v.z);
                c2[4 * s + 3] = pk(v.w, v.w);
            }
#pragma unroll
            for (int qp = 0; qp < QB / 2; ++qp) {
                f2 part = 0ull;
                const float *u = &su[buf][qp * 2 * kMvChunk];
                const float *l = &sl[buf][qp * 2 * kMvChunk];
#pragma unroll
                for (int e = 0; e < kMvChunk; e += 2) {
                    const float4 u4 = *reinterpret_cast<const float4 *>(u + 2 * e);
                    const float4 l4 = *reinterpret_cast<const float4 *>(l + 2 * e);
                    part = mv_step(c2[e], u4.x, u4.y, l4.x, l4.y, part);
                    part = mv_step(c2[e + 1], u4.z, u4.w, l4.z, l4.w, part);
                }
                acc[qp] = add2_rd(acc[qp], part);
            }
            __syncthreads();
        }
        const int64_t n = n0 + tid;
        if (n < N) {
#pragma unroll
            for (int qp = 0; qp < QB / 2; ++qp) {
                float a0, a1;
                upk(acc[qp], a0, a1);
                if (q0 + 2 * qp < Mb) lb[(size_t)(q0 + 2 * qp) * ldLb + n] = a0;
                if (q0 + 2 * qp + 1 < Mb) lb[(size_t)(q0 + 2 * qp + 1) * ldLb + n] = a1;
            }
        }
    }
}

bool lb_mv_vec4(const float *cand, int E) { return (E % 4) == 0 && (((uintptr_t)cand) & 15) == 0; }

cudaError_t launch_lb_mv(const LbMvArgs &a, cudaStream_t s) {
    if (a.N <= 0 || a.Mb <= 0) return cudaSuccess;
    const int vec4 = lb_mv_vec4(a.cand, a.E);
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
        k_lb_mv<QBV><<<(int)grid, 128, 0, s>>>(a.cand, a.N, a.E, vec4, a.U, a.Lo, a.ldE, a.Mb, a.lb, a.ldLb, \
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

// count pass: one CTA per row
__global__ void k_count_rows(const float *__restrict__ lb, int64_t N, int64_t ldLb, const float *thresh,
                             const unsigned long long *bsf, float rho, int32_t *__restrict__ counts,
                             unsigned long long *pruned) {
    const int64_t m = blockIdx.x;
    const float thr = row_thr(thresh, bsf, rho, m);
    const float *row = lb + (size_t)m * ldLb;
    int c = 0;
    for (int64_t n = threadIdx.x; n < N; n += blockDim.x) c += (row[n] <= thr);
    __shared__ int red[32];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
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

// write pass: one CTA (256 threads) per row, survivors in increasing n.  Output
// position of row m's k-th survivor: base(m) + k with base(m) = offsets[m] (flat
// list) or m * ldOut (per-row lists).  pairs (flat) receive m*N + n and lbs the
// bound; idx_out (per-row) receives n.
__global__ void k_write_rows(const float *__restrict__ lb, int64_t N, int64_t ldLb, const float *thresh,
                             const unsigned long long *bsf, float rho, const int32_t *__restrict__ offsets,
                             int64_t ldOut, uint32_t *__restrict__ pairs, float *__restrict__ lbs,
                             int32_t *__restrict__ idx_out) {
    const int64_t m = blockIdx.x;
    const float thr = row_thr(thresh, bsf, rho, m);
    const float *row = lb + (size_t)m * ldLb;
    const int64_t base = offsets ? (int64_t)offsets[m] : m * ldOut;
    __shared__ int wsum[8];
    __shared__ int running;
    if (threadIdx.x == 0) running = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t n0 = 0; n0 < N; n0 += 256) {
        const int64_t n = n0 + threadIdx.x;
        const float v = n < N ? row[n] : TC_INF;
        const bool keep = n < N && v <= thr;
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int before = running;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        if (keep) {
            const int64_t pos = base + before + __popc(bal & ((1u << lane) - 1u));
            if (pairs) {
                pairs[pos] = (uint32_t)(m * N + n);
                lbs[pos] = v;
            } else {
                idx_out[pos] = (int32_t)n;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < 8; ++w) t += wsum[w];
            running += t;
        }
        __syncthreads();
    }
}

cudaError_t launch_compact(const CompactArgs &a, cudaStream_t s) {
    if (a.M <= 0) return cudaSuccess;
    k_count_rows<<<(unsigned)a.M, 256, 0, s>>>(a.lb, a.N, a.ldLb, a.thresh, a.bsf, a.rho, a.counts, a.pruned); note_launch();
    if (a.offsets) {
        k_scan_counts<<<1, 1024, 0, s>>>(a.counts, a.M, a.offsets, a.total);
        note_launch();
    }
    k_write_rows<<<(unsigned)a.M, 256, 0, s>>>(a.lb, a.N, a.ldLb, a.thresh, a.bsf, a.rho, a.offsets, a.ldOut, a.pairs,
                                                a.lbs, a.idx_out); note_launch();
    return cudaGetLastError();
}

// ============================================================== seeds
// Per row m (one CTA of 256 threads): the S candidates with the smallest bound
// (ties: smaller n) become seed entries m*N + n (empty slots: UINT32_MAX), and
// their bound in the row is replaced by +inf so they do not survive compaction.
constexpr int kMaxSeeds = 8;

__device__ __forceinline__ bool lex_less(float a, uint32_t ia, float b, uint32_t ib) {
    return a < b || (a == b && ia < ib);
}

__global__ void k_seed_topk(float *__restrict__ lb, int64_t N, int64_t ldLb, int S, uint32_t *__restrict__ seeds) {
    const int64_t m = blockIdx.x;
    float *row = lb + (size_t)m * ldLb;
    float bv[kMaxSeeds];
    uint32_t bi[kMaxSeeds];
#pragma unroll
    for (int k = 0; k < kMaxSeeds; ++k) { bv[k] = TC_INF; bi[k] = 0xffffffffu; }
    for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
        float v = row[n];
        uint32_t iv = (uint32_t)n;
        if (!(v < TC_INF)) continue;
#pragma unroll
        for (int k = 0; k < kMaxSeeds; ++k) {  // insertion into the sorted local list
            if (k < S && lex_less(v, iv, bv[k], bi[k])) {
                float tv = bv[k]; uint32_t ti = bi[k];
                bv[k] = v; bi[k] = iv;
                v = tv; iv = ti;
            }
        }
    }
    __shared__ float cv[256 / 32][kMaxSeeds];
    __shared__ uint32_t ci[256 / 32][kMaxSeeds];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int head = 0;
    // warp level: S rounds of arg-min over the lanes' list heads
    for (int r = 0; r < S; ++r) {
        float v = head < S ? bv[0] : TC_INF;
        uint32_t iv = head < S ? bi[0] : 0xffffffffu;
        float wv = v; uint32_t wi = iv;
        for (int o = 16; o > 0; o >>= 1) {
            float ov = __shfl_xor_sync(0xffffffffu, wv, o);
            uint32_t oi = __shfl_xor_sync(0xffffffffu, wi, o);
            if (lex_less(ov, oi, wv, wi)) { wv = ov; wi = oi; }
        }
        if (lane == 0) { cv[warp][r] = wv; ci[warp][r] = wi; }
        if (wi == iv && wi != 0xffffffffu) {  // this lane's head won: pop it
#pragma unroll
            for (int k = 0; k + 1 < kMaxSeeds; ++k) { bv[k] = bv[k + 1]; bi[k] = bi[k + 1]; }
            bv[kMaxSeeds - 1] = TC_INF; bi[kMaxSeeds - 1] = 0xffffffffu;
            ++head;
        }
    }
    __syncthreads();
    if (warp == 0) {
        // merge the per-warp lists (each sorted): lane l < 8 walks warp l's list
        int pos = 0;
        const int nw = blockDim.x >> 5;
        for (int r = 0; r < S; ++r) {
            float v = (lane < nw && pos < S) ? cv[lane][pos] : TC_INF;
            uint32_t iv = (lane < nw && pos < S) ? ci[lane][pos] : 0xffffffffu;
            float wv = v; uint32_t wi = iv;
            for (int o = 16; o > 0; o >>= 1) {
                float ov = __shfl_xor_sync(0xffffffffu, wv, o);
                uint32_t oi = __shfl_xor_sync(0xffffffffu, wi, o);
                if (lex_less(ov, oi, wv, wi)) { wv = ov; wi = oi; }
            }
            if (wi == iv && wi != 0xffffffffu) ++pos;
            if (lane == 0) {
                seeds[m * S + r] = (wi == 0xffffffffu) ? 0xffffffffu : (uint32_t)(m * N + wi);
                if (wi != 0xffffffffu) row[wi] = TC_INF;
            }
        }
    }
}

cudaError_t launch_seed_topk(float *lb, int64_t M, int64_t N, int64_t ldLb, int S, uint32_t *seeds, cudaStream_t s) {
    if (M <= 0 || S <= 0) return cudaSuccess;
    if (S > kMaxSeeds) S = kMaxSeeds;
    k_seed_topk<<<(unsigned)M, 256, 0, s>>>(lb, N, ldLb, S, seeds); note_launch();
    return cudaGetLastError();
}

// ============================================================== LB_PC / LB_TI on listed pairs
// One warp per entry.  Entry e (e < *count): pair id pairs[e] = m*N + n and its
// current bound lbv[e] (+inf: already dropped).  The gate of selective deployment
// (Section 6): the tight bound runs only if e_gate * bsf < lbv[e] <= threshold.
// A pair whose bound exceeds the threshold gets lbv[e] = +inf.
__device__ __forceinline__ float warp_sum_rd(float v) {
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rd(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <int DMAX>
__global__ void __launch_bounds__(128) k_lb_pc_list(PairListArgs a, const float *__restrict__ boxes,
                                                    const int32_t *__restrict__ counts, int K, int w,
                                                    const unsigned long long *bsf, float rho, float e_gate,
                                                    unsigned long long *stat_pruned) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n_entries = a.count ? (int64_t)*a.count : a.n_static;
    const int L = a.L, D = a.D;
    const int G = (L + w - 1) / w;
    unsigned long long pruned = 0;
    for (int64_t e = warp; e < n_entries; e += nwarps) {
        const uint32_t pid = a.pairs[e];
        if (pid == 0xffffffffu) continue;
        const float cur = a.lb[e];
        if (!(cur < TC_INF)) continue;
        const int64_t m = pid / (uint64_t)a.N, n = pid - m * a.N;
        const unsigned long long key = ld_volatile_u64(bsf + m);
        const float thr = prune_threshold(key, rho);
        if (cur > thr) continue;  // dropped (and counted) when the DTW stage fetches it
        if (!(cur > e_gate * best_dist(key))) continue;
        const float *c = a.C + (size_t)n * L * D;
        const float *bx_m = boxes + (size_t)m * G * K * 2 * D;
        const int32_t *cnt_m = counts + (size_t)m * G;
        float acc = 0.f;
        bool dropped = false;
        for (int j0 = 0; j0 < L; j0 += 32) {
            const int j = j0 + lane;
            if (j < L) {
                float x[DMAX];
#pragma unroll
                for (int p = 0; p < DMAX; ++p) x[p] = p < D ? __ldg(c + (size_t)j * D + p) : 0.f;
                const int g = j / w;
                const int nb = cnt_m[g];
                const float *bx = bx_m + (size_t)g * K * 2 * D;
                float best = TC_INF;
                for (int k = 0; k < nb; ++k) {
                    float s = 0.f;
#pragma unroll
                    for (int p = 0; p < DMAX; ++p)
                        if (p < D) s = acc_box(x[p], __ldg(bx + k * 2 * D + p), __ldg(bx + k * 2 * D + D + p), s);
                    best = fminf(best, s);
                }
                acc = __fadd_rd(acc, best);
            }
            const float tot = warp_sum_rd(acc);
            if (tot > prune_threshold(ld_volatile_u64(bsf + m), rho)) { dropped = true; break; }
        }
        const float tot = warp_sum_rd(acc);
        if (lane == 0) {
            if (dropped) { a.lb[e] = TC_INF; ++pruned; }
            else a.lb[e] = fmaxf(cur, tot);
        }
    }
    if (lane == 0 && pruned && stat_pruned) atomicAdd(stat_pruned, pruned);
}

// LB_TI (TIP_TOP).  Lane = candidate point j (column of the cost matrix).  The
// rows of its window are i in [i0, i1] = [max(0, j-W), min(L-1, j+W)].  Row i0 is
// exact (it is either the top of the window of row i0 = j-W, or row 0, and
// 0 mod P == 0); rows with i mod P == 0 are exact; the others follow
//   Lb = max(Lb_prev - dq_i, dq_i - Ub_prev, 0),  Ub = Ub_prev + dq_i
// with dq_i taken rounded up where it is subtracted from Lb / added to Ub and
// rounded down where Ub is subtracted from it.  m_j = min Lb; bound = sum m_j^2.
template <int DMAX>
__device__ __forceinline__ void exact_interval(const float *__restrict__ qi, const float (&x)[DMAX], int D, float *lo,
                                               float *hi) {
    float sl = 0.f, sh = 0.f;
#pragma unroll
    for (int p = 0; p < DMAX; ++p) {
        if (p < D) {
            const float y = __ldg(qi + p);
            const float dl = fmaxf(__fsub_rd(x[p], y), __fsub_rd(y, x[p]));
            const float dh = fmaxf(__fsub_ru(x[p], y), __fsub_ru(y, x[p]));
            sl = __fmaf_rd(dl, dl, sl);
            sh = __fmaf_ru(dh, dh, sh);
        }
    }
    *lo = __fsqrt_rd(sl);
    *hi = __fsqrt_ru(sh);
}

template <int DMAX>
__global__ void __launch_bounds__(128) k_lb_ti_list(PairListArgs a, const float *__restrict__ dq_lo,
                                                    const float *__restrict__ dq_hi, int P,
                                                    const unsigned long long *bsf, float rho, float e_gate,
                                                    unsigned long long *stat_pruned) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n_entries = a.count ? (int64_t)*a.count : a.n_static;
    const int L = a.L, D = a.D, W = a.W;
    unsigned long long pruned = 0;
    for (int64_t e = warp; e < n_entries; e += nwarps) {
        const uint32_t pid = a.pairs[e];
        if (pid == 0xffffffffu) continue;
        const float cur = a.lb[e];
        if (!(cur < TC_INF)) continue;
        const int64_t m = pid / (uint64_t)a.N, n = pid - m * a.N;
        const unsigned long long key = ld_volatile_u64(bsf + m);
        const float thr = prune_threshold(key, rho);
        if (cur > thr) continue;  // dropped (and counted) when the DTW stage fetches it
        if (!(cur > e_gate * best_dist(key))) continue;
        const float *c = a.C + (size_t)n * L * D;
        const float *q = a.Q + (size_t)m * L * D;
        const float *dql = dq_lo + (size_t)m * L, *dqh = dq_hi + (size_t)m * L;
        float acc = 0.f;
        bool dropped = false;
        for (int j0 = 0; j0 < L; j0 += 32) {
            const int j = j0 + lane;
            if (j < L) {
                float x[DMAX];
#pragma unroll
                for (int p = 0; p < DMAX; ++p) x[p] = p < D ? __ldg(c + (size_t)j * D + p) : 0.f;
                const int i0 = max(0, j - W), i1 = min(L - 1, j + W);
                float lbv, ubv;
                exact_interval<DMAX>(q + (size_t)i0 * D, x, D, &lbv, &ubv);
                float mj = lbv;
                int next_exact = (i0 / P + 1) * P;
                for (int i = i0 + 1; i <= i1; ++i) {
                    if (i == next_exact) {
                        exact_interval<DMAX>(q + (size_t)i * D, x, D, &lbv, &ubv);
                        next_exact += P;
                    } else {
                        const float dl = __ldg(dql + i), dh = __ldg(dqh + i);
                        const float nl = fmaxf(fmaxf(__fsub_rd(lbv, dh), __fsub_rd(dl, ubv)), 0.f);
                        ubv = __fadd_ru(ubv, dh);
                        lbv = nl;
                    }
                    mj = fminf(mj, lbv);
                }
                acc = __fmaf_rd(mj, mj, acc);
            }
            const float tot = warp_sum_rd(acc);
            if (tot > prune_threshold(ld_volatile_u64(bsf + m), rho)) { dropped = true; break; }
        }
        const float tot = warp_sum_rd(acc);
        if (lane == 0) {
            if (dropped) { a.lb[e] = TC_INF; ++pruned; }
            else a.lb[e] = fmaxf(cur, tot);
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
    const int blocks = list_blocks(n_hint, sms);
#define TC_TI_CALL(DM) k_lb_ti_list<DM><<<blocks, 128, 0, s>>>(a, dq_lo, dq_hi, P, bsf, rho, e_gate, stat_pruned)
    TC_DMAX_DISPATCH(a.D, TC_TI_CALL); note_launch();
#undef TC_TI_CALL
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

__global__ void k_finalize(int64_t Mb, const unsigned long long *__restrict__ best64,
                           const unsigned long long *__restrict__ best_idx, int64_t *__restrict__ idx,
                           double *__restrict__ dist) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Mb) return;
    idx[m] = (int64_t)best_idx[m];
    dist[m] = __longlong_as_double((long long)best64[m]);
}

__global__ void k_init_block(int64_t Mb, unsigned long long *bsf, unsigned long long *best64,
                             unsigned long long *best_idx) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= Mb) return;
    bsf[m] = pack_best(TC_INF, 0xffffffffu);  // +inf: every finite distance is smaller
    if (best64) best64[m] = 0x7ff0000000000000ull;
    if (best_idx) best_idx[m] = ~0ull;
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
cudaError_t launch_finalize(int64_t Mb, const unsigned long long *best64, const unsigned long long *best_idx,
                            int64_t *idx, double *dist, cudaStream_t s) {
    k_finalize<<<(unsigned)((Mb + 255) / 256), 256, 0, s>>>(Mb, best64, best_idx, idx, dist); note_launch();
    return cudaGetLastError();
}
cudaError_t launch_init_block(int64_t Mb, unsigned long long *bsf, unsigned long long *best64,
                              unsigned long long *best_idx, cudaStream_t s) {
    k_init_block<<<(unsigned)((Mb + 255) / 256), 256, 0, s>>>(Mb, bsf, best64, best_idx); note_launch();
    return cudaGetLastError();
}

}  // namespace tc
