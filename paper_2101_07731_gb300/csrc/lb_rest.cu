// lb_rest.cu -- LB_MV with early abandoning (Section 7.1: abandoning applies to the
// lower-bound computations as well as to DTW).
//
// The dense stream (lb.cu) first sums the elements [0, E0) of every (query, candidate)
// pair.  A pair whose prefix sum already exceeds its query's threshold is abandoned
// there: every LB_MV term is >= 0, so the prefix sum is a lower bound of LB_MV, hence
// of DTW, and it already exceeds the threshold, which is all the search needs of it.
// The pairs left at or under the threshold (on nearest-neighbour workloads usually a
// small share) are completed here, over the elements [E0, E).
//
// CTA = TC candidates (TC <= kRestTC) x up to qg <= kRestQG queries.  The CTA lists the
// live (query, candidate) pairs of its tile (in a per-CTA global scratch region), then
// streams the elements [E0, E) of its candidates and of its queries' envelopes through
// shared memory in chunks of 32 (cp.async, double buffered; every 128-byte row stored
// with its 16-byte segments XOR-swizzled by row & 7, so that threads reading different
// rows mostly hit different banks); each thread advances up to kRestEpt listed pairs
// by one chunk per step.  Every kRestCheck chunks a pair whose running sum has passed
// the threshold is abandoned again (its partial sum is written, a lower bound above
// the threshold); a check that finds no listed pair left ends the stream.
// Rounding as in the dense stream: terms and sums rounded down, so every stored value
// is at most the exact LB_MV.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "lb_device.cuh"
#include "lb_kernels.cuh"

namespace tc {

namespace {

constexpr int kRestThreads = 512;
constexpr int kRestEpt = 4;                          // listed pairs per thread per round
constexpr int kRestRound = kRestThreads * kRestEpt;  // listed pairs per round
constexpr int kRestCheck = 16;                       // chunks between abandoning checks

// Two consecutive elements of one pair: c2 = {c_e, c_e+1} against {U_e, U_e+1},
// {Lo_e, Lo_e+1}; the squared excess of each is added (rounded down) into its half of
// part.
__device__ __forceinline__ f2 rest_step(f2 c2, f2 u2, f2 l2, f2 part) {
    float a0, a1, b0, b1;
    upk(sub2_rd(c2, u2), a0, a1);
    upk(sub2_rd(l2, c2), b0, b1);
    const float m0 = max3f(a0, b0, 0.f), m1 = max3f(a1, b1, 0.f);
    const f2 m2 = pk(m0, m1);
    return fma2_rd(m2, m2, part);
}

// Copies chunk [e0, e0+32) of the tile's candidates and queries into one buffer.
__device__ __forceinline__ void rest_issue(const LbMvRestArgs &a, int64_t n0, int tn, int q0, int nq, int e0,
                                           bool vec4, float *sc, float *se) {
    const int tid = threadIdx.x;
    if (vec4) {
        for (int idx = tid; idx < tn * 8; idx += kRestThreads) {
            const int row = idx >> 3, seg = idx & 7;
            const int64_t n = n0 + row;
            const int e = e0 + seg * 4;
            const bool ok = n < a.N && e < a.E;
            const float *src = ok ? a.cand + (size_t)n * a.ldC + e : a.cand;
            cp_async16(sc + row * 32 + ((seg ^ (row & 7)) << 2), src, ok ? 16 : 0);
        }
    } else {
        for (int idx = tid; idx < tn * 32; idx += kRestThreads) {
            const int row = idx >> 5, el = idx & 31;
            const int64_t n = n0 + row;
            const int e = e0 + el;
            const bool ok = n < a.N && e < a.E;
            const float *src = ok ? a.cand + (size_t)n * a.ldC + e : a.cand;
            cp_async4(sc + row * 32 + (((el >> 2) ^ (row & 7)) << 2) + (el & 3), src, ok ? 4 : 0);
        }
    }
    // envelope rows are padded with +inf / -inf up to ldP (a multiple of 32), so a
    // chunk that starts below E lies inside the row, and its elements >= E add 0
    for (int idx = tid; idx < nq * 16; idx += kRestThreads) {
        const int row = idx >> 4, h = (idx >> 3) & 1, seg = idx & 7;
        const float *src = (h ? a.Lp : a.Up) + (size_t)(q0 + row) * a.ldP + e0 + seg * 4;
        cp_async16(se + row * 64 + h * 32 + ((seg ^ (row & 7)) << 2), src, 16);
    }
}

__global__ void __launch_bounds__(kRestThreads, 1) k_lb_mv_rest(const LbMvRestArgs a, int tn, int qg, int vec4) {
    extern __shared__ __align__(16) float rs[];
    // buffer b: candidates at rs + b * tn * 32, envelopes at env0 + b * qg * 64
    float *const env0 = rs + 2 * tn * 32;
    float *thr = env0 + 2 * qg * 64;
    int *s_cnt = reinterpret_cast<int *>(thr + qg);
    uint32_t *list = a.list + (size_t)blockIdx.x * tn * qg;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nchunks = (a.E + kMvChunk - 1) / kMvChunk, c0 = a.E0 / kMvChunk;
    const int64_t n_tiles = (a.N + tn - 1) / tn;
    unsigned long long terms = 0;  // (element, pair) terms this thread summed
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t n0 = tile * tn;
        for (int q0 = 0; q0 < a.Mb; q0 += qg) {
            const int nq = min(qg, a.Mb - q0);
            __syncthreads();  // the previous pass is done with the thresholds and the list
            if (tid == 0) *s_cnt = 0;
            for (int k = tid; k < nq; k += kRestThreads)
                thr[k] = a.thresh ? a.thresh[q0 + k] : prune_threshold(ld_volatile_u64(a.bsf + q0 + k), a.rho);
            __syncthreads();
            // the live pairs of the tile; whole warps take part in every ballot
            // (nq * tn is a multiple of 32)
            for (int base = 0; base < nq * tn; base += kRestThreads) {
                const int idx = base + tid;
                const int ql = idx / tn, nl = idx - ql * tn;
                bool live = false;
                if (ql < nq && n0 + nl < a.N) {
                    const float v = a.lb[(size_t)(q0 + ql) * a.ldLb + n0 + nl];
                    live = v < TC_INF && v <= thr[ql];
                }
                const unsigned bal = __ballot_sync(0xffffffffu, live);
                int pos = 0;
                if (lane == 0 && bal) pos = atomicAdd(s_cnt, __popc(bal));
                pos = __shfl_sync(0xffffffffu, pos, 0);
                if (live) list[pos + __popc(bal & ((1u << lane) - 1u))] = ((uint32_t)ql << 16) | (uint32_t)nl;
            }
            __syncthreads();  // the list (global, this CTA's region) and its count
            const int cnt = *s_cnt;
            for (int r0 = 0; r0 < cnt; r0 += kRestRound) {
                int qk[kRestEpt], nk[kRestEpt];
                float acc[kRestEpt], th[kRestEpt];
                bool act[kRestEpt];
#pragma unroll
                for (int k = 0; k < kRestEpt; ++k) {
                    const int i = r0 + k * kRestThreads + tid;
                    act[k] = i < cnt;
                    const uint32_t en = act[k] ? __ldcg(list + i) : 0u;
                    qk[k] = (int)(en >> 16);
                    nk[k] = (int)(en & 0xffffu);
                    acc[k] = act[k] ? a.lb[(size_t)(q0 + qk[k]) * a.ldLb + n0 + nk[k]] : 0.f;
                    th[k] = thr[qk[k]];
                }
                rest_issue(a, n0, tn, q0, nq, c0 * kMvChunk, vec4, rs, env0);
                cp_async_commit();
                for (int c = c0; c < nchunks; ++c) {
                    const int buf = (c - c0) & 1;
                    if (c + 1 < nchunks) {
                        rest_issue(a, n0, tn, q0, nq, (c + 1) * kMvChunk, vec4, rs + (buf ^ 1) * tn * 32,
                                   env0 + (buf ^ 1) * qg * 64);
                        cp_async_commit();
                        cp_async_wait<1>();
                    } else {
                        cp_async_wait<0>();
                    }
                    __syncthreads();
#pragma unroll
                    for (int k = 0; k < kRestEpt; ++k) {
                        if (!act[k]) continue;
                        const float *cr = rs + buf * tn * 32 + nk[k] * 32;
                        const float *ur = env0 + buf * qg * 64 + qk[k] * 64, *lr = ur + 32;
                        const int cs = nk[k] & 7, es = qk[k] & 7;
                        f2 p = 0ull;
#pragma unroll
                        for (int sg = 0; sg < 8; ++sg) {
                            const float4 cv = *reinterpret_cast<const float4 *>(cr + ((sg ^ cs) << 2));
                            const float4 uv = *reinterpret_cast<const float4 *>(ur + ((sg ^ es) << 2));
                            const float4 lv = *reinterpret_cast<const float4 *>(lr + ((sg ^ es) << 2));
                            p = rest_step(pk(cv.x, cv.y), pk(uv.x, uv.y), pk(lv.x, lv.y), p);
                            p = rest_step(pk(cv.z, cv.w), pk(uv.z, uv.w), pk(lv.z, lv.w), p);
                        }
                        float p0, p1;
                        upk(p, p0, p1);
                        acc[k] = __fadd_rd(acc[k], __fadd_rd(p0, p1));
                        terms += (unsigned)min(kMvChunk, a.E - c * kMvChunk);
                    }
                    if ((c - c0) % kRestCheck == kRestCheck - 1) {
                        bool any = false;
#pragma unroll
                        for (int k = 0; k < kRestEpt; ++k) {
                            if (act[k] && acc[k] > th[k]) {  // abandoned: its partial sum
                                a.lb[(size_t)(q0 + qk[k]) * a.ldLb + n0 + nk[k]] = acc[k];
                                act[k] = false;
                            }
                            any |= act[k];
                        }
                        // (also the barrier before the other buffer is refilled)
                        if (!__syncthreads_or(any)) break;
                    } else {
                        __syncthreads();
                    }
                }
#pragma unroll
                for (int k = 0; k < kRestEpt; ++k)
                    if (act[k]) a.lb[(size_t)(q0 + qk[k]) * a.ldLb + n0 + nk[k]] = acc[k];
                cp_async_wait<0>();  // a stream left early may still have a chunk in flight
                __syncthreads();
            }
        }
    }
    if (a.terms) {
        for (int o = 16; o > 0; o >>= 1) terms += __shfl_xor_sync(0xffffffffu, terms, o);
        if (lane == 0 && terms) atomicAdd(a.terms, terms);
    }
}

int g_rest_attr_dev = -1;

}  // namespace

int lb_mv_rest_tile(int64_t N, int sms) {
    // tiles of at most kRestTC candidates, as few waves of one CTA per SM as that allows
    if (sms < 1) sms = 1;
    const int64_t waves = ((N + kRestTC - 1) / kRestTC + sms - 1) / sms;
    int64_t tn = (N + waves * sms - 1) / (waves * sms);
    tn = (tn + 31) / 32 * 32;
    if (tn > kRestTC) tn = kRestTC;
    if (tn < 32) tn = 32;
    return (int)tn;
}

int64_t lb_mv_rest_list_entries(int64_t N, int Mb, int sms) {
    const int tn = lb_mv_rest_tile(N, sms);
    const int qg = Mb < kRestQG ? Mb : kRestQG;
    const int64_t tiles = (N + tn - 1) / tn;
    const int64_t grid = tiles < sms ? tiles : sms;
    return grid * tn * qg;
}

cudaError_t launch_lb_mv_rest(const LbMvRestArgs &a, cudaStream_t s) {
    if (a.N <= 0 || a.Mb <= 0 || a.E0 >= a.E) return cudaSuccess;
    if (a.E0 % kMvChunk != 0 || a.ldP % kMvChunk != 0 || a.ldP < a.E ||
        (((uintptr_t)a.Up) & 15) != 0 || (((uintptr_t)a.Lp) & 15) != 0)
        return cudaErrorInvalidValue;
    const int sms = a.sms > 0 ? a.sms : 1;
    const int tn = lb_mv_rest_tile(a.N, sms);
    const int qg = a.Mb < kRestQG ? a.Mb : kRestQG;
    const int64_t tiles = (a.N + tn - 1) / tn;
    const int64_t grid = tiles < sms ? tiles : sms;
    if (a.list_entries < grid * tn * qg) return cudaErrorInvalidValue;
    const size_t smem = ((size_t)2 * tn * 32 + (size_t)2 * qg * 64 + qg + 4) * sizeof(float);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (g_rest_attr_dev != dev) {
        e = cudaFuncSetAttribute(k_lb_mv_rest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRestSmemMax);
        if (e != cudaSuccess) return e;
        g_rest_attr_dev = dev;
    }
    const int vec4 = (a.E % 4) == 0 && (a.ldC % 4) == 0 && (((uintptr_t)a.cand) & 15) == 0;
    k_lb_mv_rest<<<(unsigned)grid, kRestThreads, smem, s>>>(a, tn, qg, vec4);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tc
