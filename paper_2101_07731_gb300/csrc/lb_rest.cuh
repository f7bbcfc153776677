// lb_rest.cuh -- the completion pass of LB_MV with early abandoning (lb_rest.cu), as
// device routines shared by the single-set kernels and the batched search (batch.cu):
// list the live pairs of a candidate tile, then stream the rest of their elements.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "lb_device.cuh"
#include "lb_kernels.cuh"

namespace tc {
namespace {


constexpr int kRestEpt = 4;      // listed pairs per consumer thread per round
constexpr int kRestCheck = 16;   // chunks between abandoning checks
// bulk-tensor form: 15 consumer warps + the producer warp, four warps per SM
// sub-partition (a 17th warp would cap every thread at 96 registers)
constexpr int kRestCons = 480;
constexpr int kRestTmaThreads = kRestCons + 32;
constexpr int kRestCpThreads = 512;  // cp.async form: every thread consumes

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

// One chunk of one pair: candidate row cr, envelope rows ur / lr (32 floats each,
// segments swizzled by cs / es); returns the chunk's sum, rounded down.
__device__ __forceinline__ float rest_chunk(const float *cr, const float *ur, const float *lr, int cs, int es) {
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
    return __fadd_rd(p0, p1);
}

// The live pairs (bound at or under the query's threshold) of candidates [n0, n0+tn)
// x queries [q0, q0+nq), appended to list as (query - q0) << 16 | (candidate - n0);
// *cnt counts them.  Every thread of the CTA calls it (blockDim.x a multiple of 32:
// whole warps take part in every ballot, nq * tn being a multiple of 32).
__device__ __forceinline__ void rest_list(const LbMvRestArgs &a, int64_t n0, int tn, int q0, int nq,
                                          const float *thr, int *cnt, uint32_t *list) {
    const int lane = threadIdx.x & 31;
    for (int base = 0; base < nq * tn; base += blockDim.x) {
        const int idx = base + threadIdx.x;
        const int ql = idx / tn, nl = idx - ql * tn;
        bool live = false;
        if (ql < nq && n0 + nl < a.N) {
            const float v = a.lb[(size_t)(q0 + ql) * a.ldLb + n0 + nl];
            live = v < TC_INF && v <= thr[ql];
        }
        const unsigned bal = __ballot_sync(0xffffffffu, live);
        int pos = 0;
        if (lane == 0 && bal) pos = atomicAdd(cnt, __popc(bal));
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (live) list[pos + __popc(bal & ((1u << lane) - 1u))] = ((uint32_t)ql << 16) | (uint32_t)nl;
    }
}

// The first row chunk at or after c that the sample did not cover (nchunks: none).
__device__ __forceinline__ int rest_next(const LbMvRestArgs &a, int c, int nchunks) {
    while (c < nchunks && lb_mv_sampled(c, a.samp, a.sstride)) ++c;
    return c;
}

__device__ __forceinline__ float rest_threshold(const LbMvRestArgs &a, int q) {
    return a.thresh ? a.thresh[q] : prune_threshold(ld_volatile_u64(a.bsf + q), a.rho);
}

// The round's listed pairs of consumer thread t of nc: entries r0 + k * nc + t.
struct RestPairs {
    int q[kRestEpt], n[kRestEpt];
    float acc[kRestEpt], th[kRestEpt];
    bool act[kRestEpt];
};

__device__ __forceinline__ void rest_load(RestPairs &p, const LbMvRestArgs &a, const uint32_t *list, int r0, int t,
                                          int nc, int cnt, int64_t n0, int q0, const float *thr) {
#pragma unroll
    for (int k = 0; k < kRestEpt; ++k) {
        const int i = r0 + k * nc + t;
        p.act[k] = i < cnt;
        const uint32_t en = p.act[k] ? __ldcg(list + i) : 0u;
        p.q[k] = (int)(en >> 16);
        p.n[k] = (int)(en & 0xffffu);
        p.acc[k] = p.act[k] ? a.lb[(size_t)(q0 + p.q[k]) * a.ldLb + n0 + p.n[k]] : 0.f;
        p.th[k] = thr[p.q[k]];
    }
}

// Abandons the pairs whose running sum passed their threshold (writing the partial
// sum); true while any pair of this thread is still active.
__device__ __forceinline__ bool rest_check(RestPairs &p, const LbMvRestArgs &a, int64_t n0, int q0) {
    bool any = false;
#pragma unroll
    for (int k = 0; k < kRestEpt; ++k) {
        if (p.act[k] && p.acc[k] > p.th[k]) {
            a.lb[(size_t)(q0 + p.q[k]) * a.ldLb + n0 + p.n[k]] = p.acc[k];
            p.act[k] = false;
        }
        any |= p.act[k];
    }
    return any;
}

__device__ __forceinline__ void rest_store(const RestPairs &p, const LbMvRestArgs &a, int64_t n0, int q0) {
#pragma unroll
    for (int k = 0; k < kRestEpt; ++k)
        if (p.act[k]) a.lb[(size_t)(q0 + p.q[k]) * a.ldLb + n0 + p.n[k]] = p.acc[k];
}

// OR of v over the consumer threads (named barrier 1; the producer warp never joins).
__device__ __forceinline__ bool consumers_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(kRestCons)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void rest_terms_flush(const LbMvRestArgs &a, unsigned long long terms) {
    if (!a.terms) return;
    for (int o = 16; o > 0; o >>= 1) terms += __shfl_xor_sync(0xffffffffu, terms, o);
    if ((threadIdx.x & 31) == 0 && terms) atomicAdd(a.terms, terms);
}


// Copies chunk [e0, e0+32) of the tile's candidates and queries into one buffer:
// candidate rows [tn][32], query rows [qg][64] (U then Lo), segments swizzled by row.
__device__ __forceinline__ void rest_issue(const LbMvRestArgs &a, int64_t n0, int tn, int q0, int nq, int e0,
                                           bool vec4, float *sc, float *se) {
    const int tid = threadIdx.x;
    if (vec4) {
        for (int idx = tid; idx < tn * 8; idx += kRestCpThreads) {
            const int row = idx >> 3, seg = idx & 7;
            const int64_t n = n0 + row;
            const int e = e0 + seg * 4;
            const bool ok = n < a.N && e < a.E;
            const float *src = ok ? a.cand + (size_t)n * a.ldC + e : a.cand;
            cp_async16(sc + row * 32 + ((seg ^ (row & 7)) << 2), src, ok ? 16 : 0);
        }
    } else {
        for (int idx = tid; idx < tn * 32; idx += kRestCpThreads) {
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
    for (int idx = tid; idx < nq * 16; idx += kRestCpThreads) {
        const int row = idx >> 4, h = (idx >> 3) & 1, seg = idx & 7;
        const float *src = (h ? a.Lp : a.Up) + (size_t)(q0 + row) * a.ldP + e0 + seg * 4;
        cp_async16(se + row * 64 + h * 32 + ((seg ^ (row & 7)) << 2), src, 16);
    }
}

constexpr size_t rest_cp_smem(int tn, int qg) {
    return ((size_t)2 * tn * 32 + (size_t)2 * qg * 64 + qg + 4) * sizeof(float);
}
static_assert(rest_cp_smem(kRestTC, kRestQG) <= 227 * 1024, "one CTA of the completion stream per SM");

// One pass of the cp.async form over candidates [n0, n0+tn) x queries [q0, q0+nq) (nq
// <= qg): list the live pairs, then complete them in rounds of kRestCpThreads *
// kRestEpt.  rs: shared memory of rest_cp_smem(tn, qg) bytes; list: this CTA's scratch
// (tn * qg entries).  Every thread of a kRestCpThreads-thread CTA calls it.
__device__ __forceinline__ void rest_pass_cp(const LbMvRestArgs &a, int64_t n0, int tn, int q0, int nq, int qg,
                                             int vec4, float *rs, uint32_t *list, unsigned long long &terms) {
    float *const env0 = rs + 2 * tn * 32;
    float *thr = env0 + 2 * qg * 64;
    int *s_cnt = reinterpret_cast<int *>(thr + qg);
    const int tid = threadIdx.x;
    const int nchunks = (a.E + kMvChunk - 1) / kMvChunk;
    __syncthreads();  // the previous pass is done with the thresholds and the list
    if (tid == 0) *s_cnt = 0;
    for (int k = tid; k < nq; k += blockDim.x) thr[k] = rest_threshold(a, q0 + k);
    __syncthreads();
    rest_list(a, n0, tn, q0, nq, thr, s_cnt, list);
    __syncthreads();  // the list (global, this CTA's region) and its count
    const int cnt = *s_cnt;
    for (int r0 = 0; r0 < cnt; r0 += kRestCpThreads * kRestEpt) {
        RestPairs p;
        rest_load(p, a, list, r0, tid, kRestCpThreads, cnt, n0, q0, thr);
        int c = rest_next(a, 0, nchunks);
        if (c < nchunks) rest_issue(a, n0, tn, q0, nq, c * kMvChunk, vec4, rs, env0);
        cp_async_commit();
        for (int step = 0; c < nchunks; ++step) {
            const int buf = step & 1;
            const int cn = rest_next(a, c + 1, nchunks);
            if (cn < nchunks) {
                rest_issue(a, n0, tn, q0, nq, cn * kMvChunk, vec4, rs + (buf ^ 1) * tn * 32,
                           env0 + (buf ^ 1) * qg * 64);
                cp_async_commit();
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const float *cb = rs + buf * tn * 32, *eb = env0 + buf * qg * 64;
#pragma unroll
            for (int k = 0; k < kRestEpt; ++k) {
                if (!p.act[k]) continue;
                const float *ur = eb + p.q[k] * 64;
                p.acc[k] = __fadd_rd(p.acc[k], rest_chunk(cb + p.n[k] * 32, ur, ur + 32, p.n[k] & 7, p.q[k] & 7));
                terms += (unsigned)min(kMvChunk, a.E - c * kMvChunk);
            }
            if (step % kRestCheck == kRestCheck - 1) {
                // (also the barrier before the other buffer is refilled)
                if (!__syncthreads_or(rest_check(p, a, n0, q0))) break;
            } else {
                __syncthreads();
            }
            c = cn;
        }
        rest_store(p, a, n0, q0);
        cp_async_wait<0>();  // a stream left early may still have a chunk in flight
        __syncthreads();
    }
}

}  // namespace
}  // namespace tc
