// lb_rest.cu -- LB_MV with early abandoning (Section 7.1: abandoning applies to the
// lower-bound computations as well as to DTW).
//
// The dense stream (lb.cu) first sums a sample of the elements of every (query,
// candidate) pair: samp chunks of 32 spread evenly over the row.  A pair whose sample
// sum already exceeds its query's threshold is abandoned there: every LB_MV term is
// >= 0, so a sum over any subset of the terms is a lower bound of LB_MV, hence of DTW,
// and it already exceeds the threshold, which is all the search needs of it.  The pairs
// left at or under the threshold (on nearest-neighbour workloads usually a small share)
// are completed here, over the chunks the sample did not cover.
//
// CTA = tn candidates (tn <= kRestTC) x up to qg <= kRestQG queries.  The CTA lists the
// live (query, candidate) pairs of its tile (in a per-CTA global scratch region), then
// streams the remaining chunks of its candidates and of its queries' envelopes through
// shared memory in chunks of 32, two stages deep, every 128-byte row stored with its
// 16-byte segments XOR-swizzled by row & 7.  The consumers advance their listed pairs by
// one chunk per stage (bulk-tensor form: groups of 8 lanes per pair, see below; cp.async
// form: one thread per pair).  Every kRestCheck chunks a pair whose running sum has passed
// the threshold is abandoned again (its partial sum is written, a lower bound above
// the threshold); a check that finds no listed pair left ends the stream.
//
// Two forms of the stream.  k_lb_mv_rest_tma: one producer thread issues, per chunk,
// three 2-D bulk-tensor copies (candidate rows [tn][32], U and Lo rows [qg][32], the
// 128-byte swizzle above) that complete on the stage's "full" mbarrier, and the 480
// consumer threads only compute (a thread-issued copy costs address arithmetic per
// 16 bytes, which at ~92 KB per chunk is as much work as the sums).  Every wait is
// bounded (TCDTW_ERR_TIMEOUT in the status word, then the CTA winds down, waiting --
// bounded again -- for its copies in flight).  k_lb_mv_rest_cp, the fallback for rows
// whose stride is not a multiple of 16 bytes: every thread issues cp.async copies.
//
// Rounding as in the dense stream: terms and sums rounded down, so every stored value
// is at most the exact LB_MV.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "api_internal.h"
#include "common.cuh"
#include "lb_device.cuh"
#include "lb_kernels.cuh"
#include "lb_rest.cuh"
#include "tma.cuh"

namespace tc {

namespace {

// ------------------------------------------------------------------ bulk-tensor form
// Shared memory from a 1024-byte aligned base: two stages of [cand tn x 128 B | U qgp x
// 128 B | Lo qgp x 128 B] (qgp = qg rounded up to 8 rows, so every region starts on a
// 1024-byte boundary, as the 128-byte swizzle needs), then full[2], empty[2] mbarriers,
// four flags (stop, abort, issued, count) and the thresholds.
__host__ __device__ constexpr uint32_t rest_tma_stage_bytes(int tn, int qg) {
    return (uint32_t)(tn + 2 * ((qg + 7) / 8 * 8)) * 128u;
}
constexpr size_t rest_tma_smem(int tn, int qg) {
    return 1024 + 2 * (size_t)rest_tma_stage_bytes(tn, qg) + 32 + 16 + (size_t)qg * 4;
}
static_assert(rest_tma_smem(kRestTC, kRestQG) <= 227 * 1024, "one CTA of the completion stream per SM");

// Consumers of the bulk-tensor form in groups of 8 lanes: a group advances one listed
// pair at a time and lane s takes 16-byte segment s of the chunk (four elements) of its
// candidate row and of its query's U and Lo rows -- the 8 lanes read all 8 segments of
// each 128-byte row, so a phase of a shared-memory load touches all 32 banks once (one
// thread per pair read 8 different rows per phase, whose swizzled segments collided).
// Each lane keeps its own partial sum; the pair's sum is the 8 partials added, rounded
// down, in a fixed xor-shuffle order (the same on every lane), at every check and at the
// end.
constexpr int kRestGroupEpt = 14;          // listed pairs per 8-lane group per round
constexpr int kRestGroups = kRestCons / 8;
constexpr int kRestGroupRound = kRestGroups * kRestGroupEpt;

struct RestGroupPairs {
    int q[kRestGroupEpt], n[kRestGroupEpt];
    float acc[kRestGroupEpt], th[kRestGroupEpt];
    bool act[kRestGroupEpt];
};

__device__ __forceinline__ float group8_sum_rd(float v) {
    v = __fadd_rd(v, __shfl_xor_sync(0xffffffffu, v, 1));
    v = __fadd_rd(v, __shfl_xor_sync(0xffffffffu, v, 2));
    return __fadd_rd(v, __shfl_xor_sync(0xffffffffu, v, 4));
}

__global__ void __launch_bounds__(kRestTmaThreads, 1)
    k_lb_mv_rest_tma(const __grid_constant__ CUtensorMap cmap, const __grid_constant__ CUtensorMap umap,
                     const __grid_constant__ CUtensorMap lmap, const LbMvRestArgs a, int tn, int qg,
                     uint64_t wait_ns) {
    extern __shared__ unsigned char rest_raw[];
    const uint32_t raw = smem_u32(rest_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *sb = rest_raw + (base - raw);
    const int qgp = (qg + 7) / 8 * 8;
    const uint32_t stage = rest_tma_stage_bytes(tn, qg);
    const uint32_t full0 = base + 2 * stage, empty0 = full0 + 16;
    volatile int *flags = reinterpret_cast<volatile int *>(sb + 2 * stage + 32);  // stop, abort, issued, count
    float *thr = reinterpret_cast<float *>(sb + 2 * stage + 48);
    uint32_t *list = a.list + (size_t)blockIdx.x * tn * qg;
    const int tid = threadIdx.x, lane = tid & 31;
    const bool producer = tid >= kRestCons;
    const int nchunks = (a.E + kMvChunk - 1) / kMvChunk;
    const uint32_t tx = (uint32_t)(tn + 2 * qg) * 128u;  // bytes the three boxes deliver
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, kRestCons / 32);
        }
        flags[0] = flags[1] = flags[2] = flags[3] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (tid == kRestCons) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(&cmap) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&umap) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&lmap) : "memory");
    }
    __syncthreads();
    uint32_t kp = 0, kc = 0;  // stages issued (producer thread) / consumed (every consumer)
    unsigned long long terms = 0;
    const int64_t n_tiles = (a.N + tn - 1) / tn;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t n0 = tile * tn;
        for (int q0 = 0; q0 < a.Mb; q0 += qg) {
            const int nq = min(qg, a.Mb - q0);
            __syncthreads();  // the previous pass is done with the thresholds and the list
            if (tid == 0) flags[3] = 0;
            for (int k = tid; k < nq; k += blockDim.x) thr[k] = rest_threshold(a, q0 + k);
            __syncthreads();
            rest_list(a, n0, tn, q0, nq, thr, (int *)&flags[3], list);
            __syncthreads();  // the list (global, this CTA's region) and its count
            const int cnt = flags[3];
            for (int r0 = 0; r0 < cnt; r0 += kRestGroupRound) {
                int consumed = 0;
                if (producer) {
                    if (lane == 0) {
                        int issued = 0;
                        for (int c = rest_next(a, 0, nchunks); c < nchunks && !flags[0] && !flags[1] && !a.stall;
                             c = rest_next(a, c + 1, nchunks)) {
                            const uint32_t s = kp & 1u;
                            // the stage's previous chunk must have been released (the wait
                            // also gives up when the consumers stop the stream)
                            if (kp >= 2 && !mbar_wait(empty0 + 8 * s, ((kp >> 1) - 1) & 1u, flags, wait_ns)) {
                                if (!flags[0] && !flags[1]) {
                                    set_error(a.status, TCDTW_ERR_TIMEOUT, 50);
                                    flags[1] = 1;
                                }
                                break;
                            }
                            const uint32_t dst = base + s * stage, full = full0 + 8 * s;
                            mbar_expect_tx(full, tx);
                            tma_load_2d(dst, &cmap, c * kMvChunk, (int)n0, full);
                            tma_load_2d(dst + (uint32_t)tn * 128u, &umap, c * kMvChunk, q0, full);
                            tma_load_2d(dst + (uint32_t)(tn + qgp) * 128u, &lmap, c * kMvChunk, q0, full);
                            ++kp;
                            ++issued;
                        }
                        flags[2] = issued;
                    }
                } else {
                    const int grp = tid >> 3, seg = tid & 7;
                    RestGroupPairs p;
#pragma unroll
                    for (int k = 0; k < kRestGroupEpt; ++k) {
                        const int i = r0 + k * kRestGroups + grp;
                        p.act[k] = i < cnt;
                        const uint32_t en = p.act[k] ? __ldcg(list + i) : 0u;
                        p.q[k] = (int)(en >> 16);
                        p.n[k] = (int)(en & 0xffffu);
                        // the sample sum enters once, through lane 0 of the group
                        p.acc[k] = p.act[k] && seg == 0 ? a.lb[(size_t)(q0 + p.q[k]) * a.ldLb + n0 + p.n[k]] : 0.f;
                        p.th[k] = thr[p.q[k]];
                    }
                    int step = 0;
                    for (int c = rest_next(a, 0, nchunks); c < nchunks; c = rest_next(a, c + 1, nchunks), ++step) {
                        const uint32_t s = kc & 1u;
                        if (!mbar_wait(full0 + 8 * s, (kc >> 1) & 1u, flags + 1, wait_ns) && !flags[1]) {
                            set_error(a.status, TCDTW_ERR_TIMEOUT, 51);
                            flags[1] = 1;
                        }
                        ++kc;
                        ++consumed;
                        if (!flags[1]) {
                            const float *cb = reinterpret_cast<const float *>(sb + s * stage);
                            const float *ub = cb + tn * 32, *lbp = ub + qgp * 32;
                            const unsigned el = (unsigned)min(kMvChunk, a.E - c * kMvChunk);
#pragma unroll
                            for (int k = 0; k < kRestGroupEpt; ++k) {
                                if (!p.act[k]) continue;
                                const int cs = (seg ^ (p.n[k] & 7)) << 2, es = (seg ^ (p.q[k] & 7)) << 2;
                                const float4 cv = *reinterpret_cast<const float4 *>(cb + p.n[k] * 32 + cs);
                                const float4 uv = *reinterpret_cast<const float4 *>(ub + p.q[k] * 32 + es);
                                const float4 lv = *reinterpret_cast<const float4 *>(lbp + p.q[k] * 32 + es);
                                f2 pp = rest_step(pk(cv.x, cv.y), pk(uv.x, uv.y), pk(lv.x, lv.y), 0ull);
                                pp = rest_step(pk(cv.z, cv.w), pk(uv.z, uv.w), pk(lv.z, lv.w), pp);
                                float p0, p1;
                                upk(pp, p0, p1);
                                p.acc[k] = __fadd_rd(p.acc[k], __fadd_rd(p0, p1));
                                if (seg == 0) terms += el;
                            }
                        }
                        __syncwarp();
                        if (lane == 0) mbar_arrive(empty0 + 8 * s);
                        if (step % kRestCheck == kRestCheck - 1) {
                            bool any = false;
#pragma unroll
                            for (int k = 0; k < kRestGroupEpt; ++k) {
                                const float tot = group8_sum_rd(p.acc[k]);  // every lane takes part
                                if (p.act[k] && tot > p.th[k]) {  // abandoned: its partial sum
                                    if (seg == 0) a.lb[(size_t)(q0 + p.q[k]) * a.ldLb + n0 + p.n[k]] = tot;
                                    p.act[k] = false;
                                }
                                any |= p.act[k];
                            }
                            if (!consumers_any(any && !flags[1])) {
                                if (tid == 0) flags[0] = 1;  // stop the producer
                                break;
                            }
                        }
                    }
                    if (!flags[1]) {
#pragma unroll
                        for (int k = 0; k < kRestGroupEpt; ++k) {
                            const float tot = group8_sum_rd(p.acc[k]);
                            if (p.act[k] && seg == 0) a.lb[(size_t)(q0 + p.q[k]) * a.ldLb + n0 + p.n[k]] = tot;
                        }
                    }
                }
                __syncthreads();  // the producer is done issuing this round's chunks
                if (!producer) {
                    // chunks the producer issued past the consumers' stop: let them land
                    // and release their stages, so the stage parities stay in step
                    const int issued = flags[2];
                    for (; consumed < issued; ++consumed, ++kc) {
                        const uint32_t s = kc & 1u;
                        mbar_wait(full0 + 8 * s, (kc >> 1) & 1u, nullptr, wait_ns);
                        __syncwarp();
                        if (lane == 0) mbar_arrive(empty0 + 8 * s);
                    }
                    if (tid == 0) flags[0] = 0;
                }
                __syncthreads();
            }
        }
    }
    if (!producer) rest_terms_flush(a, terms);
    // no copy may still be landing when the CTA exits (after a timeout the consumers may
    // have stopped waiting for some): the producer waits, bounded, for the last phase of
    // each stage it issued
    if (tid == kRestCons)
        for (uint32_t j = kp >= 2 ? kp - 2 : 0; j < kp; ++j) mbar_wait(full0 + 8 * (j & 1u), (j >> 1) & 1u, nullptr, wait_ns);
}

// ------------------------------------------------------------------ cp.async form
__global__ void __launch_bounds__(kRestCpThreads, 1) k_lb_mv_rest_cp(const LbMvRestArgs a, int tn, int qg, int vec4) {
    extern __shared__ __align__(16) float rs[];
    uint32_t *list = a.list + (size_t)blockIdx.x * tn * qg;
    const int64_t n_tiles = (a.N + tn - 1) / tn;
    unsigned long long terms = 0;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x)
        for (int q0 = 0; q0 < a.Mb; q0 += qg)
            rest_pass_cp(a, tile * tn, tn, q0, min(qg, a.Mb - q0), qg, vec4, rs, list, terms);
    rest_terms_flush(a, terms);
}

int g_attr_dev_tma = -1, g_attr_dev_cp = -1;

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
    if (a.N <= 0 || a.Mb <= 0) return cudaSuccess;
    if (a.samp < 1 || a.sstride < 1 || (int64_t)(a.samp - 1) * a.sstride * kMvChunk + kMvChunk > a.E ||
        a.ldP % kMvChunk != 0 || a.ldP < a.E || (((uintptr_t)a.Up) & 15) != 0 ||
        (((uintptr_t)a.Lp) & 15) != 0)
        return cudaErrorInvalidValue;
    const int sms = a.sms > 0 ? a.sms : 1;
    const int tn = lb_mv_rest_tile(a.N, sms);
    const int qg = a.Mb < kRestQG ? a.Mb : kRestQG;
    const int64_t tiles = (a.N + tn - 1) / tn;
    const int64_t grid = tiles < sms ? tiles : sms;
    if (a.list_entries < grid * tn * qg) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    // bulk-tensor copies need 16-byte aligned rows (and a status word for the waits)
    CUtensorMap cm, um, lm;
    const bool tma = a.status && (a.ldC % 4) == 0 && (((uintptr_t)a.cand) & 15) == 0 && a.N < ((int64_t)1 << 31) &&
                     encode_2d(&cm, a.cand, (uint64_t)a.E, (uint64_t)a.N, (uint64_t)a.ldC * 4, kMvChunk, tn,
                               CU_TENSOR_MAP_SWIZZLE_128B) &&
                     encode_2d(&um, a.Up, (uint64_t)a.ldP, (uint64_t)a.Mb, (uint64_t)a.ldP * 4, kMvChunk, qg,
                               CU_TENSOR_MAP_SWIZZLE_128B) &&
                     encode_2d(&lm, a.Lp, (uint64_t)a.ldP, (uint64_t)a.Mb, (uint64_t)a.ldP * 4, kMvChunk, qg,
                               CU_TENSOR_MAP_SWIZZLE_128B);
    if (tma) {
        if (g_attr_dev_tma != dev) {
            e = cudaFuncSetAttribute(k_lb_mv_rest_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)rest_tma_smem(kRestTC, kRestQG));
            if (e != cudaSuccess) return e;
            g_attr_dev_tma = dev;
        }
        k_lb_mv_rest_tma<<<(unsigned)grid, kRestTmaThreads, rest_tma_smem(tn, qg), s>>>(
            cm, um, lm, a, tn, qg, a.wait_ns ? a.wait_ns : kWaitNs);
    } else {
        if (a.stall) return cudaErrorNotSupported;  // the self-test needs the bulk-tensor form
        if (g_attr_dev_cp != dev) {
            e = cudaFuncSetAttribute(k_lb_mv_rest_cp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)rest_cp_smem(kRestTC, kRestQG));
            if (e != cudaSuccess) return e;
            g_attr_dev_cp = dev;
        }
        const int vec4 = (a.E % 4) == 0 && (a.ldC % 4) == 0 && (((uintptr_t)a.cand) & 15) == 0;
        k_lb_mv_rest_cp<<<(unsigned)grid, kRestCpThreads, rest_cp_smem(tn, qg), s>>>(a, tn, qg, vec4);
    }
    note_launch();
    return cudaGetLastError();
}

}  // namespace tc

// Failure-detection self-test: one completion launch whose producer issues nothing, so
// its consumers' first wait on a chunk runs out after wait_us microseconds; the launch
// records TCDTW_ERR_TIMEOUT and ends by itself.
extern "C" int tcdtw_lb_mv_rest_selftest_timeout(int64_t wait_us, void *stream) {
    using namespace tc;
    if (wait_us < 1 || wait_us > 10000000) return TCDTW_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    // 32 candidates of 64 elements (chunk 0 sampled, chunk 1 to complete), 2 queries
    const int N = 32, E = 64, M = 2;
    const int64_t list_n = lb_mv_rest_list_entries(N, M, 1);
    const size_t floats = (size_t)N * E + 2 * (size_t)M * E + (size_t)M * N;
    float *buf = nullptr;
    uint32_t *list = nullptr;
    DevStatus *st = nullptr;
    if (dev_malloc((void **)&buf, floats * sizeof(float)) != cudaSuccess) return TCDTW_ERR_NOMEM;
    if (dev_malloc((void **)&list, (size_t)list_n * sizeof(uint32_t)) != cudaSuccess ||
        dev_malloc((void **)&st, sizeof(DevStatus)) != cudaSuccess) {
        cudaFree(buf);
        cudaFree(list);
        return TCDTW_ERR_NOMEM;
    }
    // zero candidates, envelopes and bounds: every pair's sample sum (0) is under the
    // +inf threshold, so every pair is listed and the consumers wait for chunk 1
    cudaError_t e = cudaMemsetAsync(buf, 0, floats * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    LbMvRestArgs a;
    a.cand = buf; a.N = N; a.E = E; a.samp = 1; a.sstride = 2; a.ldC = E;
    a.Up = buf + (size_t)N * E; a.Lp = a.Up + (size_t)M * E; a.ldP = E; a.Mb = M;
    a.lb = buf + (size_t)N * E + 2 * (size_t)M * E; a.ldLb = N; a.thresh = nullptr; a.bsf = nullptr; a.rho = 1.f;
    a.list = list; a.list_entries = list_n; a.sms = 1; a.status = st;
    a.wait_ns = (uint64_t)wait_us * 1000; a.stall = 1;
    // thresholds +inf (bsf is not read when thresholds are given)
    float *dthr = nullptr;
    if (e == cudaSuccess) e = dev_malloc((void **)&dthr, M * sizeof(float));
    if (e == cudaSuccess) {
        const float inf[M] = {INFINITY, INFINITY};
        e = cudaMemcpyAsync(dthr, inf, sizeof(inf), cudaMemcpyHostToDevice, s);
        a.thresh = dthr;
    }
    if (e == cudaSuccess) e = launch_lb_mv_rest(a, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    DevStatus h{0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(&h, st, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    cudaFree(list);
    cudaFree(st);
    cudaFree(dthr);
    if (e != cudaSuccess) return cuda_err(e);
    return h.code == TCDTW_ERR_TIMEOUT ? TCDTW_ERR_TIMEOUT : (h.code ? h.code : TCDTW_OK);
}
