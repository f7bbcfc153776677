// lb_tma.cu -- the LB_MV stream (Section 3) fed by the Tensor Memory Accelerator.
//
// Same bound, same tiles and the same per-element arithmetic as the cp.async stream
// in lb.cu (CTA tile 128 candidates x QB queries, 32-element chunks, directed
// rounding), with a deeper pipeline for the case where few queries share a pass and
// the stream is bound by HBM rather than by FP32 issue:
//
//  * one producer warp issues, per chunk, three 2-D bulk-tensor copies into a stage
//    of an NS-deep ring: the candidate chunk [128 rows][32 floats] (128-byte swizzle,
//    the same XOR layout the consumers read), and the U and Lo envelope chunks of the
//    tile's queries ([QB/2 query pairs][64 floats], query-pair interleaved); the
//    copies complete on the stage's "full" mbarrier with a transaction count;
//  * NG consumer groups of 128 threads (one candidate row per thread) take the
//    chunks of the CTA's chunk sequence round robin (chunk k -> group k % NG);
//    NS is a multiple of NG, so each stage has exactly one consuming group and the
//    phase parity of its barriers is unambiguous; a group's four warps release the
//    stage on its "empty" mbarrier;
//  * the work (tiles x chunks) is split over the grid stream-K fashion: every CTA
//    takes an equal contiguous run of chunks (with 157 tiles of 128 candidates on
//    152 SMs, whole tiles per CTA would leave most SMs idle for the last tile), so a
//    tile may be shared by a few CTAs;
//  * at the end of a tile (or of a CTA's part of one) the groups' sums are added in
//    group order; the parts of a shared tile go to a workspace and the last CTA to
//    finish it adds them in chunk order; everything rounds down (a sum of values
//    each rounded down stays below the exact bound) and the order is fixed, so the
//    result does not depend on timing.
//
// Rows past N and elements past E are filled with zeros by the copy engine; the
// envelope holds +inf / -inf past E, so those elements add exactly 0.
//
// Every wait is bounded (about two seconds of global time); a wait that gives up
// records TCDTW_ERR_TIMEOUT in the status word, the other waits of the CTA stop
// waiting, every thread still reaches every CTA barrier, and the producer waits
// (again bounded) for the copies it has in flight before the CTA exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "api_internal.h"
#include "common.cuh"
#include "lb_device.cuh"
#include "lb_kernels.cuh"
#include "tma.cuh"

namespace tc {
namespace {

constexpr int kCandBytes = kMvRows * kMvChunk * 4;  // 16 KB per stage

__device__ __forceinline__ void consumer_sync(int nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

template <int QB, int NG, int NS>
struct MvTmaLayout {
    static_assert(NS % NG == 0, "each stage must have a single consuming group");
    static constexpr int kEnvBytes = QB * kMvChunk * 4;   // QB/2 pairs x 64 floats
    static constexpr int kCandOff = 0;                     // NS x 16 KB, 1024-aligned
    static constexpr int kEnvOff = NS * kCandBytes;        // NS x (U, Lo)
    static constexpr int kBarOff = kEnvOff + NS * 2 * kEnvBytes;
    static constexpr int kFlagOff = kBarOff + 2 * NS * 8;
    static constexpr int kXsOff = (kFlagOff + 16 + 15) / 16 * 16;
    static constexpr int kXsBytes = (NG - 1) * (QB / 2) * kMvRows * 8;
    static constexpr int kBytes = kXsOff + kXsBytes + 1024;  // + alignment slack
    static constexpr int kStageTx = kCandBytes + 2 * kEnvBytes;
    static constexpr bool kFits = kBytes <= 227 * 1024;  // shared memory of one CTA
};

// Stream-K partition of the flat work w = tile * nchunks + chunk over the grid: CTA b
// takes [w0(b), w0(b+1)), w0(b) = floor(b * total / grid), so the CTAs' shares differ
// by at most one chunk.  (With tile_aligned the shares are whole tiles instead.)
__device__ __forceinline__ int64_t sk_begin(int64_t b, int64_t total, int64_t grid) { return b * total / grid; }
// the CTA whose share holds work item x
__device__ __forceinline__ int64_t sk_owner(int64_t x, int64_t total, int64_t grid) {
    int64_t b = x * grid / total;
    while (b + 1 < grid && sk_begin(b + 1, total, grid) <= x) ++b;
    while (b > 0 && sk_begin(b, total, grid) > x) --b;
    return b;
}

template <int QB, int NG, int NS>
__global__ void __launch_bounds__(128 * NG + 32)
    k_lb_mv_tma(const __grid_constant__ CUtensorMap cmap, const __grid_constant__ CUtensorMap umap,
                const __grid_constant__ CUtensorMap lmap, int64_t N, int E, int cstride, int Mb, float *__restrict__ lb,
                int64_t ldLb, int n_ctiles, int n_qtiles, int tile_aligned, float *__restrict__ ws,
                int *__restrict__ tile_cnt, DevStatus *status, uint64_t wait_ns, int stall) {
    using Lay = MvTmaLayout<QB, NG, NS>;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *sbase = smem_raw + (base - raw);
    const uint32_t full0 = base + Lay::kBarOff, empty0 = full0 + NS * 8;
    volatile int *abort = reinterpret_cast<volatile int *>(sbase + Lay::kFlagOff);
    volatile int *last_flag = abort + 1;
    f2 *xs = reinterpret_cast<f2 *>(sbase + Lay::kXsOff);

    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 4);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    const int nchunks = (E + kMvChunk - 1) / kMvChunk;
    const int64_t ntiles = (int64_t)n_ctiles * n_qtiles;
    const int64_t total = ntiles * nchunks, grid = gridDim.x, b = blockIdx.x;
    const int64_t w0 = tile_aligned ? sk_begin(b, ntiles, grid) * nchunks : sk_begin(b, total, grid);
    const int64_t w1 = tile_aligned ? sk_begin(b + 1, ntiles, grid) * nchunks : sk_begin(b + 1, total, grid);

    if (tid >= 128 * NG) {  // ------------------------------------------ producer warp
        if (tid != 128 * NG) return;
        asm volatile("prefetch.tensormap [%0];" ::"l"(&cmap) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&umap) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&lmap) : "memory");
        int k = 0;
        for (int64_t w = w0; w < (stall ? w0 : w1); ++w, ++k) {  // stall: the self-test issues nothing
            const int s = k % NS;
            if (k >= NS && !mbar_wait(empty0 + 8 * s, ((k / NS) - 1) & 1, abort, wait_ns)) {
                if (!*abort) set_error(status, TCDTW_ERR_TIMEOUT, 40);
                *abort = 1;
            }
            if (*abort) break;
            const int64_t tile = w / nchunks;
            const int c = (int)(w - tile * nchunks);
            const int ct = (int)(tile / n_qtiles), qt = (int)(tile - (int64_t)ct * n_qtiles);
            const uint32_t full = full0 + 8 * s;
            mbar_expect_tx(full, Lay::kStageTx);
            // stream chunk c is row chunk c * cstride
            tma_load_2d(base + Lay::kCandOff + s * kCandBytes, &cmap, c * cstride * kMvChunk, ct * kMvRows, full);
            const uint32_t env = base + Lay::kEnvOff + s * 2 * Lay::kEnvBytes;
            tma_load_2d(env, &umap, c * cstride * 2 * kMvChunk, qt * (QB / 2), full);
            tma_load_2d(env + Lay::kEnvBytes, &lmap, c * cstride * 2 * kMvChunk, qt * (QB / 2), full);
        }
        // the last copies must have landed before the CTA may exit (bounded)
        for (int j = k - NS > 0 ? k - NS : 0; j < k; ++j) mbar_wait(full0 + 8 * (j % NS), (j / NS) & 1, nullptr, wait_ns);
        return;
    }

    // ------------------------------------------------------------------ consumers
    const int g = tid >> 7, t = tid & 127, lane = tid & 31;
    bool gave_up = false;
    int k = 0;
    for (int64_t w = w0; w < w1;) {
        const int64_t tile = w / nchunks;
        const int64_t tb = tile * nchunks, te = tb + nchunks;
        const int64_t seg_end = w1 < te ? w1 : te;
        const bool whole = (w == tb && seg_end == te);
        const int ct = (int)(tile / n_qtiles), qt = (int)(tile - (int64_t)ct * n_qtiles);
        f2 acc[QB / 2];
#pragma unroll
        for (int j = 0; j < QB / 2; ++j) acc[j] = 0ull;
        for (; w < seg_end; ++w, ++k) {
            if (k % NG != g) continue;
            const int s = k % NS;
            if (!gave_up && !mbar_wait(full0 + 8 * s, (k / NS) & 1, abort, wait_ns)) {
                if (!*abort) set_error(status, TCDTW_ERR_TIMEOUT, 41);
                *abort = 1;
                gave_up = true;
            }
            if (*abort) gave_up = true;
            const float *sc = reinterpret_cast<const float *>(sbase + Lay::kCandOff + s * kCandBytes);
            const float *su = reinterpret_cast<const float *>(sbase + Lay::kEnvOff + s * 2 * Lay::kEnvBytes);
            const float *sl = su + QB * kMvChunk;
            // the chunk in two halves of 16 elements (fewer live registers); each
            // query pair's chunk sum still runs over the elements in order
            f2 part[QB / 2];
#pragma unroll
            for (int qp = 0; qp < QB / 2; ++qp) part[qp] = 0ull;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                f2 c2[kMvChunk / 2];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int seg = 4 * h + j;
                    const float4 v = *reinterpret_cast<const float4 *>(&sc[t * kMvChunk + ((seg ^ (t & 7)) << 2)]);
                    c2[4 * j] = pk(v.x, v.x);
                    c2[4 * j + 1] = pk(v.y, v.y);
                    c2[4 * j + 2] = pk(v.z, v.z);
                    c2[4 * j + 3] = pk(v.w, v.w);
                }
#pragma unroll
                for (int qp = 0; qp < QB / 2; ++qp) {
                    const float *uu = su + qp * 2 * kMvChunk + h * kMvChunk;
                    const float *ll = sl + qp * 2 * kMvChunk + h * kMvChunk;
#pragma unroll
                    for (int e = 0; e < kMvChunk / 2; e += 2) {
                        const float4 u4 = *reinterpret_cast<const float4 *>(uu + 2 * e);
                        const float4 l4 = *reinterpret_cast<const float4 *>(ll + 2 * e);
                        part[qp] = mv_step(c2[e], u4.x, u4.y, l4.x, l4.y, part[qp]);
                        part[qp] = mv_step(c2[e + 1], u4.z, u4.w, l4.z, l4.w, part[qp]);
                    }
                }
            }
#pragma unroll
            for (int qp = 0; qp < QB / 2; ++qp) acc[qp] = add2_rd(acc[qp], part[qp]);
            __syncwarp();
            if (lane == 0) mbar_arrive(empty0 + 8 * s);
        }
        // the segment's sum: consumer groups in order
        if (NG > 1) {
            if (g > 0) {
#pragma unroll
                for (int qp = 0; qp < QB / 2; ++qp) xs[((g - 1) * (QB / 2) + qp) * kMvRows + t] = acc[qp];
            }
            consumer_sync(128 * NG);
            if (g == 0) {
                for (int h = 1; h < NG; ++h) {
#pragma unroll
                    for (int qp = 0; qp < QB / 2; ++qp)
                        acc[qp] = add2_rd(acc[qp], xs[((h - 1) * (QB / 2) + qp) * kMvRows + t]);
                }
            }
        }
        const int64_t n = (int64_t)ct * kMvRows + t;
        const int q0 = qt * QB;
        if (whole) {
            if (g == 0 && n < N && !gave_up && !*abort) {
#pragma unroll
                for (int qp = 0; qp < QB / 2; ++qp) {
                    float a0, a1;
                    upk(acc[qp], a0, a1);
                    if (q0 + 2 * qp < Mb) lb[(size_t)(q0 + 2 * qp) * ldLb + n] = a0;
                    if (q0 + 2 * qp + 1 < Mb) lb[(size_t)(q0 + 2 * qp + 1) * ldLb + n] = a1;
                }
            }
        } else {
            // A tile shared by several CTAs: each writes its partial to its slot
            // ws[b][0 = first segment of its share, 1 = last][QB][128]; the last of
            // the tile's contributors to arrive (counted on tile_cnt, which it resets)
            // adds the partials in the order of the shares, i.e. of the chunks.
            const int which = tile == w0 / nchunks ? 0 : 1;
            if (g == 0) {
#pragma unroll
                for (int qp = 0; qp < QB / 2; ++qp) {
                    float a0, a1;
                    upk(acc[qp], a0, a1);
                    ws[((b * 2 + which) * QB + 2 * qp) * kMvRows + t] = a0;
                    ws[((b * 2 + which) * QB + 2 * qp + 1) * kMvRows + t] = a1;
                }
                __threadfence();
            }
            const int64_t bf = sk_owner(tb, total, grid), bl = sk_owner(te - 1, total, grid);
            consumer_sync(128 * NG);
            if (tid == 0) *last_flag = atomicAdd(&tile_cnt[tile], 1) == (int)(bl - bf);
            consumer_sync(128 * NG);
            if (*last_flag) {
                if (tid == 0) tile_cnt[tile] = 0;
                if (n < N && !gave_up && !*abort) {
                    for (int j = g; j < QB; j += NG) {  // consumer groups share the queries
                        const int q = q0 + j;
                        if (q >= Mb) break;
                        float a = 0.f;
                        for (int64_t c0 = bf; c0 <= bl; c0 += 8) {  // eight loads in flight, then add in order
                            float v[8];
#pragma unroll
                            for (int r = 0; r < 8; ++r) {
                                const int64_t cb = c0 + r;
                                const int wh = cb <= bl && tile == sk_begin(cb, total, grid) / nchunks ? 0 : 1;
                                v[r] = cb <= bl ? __ldcg(&ws[((cb * 2 + wh) * QB + j) * kMvRows + t]) : 0.f;
                            }
#pragma unroll
                            for (int r = 0; r < 8; ++r)
                                if (c0 + r <= bl) a = c0 + r == bf ? v[r] : __fadd_rd(a, v[r]);
                        }
                        lb[(size_t)q * ldLb + n] = a;
                    }
                }
            }
            consumer_sync(128 * NG);  // the flag is rewritten by the next shared tile
        }
        if (NG > 1 && whole) consumer_sync(128 * NG);  // xs is rewritten by the next segment
    }
}

struct MvPlan {
    int n_ctiles, n_qtiles;
};

template <int QB, int NG, int NS>
int variant_occupancy() {
    using Lay = MvTmaLayout<QB, NG, NS>;
    constexpr int kMaxDev = 64;
    static int occ_of[kMaxDev];  // per device; 0 = not yet queried (idempotent race)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return -1;
    if (occ_of[dev] == 0) {
        auto kern = k_lb_mv_tma<QB, NG, NS>;
        int occ = 0;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::kBytes) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 128 * NG + 32, Lay::kBytes) != cudaSuccess ||
            occ < 1) {
            (void)cudaGetLastError();  // the caller falls back; leave no error behind
            return -1;
        }
        occ_of[dev] = occ;
    }
    return occ_of[dev];
}

template <int QB, int NG, int NS>
cudaError_t launch_variant(const LbMvArgs &a, const CUtensorMap &cm, const CUtensorMap &um, const CUtensorMap &lm,
                           MvPlan p, cudaStream_t s, uint64_t wait_ns = kWaitNs, int stall = 0, int ctas_per_sm = 0) {
    using Lay = MvTmaLayout<QB, NG, NS>;
    if constexpr (!Lay::kFits) {
        return cudaErrorNotSupported;
    } else {
        int occ = variant_occupancy<QB, NG, NS>();
        if (occ < 1) return cudaErrorNotSupported;
        if (ctas_per_sm > 0 && ctas_per_sm < occ) occ = ctas_per_sm;
        const int nchunks = (a.E + kMvChunk - 1) / kMvChunk;
        const int64_t tiles = (int64_t)p.n_ctiles * p.n_qtiles;
        const int64_t total = tiles * nchunks;
        int64_t grid = (int64_t)occ * a.sms;
        if (grid > total) grid = total;
        // chunk-granular shares need a slot pair per CTA and a counter per tile
        const bool fine = a.ws && a.tile_cnt && tiles <= a.tile_cnt_cap && grid * 2 * QB * kMvRows <= a.ws_floats;
        if (!fine && grid > tiles) grid = tiles;
        k_lb_mv_tma<QB, NG, NS><<<(int)grid, 128 * NG + 32, Lay::kBytes, s>>>(
            cm, um, lm, a.N, a.E, a.cstride > 0 ? a.cstride : 1, a.Mb, a.lb, a.ldLb, p.n_ctiles, p.n_qtiles,
            fine ? 0 : 1, a.ws, a.tile_cnt,
            a.status, wait_ns, stall);
        note_launch();
        return cudaGetLastError();
    }
}

}  // namespace

EncodeFn encode_fn() {
    static const EncodeFn fn = []() -> EncodeFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeFn>(p);
    }();
    return fn;
}

// 2-D FP32 tensor map: rows of `width` floats `pitch` bytes apart, box [box_h][box_w]
bool encode_2d(CUtensorMap *m, const float *ptr, uint64_t width, uint64_t height, uint64_t pitch, uint32_t box_w,
               uint32_t box_h, CUtensorMapSwizzle swz) {
    EncodeFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dim[2] = {width, height};
    const cuuint64_t stride[1] = {pitch};
    const cuuint32_t box[2] = {box_w, box_h};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dim, stride, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool lb_mv_tma_ok(const LbMvArgs &a) {
    const int64_t ldC = a.ldC > 0 ? a.ldC : a.E;
    const int Erow = a.Erow > 0 ? a.Erow : a.E;
    return a.status != nullptr && (Erow % 4) == 0 && (ldC % 4) == 0 && ldC >= Erow && (((uintptr_t)a.cand) & 15) == 0 &&
           (((uintptr_t)a.U) & 15) == 0 && (((uintptr_t)a.Lo) & 15) == 0 && (a.ldE % kMvChunk) == 0 &&
           a.N < ((int64_t)1 << 31) - 256 && a.Mb < (1 << 30) && encode_fn() != nullptr;
}

cudaError_t launch_lb_mv_tma(const LbMvArgs &a, cudaStream_t s) {
    if (a.N <= 0 || a.Mb <= 0) return cudaSuccess;
    if (!lb_mv_tma_ok(a)) return cudaErrorNotSupported;
    int QB = 32;
    if (a.Mb <= 2) QB = 2;
    else if (a.Mb <= 4) QB = 4;
    else if (a.Mb <= 8) QB = 8;
    else if (a.Mb <= 16) QB = 16;
    // 32 queries per tile are bound by FP32 issue, not by HBM: the cp.async stream
    // (more resident warps) is faster there
    if (QB == 32) return cudaErrorNotSupported;
    MvPlan p;
    p.n_ctiles = (int)((a.N + kMvRows - 1) / kMvRows);
    p.n_qtiles = (a.Mb + QB - 1) / QB;
    const int64_t n_qp = (a.Mb + 1) / 2;
    CUtensorMap cm, um, lm;
    const int64_t ldC = a.ldC > 0 ? a.ldC : a.E;
    const int Erow = a.Erow > 0 ? a.Erow : a.E;
    if (!encode_2d(&cm, a.cand, (uint64_t)Erow, (uint64_t)a.N, (uint64_t)ldC * 4, kMvChunk, kMvRows,
                   CU_TENSOR_MAP_SWIZZLE_128B) ||
        !encode_2d(&um, a.U, (uint64_t)a.ldE * 2, (uint64_t)n_qp, (uint64_t)a.ldE * 8, 2 * kMvChunk, QB / 2,
                   CU_TENSOR_MAP_SWIZZLE_NONE) ||
        !encode_2d(&lm, a.Lo, (uint64_t)a.ldE * 2, (uint64_t)n_qp, (uint64_t)a.ldE * 8, 2 * kMvChunk, QB / 2,
                   CU_TENSOR_MAP_SWIZZLE_NONE))
        return cudaErrorNotSupported;
    // consumer groups x stages and CTAs per SM measured on the 20000 x 256 x 5 stream
    // (ncu device time, 1 / 2 / 4 / 8 / 16 queries: 23 / 24 / 29 / 45 / 72 us)
    switch (QB) {
        case 2: return launch_variant<2, 2, 4>(a, cm, um, lm, p, s, kWaitNs, 0, 2);
        case 4: return launch_variant<4, 2, 4>(a, cm, um, lm, p, s, kWaitNs, 0, 2);
        case 8: return launch_variant<8, 4, 8>(a, cm, um, lm, p, s);
        default: return launch_variant<16, 4, 4>(a, cm, um, lm, p, s);
    }
}

}  // namespace tc

// Failure-detection self-test: one CTA of the TMA stream whose producer issues
// nothing, so its consumers' first wait runs out after wait_us microseconds.
extern "C" int tcdtw_lb_mv_selftest_timeout(int64_t wait_us, void *stream) {
    using namespace tc;
    if (wait_us < 1 || wait_us > 10000000) return TCDTW_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    float *buf = nullptr;
    DevStatus *st = nullptr;
    const int64_t E = kMvChunk, ldE = kMvChunk;
    const size_t floats = kMvRows * E + 2 * 2 * ldE + kMvRows;  // candidates, U, Lo (two pairs), lb
    if (dev_malloc((void **)&buf, floats * sizeof(float)) != cudaSuccess) return TCDTW_ERR_NOMEM;
    if (dev_malloc((void **)&st, sizeof(DevStatus)) != cudaSuccess) { cudaFree(buf); return TCDTW_ERR_NOMEM; }
    cudaError_t e = cudaMemsetAsync(buf, 0, floats * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    LbMvArgs a;
    a.cand = buf; a.N = kMvRows; a.E = (int)E; a.U = buf + kMvRows * E; a.Lo = a.U + 2 * ldE; a.ldE = ldE;
    a.Mb = 2; a.lb = buf + kMvRows * E + 4 * ldE; a.ldLb = kMvRows; a.sms = 1; a.status = st;
    CUtensorMap cm, um, lm;
    if (e == cudaSuccess &&
        (!encode_2d(&cm, a.cand, (uint64_t)E, kMvRows, (uint64_t)E * 4, kMvChunk, kMvRows, CU_TENSOR_MAP_SWIZZLE_128B) ||
         !encode_2d(&um, a.U, (uint64_t)ldE * 2, 1, (uint64_t)ldE * 8, 2 * kMvChunk, 1, CU_TENSOR_MAP_SWIZZLE_NONE) ||
         !encode_2d(&lm, a.Lo, (uint64_t)ldE * 2, 1, (uint64_t)ldE * 8, 2 * kMvChunk, 1, CU_TENSOR_MAP_SWIZZLE_NONE)))
        e = cudaErrorNotSupported;
    MvPlan p{1, 1};
    if (e == cudaSuccess) e = launch_variant<2, 4, 8>(a, cm, um, lm, p, s, (uint64_t)wait_us * 1000, 1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    DevStatus h{0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(&h, st, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    cudaFree(st);
    if (e != cudaSuccess) return cuda_err(e);
    return h.code == TCDTW_ERR_TIMEOUT ? TCDTW_ERR_TIMEOUT : (h.code ? h.code : TCDTW_OK);
}
