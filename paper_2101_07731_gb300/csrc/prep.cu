// prep.cu -- query-side preparation on sm_103a, done when a query block arrives
// (Section 7.1 counts this work in the search time):
//   * non-finite scan of input series;
//   * envelopes U / Lo over the Sakoe-Chiba window (Section 3, "Algorithm LB_MV");
//   * neighbour distances d(q_{i-1}, q_i) as a rounded-down / rounded-up interval
//     (Section 4.1, used by LB_TI);
//   * LB_PC quantisation boxes per expanded window (Section 5).
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "lb_kernels.cuh"

namespace tc {

// ------------------------------------------------------------------ non-finite scan
__global__ void k_check_finite(const float *__restrict__ x, int64_t n, DevStatus *st, int where) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (; i < n; i += stride) bad |= !isfinite(__ldg(x + i));
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_error(st, TCDTW_ERR_NONFINITE, where);
}

cudaError_t launch_check_finite(const float *x, int64_t n, DevStatus *st, int where, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_check_finite<<<(int)blocks, 256, 0, s>>>(x, n, st, where); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ envelope
// Block (tile t, query m) produces rows [t*TP, t*TP+TP) of U and Lo.  The query
// points those rows need, [t*TP - W, t*TP + TP - 1 + W] clipped, are staged in
// shared memory with coalesced loads when they fit; each output element is then the
// max / min over its clipped window.  Output rows are written with stride ldE per
// query (ldE >= L*D); with pad != 0 the entries [L*D, ldE) are set to +inf in U
// and -inf in Lo, so that a padded element never contributes to LB_MV.
constexpr int kEnvTP = 64;

// Output position of element e of query m: row-major (m*ldE + e) or, for the LB_MV
// stream, query-pair interleaved (((m/2)*ldE + e)*2 + m%2).
__device__ __forceinline__ size_t env_pos(int64_t m, int64_t e, int64_t ldE, bool pairs) {
    return pairs ? (size_t)(((m >> 1) * ldE + e) * 2 + (m & 1)) : (size_t)(m * ldE + e);
}

template <bool STAGE>
__global__ void k_envelope(const float *__restrict__ q, int L, int D, int W, float *__restrict__ U,
                           float *__restrict__ Lo, int64_t ldE, int pad, int pairs) {
    extern __shared__ float sh[];
    const int m = blockIdx.y;
    const int t0 = blockIdx.x * kEnvTP;
    const float *qm = q + (size_t)m * L * D;
    const int lo = max(0, t0 - W), hi = min(L - 1, t0 + kEnvTP - 1 + W);
    if (STAGE) {
        const int n = (hi - lo + 1) * D;
        for (int k = threadIdx.x; k < n; k += blockDim.x) sh[k] = __ldg(qm + (size_t)lo * D + k);
        __syncthreads();
    }
    const int rows = min(kEnvTP, L - t0);
    for (int k = threadIdx.x; k < rows * D; k += blockDim.x) {
        const int i = t0 + k / D, p = k % D;
        const int a = max(0, i - W), b = min(L - 1, i + W);
        float u = -TC_INF, l = TC_INF;
        for (int r = a; r <= b; ++r) {
            float v = STAGE ? sh[(r - lo) * D + p] : __ldg(qm + (size_t)r * D + p);
            u = fmaxf(u, v);
            l = fminf(l, v);
        }
        U[env_pos(m, (int64_t)i * D + p, ldE, pairs)] = u;
        Lo[env_pos(m, (int64_t)i * D + p, ldE, pairs)] = l;
    }
    if (pad && blockIdx.x == 0) {
        for (int64_t k = (int64_t)L * D + threadIdx.x; k < ldE; k += blockDim.x) {
            U[env_pos(m, k, ldE, pairs)] = TC_INF;
            Lo[env_pos(m, k, ldE, pairs)] = -TC_INF;
        }
    }
}

static cudaError_t envelope_impl(const float *q, int64_t M, int L, int D, int W, float *U, float *Lo, int ldE,
                                 int pairs, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    if (W > L - 1) W = L - 1;
    dim3 grid((L + kEnvTP - 1) / kEnvTP, (unsigned)M);
    const size_t sh = (size_t)(kEnvTP + 2 * W) * D * sizeof(float);
    const int pad = ldE > L * D;
    if (sh <= 48 * 1024)
        k_envelope<true><<<grid, 128, sh, s>>>(q, L, D, W, U, Lo, ldE, pad, pairs);
    else
        k_envelope<false><<<grid, 128, 0, s>>>(q, L, D, W, U, Lo, ldE, pad, pairs);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_envelope(const float *q, int64_t M, int L, int D, int W, float *U, float *Lo, int ldE,
                            cudaStream_t s) {
    return envelope_impl(q, M, L, D, W, U, Lo, ldE, 0, s);
}

cudaError_t launch_envelope_pairs(const float *q, int64_t M, int L, int D, int W, float *U, float *Lo, int ldE,
                                  cudaStream_t s) {
    return envelope_impl(q, M, L, D, W, U, Lo, ldE, 1, s);
}

// ------------------------------------------------------------------ neighbour distances
// |x - y| as an interval: the larger of the two directed differences is >= 0 and
// rounds in the wanted direction.
__device__ __forceinline__ float absdiff_rd(float x, float y) { return fmaxf(__fsub_rd(x, y), __fsub_rd(y, x)); }
__device__ __forceinline__ float absdiff_ru(float x, float y) { return fmaxf(__fsub_ru(x, y), __fsub_ru(y, x)); }

__global__ void k_query_dq(const float *__restrict__ q, int64_t M, int L, int D, float *__restrict__ dq_lo,
                           float *__restrict__ dq_hi) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M * L) return;
    const int64_t m = k / L;
    const int i = (int)(k % L);
    if (i == 0) {
        dq_lo[k] = 0.f;
        dq_hi[k] = 0.f;
        return;
    }
    const float *a = q + ((size_t)m * L + i - 1) * D;
    const float *b = a + D;
    float slo = 0.f, shi = 0.f;
    for (int p = 0; p < D; ++p) {
        const float x = __ldg(a + p), y = __ldg(b + p);
        const float dl = absdiff_rd(x, y), dh = absdiff_ru(x, y);
        slo = __fmaf_rd(dl, dl, slo);
        shi = __fmaf_ru(dh, dh, shi);
    }
    dq_lo[k] = __fsqrt_rd(slo);
    dq_hi[k] = __fsqrt_ru(shi);
}

cudaError_t launch_query_dq(const float *q, int64_t M, int L, int D, float *dq_lo, float *dq_hi, cudaStream_t s) {
    const int64_t n = M * L;
    if (n <= 0) return cudaSuccess;
    k_query_dq<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(q, M, L, D, dq_lo, dq_hi); note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ LB_PC boxes
// Order-preserving int image of a float (for shared-memory atomic min / max).
__device__ __forceinline__ int f2o(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float o2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// One warp per (query m, group g).  Shared memory per warp:
//   keys  [npow2] uint64 (cell key of each point, padded with ~0 and sorted),
//   dkeys [npow2] uint64 (distinct keys, in order),
//   mn, len [TCDTW_MAX_D] float,
//   box   [K][2][D] int (order-preserving images: lower then upper corner).
// The cell key is the mixed-radix number sum_p cell_p * Lq^(D-1-p): numeric order
// of keys is the lexicographic order of cell tuples with dimension 0 first.
__global__ void k_pc_boxes(const float *__restrict__ q, int L, int D, int W, int K, int Lq, int w, int G,
                           int npow2, float *__restrict__ boxes, int32_t *__restrict__ counts) {
    extern __shared__ unsigned long long shb[];
    const int lane = threadIdx.x;
    const int m = blockIdx.y;
    const int g = blockIdx.x;
    unsigned long long *keys = shb;
    unsigned long long *dkeys = keys + npow2;
    float *mn = (float *)(dkeys + npow2);
    float *len = mn + TCDTW_MAX_D;
    int *box = (int *)(len + TCDTW_MAX_D);

    const float *qm = q + (size_t)m * L * D;
    const int p0 = max(0, g * w - W), p1 = min(L - 1, g * w + w - 1 + W);
    const int n = p1 - p0 + 1;
    // per-dimension range and FP32 cell length (round-to-nearest sub and div)
    for (int p = lane; p < D; p += 32) {
        float lo = __ldg(qm + (size_t)p0 * D + p), hi = lo;
        for (int k = p0 + 1; k <= p1; ++k) {
            float v = __ldg(qm + (size_t)k * D + p);
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
        const float seg = __fdiv_rn(__fsub_rn(hi, lo), (float)Lq);
        mn[p] = lo;
        len[p] = seg > 1e-5f ? seg : 1e-5f;
    }
    __syncwarp();
    // cell key of every point
    for (int t = lane; t < npow2; t += 32) {
        unsigned long long key = ~0ull;
        if (t < n) {
            key = 0;
            const float *x = qm + (size_t)(p0 + t) * D;
            for (int p = 0; p < D; ++p) {
                const float r = __fdiv_rn(__fsub_rn(__ldg(x + p), mn[p]), len[p]);
                int id = (int)floorf(r);
                if (id > Lq - 1) id = Lq - 1;
                key = key * (unsigned long long)Lq + (unsigned long long)id;
            }
        }
        keys[t] = key;
    }
    __syncwarp();
    // bitonic sort of the keys (ascending)
    for (int size = 2; size <= npow2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < npow2 / 2; t += 32) {
                const int lo_i = 2 * t - (t & (stride - 1));
                const int hi_i = lo_i + stride;
                const bool asc = ((lo_i & size) == 0);
                unsigned long long a = keys[lo_i], b = keys[hi_i];
                if ((a > b) == asc) {
                    keys[lo_i] = b;
                    keys[hi_i] = a;
                }
            }
            __syncwarp();
        }
    }
    // distinct keys in order (warp-wide prefix over chunks of 32)
    int base = 0;
    for (int t0 = 0; t0 < n; t0 += 32) {
        const int t = t0 + lane;
        const bool first = t < n && (t == 0 || keys[t] != keys[t - 1]);
        const unsigned bal = __ballot_sync(0xffffffffu, first);
        if (first) dkeys[base + __popc(bal & ((1u << lane) - 1u))] = keys[t];
        base += __popc(bal);
    }
    // empty boxes
    const int nb = min(base, K);
    for (int k = lane; k < nb * D; k += 32) {
        box[(k / D) * 2 * D + (k % D)] = f2o(TC_INF);
        box[(k / D) * 2 * D + D + (k % D)] = f2o(-TC_INF);
    }
    __syncwarp();
    // each point joins the box of its cell's rank (ranks >= K-1 share box K-1)
    for (int t = lane; t < n; t += 32) {
        const float *x = qm + (size_t)(p0 + t) * D;
        unsigned long long key = 0;
        for (int p = 0; p < D; ++p) {
            const float r = __fdiv_rn(__fsub_rn(__ldg(x + p), mn[p]), len[p]);
            int id = (int)floorf(r);
            if (id > Lq - 1) id = Lq - 1;
            key = key * (unsigned long long)Lq + (unsigned long long)id;
        }
        int a = 0, b = base - 1;  // binary search in dkeys
        while (a < b) {
            const int c = (a + b) >> 1;
            if (dkeys[c] < key) a = c + 1; else b = c;
        }
        const int slot = min(a, K - 1);
        for (int p = 0; p < D; ++p) {
            const int v = f2o(__ldg(x + p));
            atomicMin(&box[slot * 2 * D + p], v);
            atomicMax(&box[slot * 2 * D + D + p], v);
        }
    }
    __syncwarp();
    float *out = boxes + ((size_t)m * G + g) * K * 2 * D;
    for (int k = lane; k < nb * 2 * D; k += 32) out[k] = o2f(box[k]);
    if (lane == 0) counts[(size_t)m * G + g] = nb;
}

size_t pc_boxes_smem(int L, int D, int W, int K, int w, int *npow2_out) {
    if (W > L - 1) W = L - 1;
    int maxpts = w + 2 * W;
    if (maxpts > L) maxpts = L;
    int np2 = 32;
    while (np2 < maxpts) np2 <<= 1;
    if (npow2_out) *npow2_out = np2;
    return (size_t)np2 * 16 + 2 * TCDTW_MAX_D * sizeof(float) + (size_t)K * 2 * D * sizeof(int);
}

cudaError_t launch_pc_boxes(const float *q, int64_t M, int L, int D, int W, int K, int Lq, int w, float *boxes,
                            int32_t *counts, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    if (W > L - 1) W = L - 1;
    int np2 = 0;
    const size_t sh = pc_boxes_smem(L, D, W, K, w, &np2);
    if (sh > 227 * 1024) return cudaErrorInvalidValue;
    if (sh > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_pc_boxes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        if (e != cudaSuccess) return e;
    }
    const int G = (L + w - 1) / w;
    dim3 grid(G, (unsigned)M);
    k_pc_boxes<<<grid, 32, sh, s>>>(q, L, D, W, K, Lq, w, G, np2, boxes, counts); note_launch();
    return cudaGetLastError();
}

}  // namespace tc
