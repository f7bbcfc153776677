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
#include "prep_device.cuh"

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
// Window scan (series longer than the van Herk kernel below stages): block (tile t,
// query m) produces rows [t*TP, t*TP+TP) of U and Lo.  The query
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

// Sliding max / min by van Herk / Gil-Werman: in padded coordinates x' = i + W
// (positions outside [0, L-1] hold -inf for the maximum and +inf for the minimum) the
// window of output i is [i, i + 2W], of width w = 2W + 1.  Cut the padded series into
// blocks of w starting at 0; a window either is one whole block or spans the end of one
// block and the start of the next, so U[i] = max(suffix max of i within its block,
// prefix max of i + 2W within its block) -- about three comparisons per element,
// whatever W.  One CTA per (query, group of Dg dimensions) stages the group's L x Dg
// values in shared memory, computes the suffixes of every block (phase 1), then scans
// the prefixes forward and writes the outputs (phase 2); each (dimension, block) pair
// is one thread's sequential scan.  Exact (max / min only).
constexpr int kEnvVhThreads = 128;
constexpr size_t kEnvVhSmemMax = 96 * 1024;

__global__ void __launch_bounds__(kEnvVhThreads) k_envelope_vhgw(const float *__restrict__ q, int L, int D, int W,
                                                                 int Dg, float *__restrict__ U,
                                                                 float *__restrict__ Lo, int64_t ldE, int pad,
                                                                 int pairs, float *__restrict__ U2,
                                                                 float *__restrict__ Lo2) {
    extern __shared__ float sh[];
    float *x = sh, *hmax = sh + (size_t)L * Dg, *hmin = hmax + (size_t)L * Dg;
    const int m = blockIdx.y, p0 = blockIdx.x * Dg, ng = min(Dg, D - p0);
    const float *qm = q + (size_t)m * L * D;
    for (int k = threadIdx.x; k < L * ng; k += blockDim.x) {
        const int i = k / ng, pp = k - i * ng;
        x[i * Dg + pp] = __ldg(qm + (size_t)i * D + p0 + pp);
    }
    __syncthreads();
    const int w = 2 * W + 1, Lp = L + 2 * W;
    // phase 1: suffix max / min within each block, kept where an output window starts
    const int nb1 = (L - 1) / w + 1;
    for (int u = threadIdx.x; u < nb1 * ng; u += blockDim.x) {
        const int b = u / ng, pp = u - b * ng;
        float mx = -TC_INF, mn = TC_INF;
        for (int xp = min(b * w + w - 1, Lp - 1); xp >= b * w; --xp) {
            const int i = xp - W;
            if (i >= 0 && i < L) {
                const float v = x[i * Dg + pp];
                mx = fmaxf(mx, v);
                mn = fminf(mn, v);
            }
            if (xp < L) {
                hmax[xp * Dg + pp] = mx;
                hmin[xp * Dg + pp] = mn;
            }
        }
    }
    __syncthreads();
    // phase 2: prefix max / min within each block; position xp ends the window of output
    // xp - 2W
    const int nb2 = (Lp - 1) / w + 1;
    for (int u = threadIdx.x; u < nb2 * ng; u += blockDim.x) {
        const int b = u / ng, pp = u - b * ng, p = p0 + pp;
        float mx = -TC_INF, mn = TC_INF;
        for (int xp = b * w; xp < min(b * w + w, Lp); ++xp) {
            const int i = xp - W;
            if (i >= 0 && i < L) {
                const float v = x[i * Dg + pp];
                mx = fmaxf(mx, v);
                mn = fminf(mn, v);
            }
            const int o = xp - 2 * W;
            if (o >= 0 && o < L) {
                const float u = fmaxf(hmax[o * Dg + pp], mx), l = fminf(hmin[o * Dg + pp], mn);
                U[env_pos(m, (int64_t)o * D + p, ldE, pairs)] = u;
                Lo[env_pos(m, (int64_t)o * D + p, ldE, pairs)] = l;
                if (U2) {  // the same envelope, one query per row
                    U2[(size_t)m * ldE + (size_t)o * D + p] = u;
                    Lo2[(size_t)m * ldE + (size_t)o * D + p] = l;
                }
            }
        }
    }
    if (pad && blockIdx.x == 0) {
        for (int64_t k = (int64_t)L * D + threadIdx.x; k < ldE; k += blockDim.x) {
            U[env_pos(m, k, ldE, pairs)] = TC_INF;
            Lo[env_pos(m, k, ldE, pairs)] = -TC_INF;
            if (U2) {
                U2[(size_t)m * ldE + k] = TC_INF;
                Lo2[(size_t)m * ldE + k] = -TC_INF;
            }
        }
    }
}

static cudaError_t envelope_impl(const float *q, int64_t M, int L, int D, int W, float *U, float *Lo, int ldE,
                                 int pairs, cudaStream_t s, float *U2 = nullptr, float *Lo2 = nullptr) {
    if (M <= 0) return cudaSuccess;
    if (W > L - 1) W = L - 1;
    const int pad = ldE > L * D;
    // van Herk / Gil-Werman when a CTA can stage at least one dimension of the series
    int Dg = (int)(kEnvVhSmemMax / ((size_t)3 * L * sizeof(float)));
    if (Dg > D) Dg = D;
    if (Dg >= 1) {
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(k_envelope_vhgw, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kEnvVhSmemMax);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        dim3 grid((D + Dg - 1) / Dg, (unsigned)M);
        const size_t sh = (size_t)3 * L * Dg * sizeof(float);
        k_envelope_vhgw<<<grid, kEnvVhThreads, sh, s>>>(q, L, D, W, Dg, U, Lo, ldE, pad, pairs, U2, Lo2);
        note_launch();
        return cudaGetLastError();
    }
    dim3 grid((L + kEnvTP - 1) / kEnvTP, (unsigned)M);
    const size_t sh = (size_t)(kEnvTP + 2 * W) * D * sizeof(float);
    if (sh <= 48 * 1024)
        k_envelope<true><<<grid, 128, sh, s>>>(q, L, D, W, U, Lo, ldE, pad, pairs);
    else
        k_envelope<false><<<grid, 128, 0, s>>>(q, L, D, W, U, Lo, ldE, pad, pairs);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !U2) return e;
    return envelope_impl(q, M, L, D, W, U2, Lo2, ldE, 0, s);  // the one-query-per-row copy
}

cudaError_t launch_envelope(const float *q, int64_t M, int L, int D, int W, float *U, float *Lo, int ldE,
                            cudaStream_t s) {
    return envelope_impl(q, M, L, D, W, U, Lo, ldE, 0, s);
}

cudaError_t launch_envelope_pairs(const float *q, int64_t M, int L, int D, int W, float *U, float *Lo, int ldE,
                                  cudaStream_t s) {
    return envelope_impl(q, M, L, D, W, U, Lo, ldE, 1, s);
}

cudaError_t launch_envelope_pairs_plain(const float *q, int64_t M, int L, int D, int W, float *U, float *Lo,
                                        float *U2, float *Lo2, int ldE, cudaStream_t s) {
    return envelope_impl(q, M, L, D, W, U, Lo, ldE, 1, s, U2, Lo2);
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


__global__ void k_pc_boxes(const float *__restrict__ q, int L, int D, int W, int K, int Lq, int w, int G, int npow2,
                           float *__restrict__ boxes, int32_t *__restrict__ counts) {
    extern __shared__ unsigned long long shb[];
    const int m = blockIdx.y, g = blockIdx.x;
    pc_boxes_group(q + (size_t)m * L * D, L, D, W, K, Lq, w, g, npow2, shb, boxes + ((size_t)m * G + g) * K * 2 * D,
                   counts + (size_t)m * G + g);
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
