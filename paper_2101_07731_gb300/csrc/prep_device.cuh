// prep_device.cuh -- device building blocks of the query preparation (LB_PC boxes),
// shared by prep.cu and the batched persistent kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace tc {

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
// Boxes of group g of query qm (one warp; shb: this warp's shared scratch of
// pc_boxes_smem bytes); writes out_boxes [K][2][D] and *out_count.
__device__ inline void pc_boxes_group(const float *__restrict__ qm, int L, int D, int W, int K, int Lq, int w, int g,
                                      int npow2, unsigned long long *shb, float *__restrict__ out_boxes,
                                      int32_t *__restrict__ out_count) {
    const int lane = threadIdx.x & 31;
    unsigned long long *keys = shb;
    unsigned long long *dkeys = keys + npow2;
    float *mn = (float *)(dkeys + npow2);
    float *len = mn + TCDTW_MAX_D;
    int *box = (int *)(len + TCDTW_MAX_D);

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
    for (int k = lane; k < nb * 2 * D; k += 32) out_boxes[k] = o2f(box[k]);
    if (lane == 0) *out_count = nb;
    __syncwarp();
}

}  // namespace tc
