// df.cuh -- double-float (pairs of FP32) DTW for the refine step.
//
// The exact nearest neighbour is the FP64 argmin of Eq. (1) (ties: smallest
// index).  FP64 issues at a small fraction of the FP32 rate on this GPU, so the
// candidates that FP32 cannot separate from the best one are first recomputed in
// double-float arithmetic (a value hi + lo of two floats, ~2^-48 relative per
// operation) with a proven relative error bound; only candidates whose double-float
// intervals still overlap the best one's go on to a native FP64 recompute.
//
// Cell cost.  For each dimension p, TwoSum gives th + tl = a_p - b_p exactly and
// TwoProd gives ph + pl = th^2 exactly; the large parts ph are summed exactly by
// TwoSum into sh (the rounding errors e go to the small part), the small parts
// e + pl + 2 th tl + tl^2 (each at most ~D u of the cost) are summed in FP32 into
// sl.  Only the FP32 sum of the small parts rounds: the relative error of a cell
// cost is at most (3D+2)(D+3) u^2 / (1 - (3D+2) u), u = 2^-24.
//
// DP.  R(i,j) = cost + min(up, left, diag) with a double-word addition of relative
// error at most 3u^2 (1 + O(u)) for non-negative operands (df_add; bounded by 4u^2
// below); the minimum compares (hi, lo) exactly.  By induction over the DP, with the
// minimum taken over values that are each within the bound of their exact values,
// the computed R(L-1, L-1) is within a relative (1 + e_cost)(1 + 4u^2)^(2L) - 1 of
// the exact DTW, 2L-1 being the longest warping path (the host computes the bound,
// see refine_kappa).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "dtw_core.cuh"  // lane groups and band geometry

namespace tc {

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// (zh, zl) = (xh, xl) + (yh, yl) for non-negative finite double-words (|xl| <= u xh,
// |yl| <= u yh).  TwoSum gives s + e0 = xh + yh exactly; the low parts are added
// in two roundings, then FastTwoSum renormalises exactly.  The error is
// e0 d2 + (xl + yl)((1+d1)(1+d2) - 1) with |e0| <= u s and |xl + yl| <= u (xh + yh):
// at most 3u^2 (1 + O(u)) of the sum.  (With operands of opposite signs this short
// form can lose all accuracy; DP values and cell costs are never negative.)
__device__ __forceinline__ void df_add(float xh, float xl, float yh, float yl, float &zh, float &zl) {
    float s, e0;
    two_sum(xh, yh, s, e0);
    const float e = __fadd_rn(e0, __fadd_rn(xl, yl));
    fast_two_sum(s, e, zh, zl);
}

__device__ __forceinline__ bool df_less(float ah, float al, float bh, float bl) {
    return ah < bh || (ah == bh && al < bl);
}

// Accumulate t^2 for an exact difference t = th + tl into (sh, sl): TwoProd gives
// ph + pl = th^2 exactly, ph joins the exact running sum sh by TwoSum, and the small
// parts (the TwoSum error, pl, 2 th tl and tl^2) go to sl in FP32.
__device__ __forceinline__ void df_square_term(float th, float tl, float &sh, float &sl) {
    const float ph = __fmul_rn(th, th);
    const float pl = __fmaf_rn(th, th, -ph);                 // ph + pl = th^2
    float q = __fmaf_rn(__fadd_rn(th, th), tl, pl);          // pl + 2 th tl
    q = __fmaf_rn(tl, tl, q);                                // + tl^2
    float e;
    two_sum(sh, ph, sh, e);                                  // exact running sum of ph
    sl = __fadd_rn(sl, __fadd_rn(e, q));
}

// Double-float DTW of one pair by one warp (g.G = 32), R rows per lane, D at run
// time; same band sweep as the FP32 and FP64 passes.  Returns hi + lo rounded to
// double on the lane that computed R(L-1, L-1), +inf elsewhere.
template <int R>
__device__ double band_pass_df(const float *__restrict__ A, const float *__restrict__ B, int L, int D, int W,
                               const Grp &g) {
    const float INF = TC_INF;
    float ch[R], cl[R];
    float bot_h = INF, bot_l = 0.f, prev_h = INF, prev_l = 0.f;
    float res_h = INF, res_l = 0.f;
    const int nv = (L + R - 1) / R;
    const int vlast = (L - 1) / R;
    int v = g.lig;
    const int tau_end = v_jhi(nv - 1, R, W, L) + (nv - 1);
    int tlo = v < nv ? v_jlo(v, R, W) + v : 1 << 30;
    int thi = v < nv ? v_jhi(v, R, W, L) + v : -1;
    bool fresh = true;
    for (int tau = 0; tau <= tau_end; ++tau) {
        const float in_h = __shfl_sync(g.mask, bot_h, g.src);
        const float in_l = __shfl_sync(g.mask, bot_l, g.src);
        if (tau > thi && v < nv) {
            v += g.G;
            fresh = true;
            tlo = v < nv ? v_jlo(v, R, W) + v : 1 << 30;
            thi = v < nv ? v_jhi(v, R, W, L) + v : -1;
        }
        if (tau >= tlo && tau <= thi) {
            const int j = tau - v;
            const int i0 = v * R;
            if (fresh) {
#pragma unroll
                for (int r = 0; r < R; ++r) { ch[r] = INF; cl[r] = 0.f; }
                fresh = false;
            }
            float up_h = INF, up_l = 0.f, dg_h = INF, dg_l = 0.f;
            if (v == 0) {
                if (j == 0) dg_h = 0.f;
            } else {
                if (j <= i0 - 1 + W) { up_h = in_h; up_l = in_l; }
                if (j >= 1 && j <= i0 + W) { dg_h = prev_h; dg_l = prev_l; }
            }
            const unsigned vm = row_mask(j - W - i0, min(j + W - i0, L - 1 - i0), R);
            const float *bj = B + (size_t)j * D;
            float sh[R], sl[R];
#pragma unroll
            for (int r = 0; r < R; ++r) { sh[r] = 0.f; sl[r] = 0.f; }
            for (int p = 0; p < D; ++p) {
                const float b = __ldg(bj + p);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    float th, tl;
                    two_sum(__ldg(A + (size_t)min(i0 + r, L - 1) * D + p), -b, th, tl);  // th + tl = a - b
                    df_square_term(th, tl, sh[r], sl[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float lh = ch[r], ll = cl[r];
                float vh = INF, vl = 0.f;
                if ((vm >> r) & 1u) {
                    float mh = up_h, ml = up_l;
                    if (df_less(lh, ll, mh, ml)) { mh = lh; ml = ll; }
                    if (df_less(dg_h, dg_l, mh, ml)) { mh = dg_h; ml = dg_l; }
                    if (mh < INF) {
                        float c0, c1;
                        fast_two_sum(sh[r], sl[r], c0, c1);
                        df_add(c0, c1, mh, ml, vh, vl);
                    }
                }
                dg_h = lh; dg_l = ll;
                up_h = vh; up_l = vl;
                ch[r] = vh; cl[r] = vl;
            }
            bot_h = ch[R - 1];
            bot_l = cl[R - 1];
            if (v == vlast && j == L - 1) {
                const int rl = (L - 1) - i0;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (r == rl) { res_h = ch[r]; res_l = cl[r]; }
            }
        }
        prev_h = in_h;
        prev_l = in_l;
    }
    // the only FP64 operations: after the loop (FP64 issues at a small fraction of
    // the FP32 rate; nothing FP64 may sit in the loop body)
    return res_h < INF ? __dadd_rn((double)res_h, (double)res_l) : __longlong_as_double(0x7ff0000000000000LL);
}

// A point of D floats (D <= DM) into registers, zero-padded to DM; vec: 16-byte loads
// (D a multiple of 4, p 16-byte aligned).
template <int DM>
__device__ __forceinline__ void df_load_point(const float *p, int D, bool vec, float (&x)[DM]) {
    if (vec) {
#pragma unroll
        for (int k = 0; k < DM / 4; ++k) {
            const float4 v = 4 * k < D ? __ldg(reinterpret_cast<const float4 *>(p) + k) : make_float4(0.f, 0.f, 0.f, 0.f);
            x[4 * k] = v.x;
            x[4 * k + 1] = v.y;
            x[4 * k + 2] = v.z;
            x[4 * k + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < DM; ++k) x[k] = k < D ? __ldg(p + k) : 0.f;
    }
}

// df_cell_cost (below) of two points already in registers: the same operations in the
// same order, so the same value.
template <int DM>
__device__ __forceinline__ void df_cell_cost_regs(const float (&a)[DM], const float (&b)[DM], int D, float &c_h,
                                                  float &c_l) {
    float sh = 0.f, sl = 0.f;
#pragma unroll
    for (int p = 0; p < DM; ++p) {
        if (p < D) {
            float th, tl;
            two_sum(a[p], -b[p], th, tl);
            df_square_term(th, tl, sh, sl);
        }
    }
    fast_two_sum(sh, sl, c_h, c_l);
}

// Double-float cost of one cell (rows a and b of D floats, D <= DM), in the operation
// order of band_pass_df: (c_h, c_l) = FastTwoSum of the exact-part sum and the
// small-part sum.
template <int DM>
__device__ __forceinline__ void df_cell_cost(const float *a, const float *b, int D, float &c_h, float &c_l) {
    float sh = 0.f, sl = 0.f;
#pragma unroll
    for (int p = 0; p < DM; ++p) {
        if (p < D) {
            float th, tl;
            two_sum(a[p], -b[p], th, tl);  // th + tl = a - b
            df_square_term(th, tl, sh, sl);
        }
    }
    fast_two_sum(sh, sl, c_h, c_l);
}

// The double-float band DP of one pair by one warp (G = 32, R rows per lane) with the
// cell costs already in a table: cost[i * (2W+1) + (j - i + W)] = (c_h, c_l) of cell
// (i, j).  Same sweep and update as band_pass_df, so the result is bit-identical; a
// step is then only the two shuffles and the double-word minimum and addition, which
// is what bounds a lone warp (the cost arithmetic is a long serial chain per cell).
template <int R>
__device__ double band_pass_df_table(const float2 *cost, int L, int W, const Grp &g) {
    const float INF = TC_INF;
    const int BW = 2 * W + 1;
    float ch[R], cl[R];
    float bot_h = INF, bot_l = 0.f, prev_h = INF, prev_l = 0.f;
    float res_h = INF, res_l = 0.f;
    const int nv = (L + R - 1) / R;
    const int vlast = (L - 1) / R;
    int v = g.lig;
    const int tau_end = v_jhi(nv - 1, R, W, L) + (nv - 1);
    int tlo = v < nv ? v_jlo(v, R, W) + v : 1 << 30;
    int thi = v < nv ? v_jhi(v, R, W, L) + v : -1;
#pragma unroll
    for (int r = 0; r < R; ++r) { ch[r] = INF; cl[r] = 0.f; }
    for (int tau = 0; tau <= tau_end; ++tau) {
        const float in_h = __shfl_sync(g.mask, bot_h, g.src);
        const float in_l = __shfl_sync(g.mask, bot_l, g.src);
        if (tau > thi && v < nv) {
            v += g.G;
            tlo = v < nv ? v_jlo(v, R, W) + v : 1 << 30;
            thi = v < nv ? v_jhi(v, R, W, L) + v : -1;
#pragma unroll
            for (int r = 0; r < R; ++r) { ch[r] = INF; cl[r] = 0.f; }
        }
        if (tau >= tlo && tau <= thi) {
            const int j = tau - v;
            const int i0 = v * R;
            float up_h = INF, up_l = 0.f, dg_h = INF, dg_l = 0.f;
            if (v == 0) {
                if (j == 0) dg_h = 0.f;
            } else {
                if (j <= i0 - 1 + W) { up_h = in_h; up_l = in_l; }
                if (j >= 1 && j <= i0 + W) { dg_h = prev_h; dg_l = prev_l; }
            }
            const unsigned vm = row_mask(j - W - i0, min(j + W - i0, L - 1 - i0), R);
            float2 c[R];
#pragma unroll
            for (int r = 0; r < R; ++r)
                c[r] = ((vm >> r) & 1u) ? cost[(size_t)(i0 + r) * BW + (j - (i0 + r) + W)] : make_float2(0.f, 0.f);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float lh = ch[r], ll = cl[r];
                float vh = INF, vl = 0.f;
                if ((vm >> r) & 1u) {
                    float mh = up_h, ml = up_l;
                    if (df_less(lh, ll, mh, ml)) { mh = lh; ml = ll; }
                    if (df_less(dg_h, dg_l, mh, ml)) { mh = dg_h; ml = dg_l; }
                    if (mh < INF) df_add(c[r].x, c[r].y, mh, ml, vh, vl);
                }
                dg_h = lh; dg_l = ll;
                up_h = vh; up_l = vl;
                ch[r] = vh; cl[r] = vl;
            }
            bot_h = ch[R - 1];
            bot_l = cl[R - 1];
            if (v == vlast && j == L - 1) {
                const int rl = (L - 1) - i0;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (r == rl) { res_h = ch[r]; res_l = cl[r]; }
            }
        }
        prev_h = in_h;
        prev_l = in_l;
    }
    return res_h < INF ? __dadd_rn((double)res_h, (double)res_l) : __longlong_as_double(0x7ff0000000000000LL);
}

// The same sweep with the cost table in global memory, stored in the order the sweep
// reads it: the R costs lane l uses at step tau (its virtual lane's rows at column
// tau - v) are entries ((tau * 32 + l) * R + r) (table_dp_pos).  Each lane streams its
// own 8R bytes per step through a private ring of kDfRing steps in shared memory (ring:
// 32 * R * kDfRing float2 per warp), copied with cp.async kDfRing steps ahead, so the
// latency of the table's L2/HBM reads overlaps the sweep instead of stalling every step.
// Entries the sweep does not use (outside the band, idle lanes) are never written and
// never read as costs.  Same operations in the same order: bit-identical.
constexpr int kDfRing = 8;

__host__ __device__ inline size_t table_dp_pos(int tau, int lane, int R, int r) {
    return ((size_t)tau * 32 + lane) * R + r;
}

template <int R>
__device__ __forceinline__ void df_ring_issue(float2 *slot, const float2 *src) {
    if ((R * 8) % 16 == 0) {
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            const unsigned sa = (unsigned)__cvta_generic_to_shared(slot + 2 * k);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src + 2 * k) : "memory");
        }
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const unsigned sa = (unsigned)__cvta_generic_to_shared(slot + k);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src + k) : "memory");
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int R>
__device__ double band_pass_df_table_dp(const float2 *cost, int L, int W, const Grp &g, float2 *ring) {
    const float INF = TC_INF;
    float ch[R], cl[R];
    float bot_h = INF, bot_l = 0.f, prev_h = INF, prev_l = 0.f;
    float res_h = INF, res_l = 0.f;
    const int nv = (L + R - 1) / R;
    const int vlast = (L - 1) / R;
    int v = g.lig;
    const int tau_end = v_jhi(nv - 1, R, W, L) + (nv - 1);
    int tlo = v < nv ? v_jlo(v, R, W) + v : 1 << 30;
    int thi = v < nv ? v_jhi(v, R, W, L) + v : -1;
    float2 *myring = ring + (size_t)g.lig * R;  // slot s of this lane: myring + s * 32 * R
    // prologue: the first kDfRing steps in flight
#pragma unroll
    for (int s = 0; s < kDfRing; ++s) {
        if (s <= tau_end) df_ring_issue<R>(myring + (size_t)s * 32 * R, cost + table_dp_pos(s, g.lig, R, 0));
        else asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
#pragma unroll
    for (int r = 0; r < R; ++r) { ch[r] = INF; cl[r] = 0.f; }
    for (int tau = 0; tau <= tau_end; ++tau) {
        const int slot = tau % kDfRing;
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kDfRing - 1) : "memory");  // this step's copy is in
        float2 c[R];
#pragma unroll
        for (int r = 0; r < R; ++r) c[r] = myring[(size_t)slot * 32 * R + r];
        // the slot now holds this step's costs in registers: refill it for step tau + kDfRing
        if (tau + kDfRing <= tau_end)
            df_ring_issue<R>(myring + (size_t)slot * 32 * R, cost + table_dp_pos(tau + kDfRing, g.lig, R, 0));
        else
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        const float in_h = __shfl_sync(g.mask, bot_h, g.src);
        const float in_l = __shfl_sync(g.mask, bot_l, g.src);
        if (tau > thi && v < nv) {
            v += g.G;
            tlo = v < nv ? v_jlo(v, R, W) + v : 1 << 30;
            thi = v < nv ? v_jhi(v, R, W, L) + v : -1;
#pragma unroll
            for (int r = 0; r < R; ++r) { ch[r] = INF; cl[r] = 0.f; }
        }
        if (tau >= tlo && tau <= thi) {
            const int j = tau - v;
            const int i0 = v * R;
            float up_h = INF, up_l = 0.f, dg_h = INF, dg_l = 0.f;
            if (v == 0) {
                if (j == 0) dg_h = 0.f;
            } else {
                if (j <= i0 - 1 + W) { up_h = in_h; up_l = in_l; }
                if (j >= 1 && j <= i0 + W) { dg_h = prev_h; dg_l = prev_l; }
            }
            const unsigned vm = row_mask(j - W - i0, min(j + W - i0, L - 1 - i0), R);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float lh = ch[r], ll = cl[r];
                float vh = INF, vl = 0.f;
                if ((vm >> r) & 1u) {
                    float mh = up_h, ml = up_l;
                    if (df_less(lh, ll, mh, ml)) { mh = lh; ml = ll; }
                    if (df_less(dg_h, dg_l, mh, ml)) { mh = dg_h; ml = dg_l; }
                    if (mh < INF) df_add(c[r].x, c[r].y, mh, ml, vh, vl);
                }
                dg_h = lh; dg_l = ll;
                up_h = vh; up_l = vl;
                ch[r] = vh; cl[r] = vl;
            }
            bot_h = ch[R - 1];
            bot_l = cl[R - 1];
            if (v == vlast && j == L - 1) {
                const int rl = (L - 1) - i0;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (r == rl) { res_h = ch[r]; res_l = cl[r]; }
            }
        }
        prev_h = in_h;
        prev_l = in_l;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    return res_h < INF ? __dadd_rn((double)res_h, (double)res_l) : __longlong_as_double(0x7ff0000000000000LL);
}

}  // namespace tc
