// lb_device.cuh -- device building blocks of the lower-bound stage, shared by the
// per-stage kernels (lb.cu) and the batched persistent kernel (batch.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace tc {

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

// Candidate rows are ldC floats apart and hold Erow valid elements; e0 is the row
// element where the chunk starts.
template <int QB>
__device__ __forceinline__ void mv_issue(const float *__restrict__ cand, int64_t N, int Erow, int64_t ldC, bool vec4,
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
            const bool ok = n < N && e < Erow;
            const float *src = ok ? cand + (size_t)n * ldC + e : cand;
            cp_async16(sc + row * kMvChunk + ((seg ^ (row & 7)) << 2), src, ok ? 16 : 0);
        }
    } else {
        for (int k = 0; k < kMvRows * kMvChunk / 128; ++k) {
            const int idx = tid + 128 * k;
            const int row = idx >> 5, el = idx & 31;
            const int64_t n = n0 + row;
            const int e = e0 + el;
            const bool ok = n < N && e < Erow;
            const float *src = ok ? cand + (size_t)n * ldC + e : cand;
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

// One LB_MV tile: candidates [n0, n0+128) x queries [q0, q0+QB) of the stream, using
// the caller's shared buffers sc[2][128*32], su[2][QB*32], sl[2][QB*32] (16-byte aligned).
// The tile sums nchunks chunks of 32 elements, chunk k starting at row element
// k * cstride * 32 (cstride 1: the first nchunks chunks; rows hold Erow elements).
template <int QB>
__device__ __forceinline__ void lb_mv_tile(const float *__restrict__ cand, int64_t N, int nchunks, int cstride,
                                           int Erow, int64_t ldC, bool vec4,
                                           const float *__restrict__ UI, const float *__restrict__ LI, int64_t ldE,
                                           int Mb, float *__restrict__ lb, int64_t ldLb, int64_t n0, int q0,
                                           float (*sc)[kMvRows * kMvChunk], float (*su)[QB * kMvChunk],
                                           float (*sl)[QB * kMvChunk]) {
    const int tid = threadIdx.x;
    const int n_qp = (Mb + 1) / 2;
    f2 acc[QB / 2];
#pragma unroll
    for (int k = 0; k < QB / 2; ++k) acc[k] = 0ull;
    mv_issue<QB>(cand, N, Erow, ldC, vec4, UI, LI, ldE, n_qp, n0, q0, 0, sc[0], su[0], sl[0]);
    cp_async_commit();
    for (int c = 0; c < nchunks; ++c) {
        const int buf = c & 1;
        if (c + 1 < nchunks) {
            mv_issue<QB>(cand, N, Erow, ldC, vec4, UI, LI, ldE, n_qp, n0, q0, (c + 1) * cstride * kMvChunk,
                         sc[buf ^ 1], su[buf ^ 1], sl[buf ^ 1]);
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

constexpr int kMaxSeeds = 8;

__device__ __forceinline__ bool lex_less(float a, uint32_t ia, float b, uint32_t ib) {
    return a < b || (a == b && ia < ib);
}

// The S smallest bounds of one row (ties: smaller n), computed by the whole CTA
// (blockDim.x a multiple of 32, at most 1024).  out[r] = n of the r-th smallest
// (UINT32_MAX when the row has fewer than r+1 finite bounds); the chosen entries of
// the row are set to +inf so that they do not survive compaction.  Must be called by
// every thread of the CTA; ends with a __syncthreads().
__device__ inline void seed_topk_row(float *__restrict__ row, int64_t N, int S, uint32_t *out) {
    __shared__ float cv[32][kMaxSeeds];
    __shared__ uint32_t ci[32][kMaxSeeds];
    float bv[kMaxSeeds];
    uint32_t bi[kMaxSeeds];
#pragma unroll
    for (int k = 0; k < kMaxSeeds; ++k) { bv[k] = TC_INF; bi[k] = 0xffffffffu; }
    // four loads in flight per thread (the row is an L2-resident, latency-bound read);
    // the lexicographic (bound, n) order makes the result independent of visit order
    const int64_t bd = blockDim.x;
    for (int64_t n0 = threadIdx.x; n0 < N; n0 += 4 * bd) {
        float v4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v4[u] = n0 + u * bd < N ? row[n0 + u * bd] : TC_INF;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float v = v4[u];
            uint32_t iv = (uint32_t)(n0 + u * bd);
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
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // warp level: S rounds of arg-min over the lanes' list heads
    for (int r = 0; r < S; ++r) {
        float v = bv[0];
        uint32_t iv = bi[0];
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
        }
    }
    __syncthreads();
    if (warp == 0) {
        // merge the per-warp sorted lists: lane l < nw walks warp l's list
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
                out[r] = wi;
                if (wi != 0xffffffffu) row[wi] = TC_INF;
            }
        }
    }
    __syncthreads();
}

// ============================================================== LB_PC / LB_TI of one pair
// Warp-level: every lane of the warp calls with the same pair.  The live threshold is
// re-read from the query's packed best-so-far after every 32 candidate points; the
// function returns true (dropped) as soon as the partial bound exceeds it, else
// false with the bound (rounded down) in *bound on every lane.
// Loads of per-query data (boxes, neighbour distances): through the read-only path,
// or, for data written earlier in the same launch (kCoherent), through L2 only.
template <bool kCoherent>
__device__ __forceinline__ float ld_q(const float *p) {
    return kCoherent ? __ldcg(p) : *p;  // plain: p may also point to shared memory
}

__device__ __forceinline__ float warp_sum_rd(float v) {
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rd(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// LB_PC (Section 5): candidate point j is bounded by its nearest box among the boxes
// of group j / w (boxes of this query: bx_m [G][K][2][D], counts cnt_m [G]).
template <int DMAX, bool kCoherent = false>
__device__ __forceinline__ bool lb_pc_pair(const float *__restrict__ c, const float *__restrict__ bx_m,
                                           const int32_t *__restrict__ cnt_m, int L, int D, int K, int w,
                                           const unsigned long long *bsf_m, float rho, float *bound) {
    const int lane = threadIdx.x & 31;
    float acc = 0.f;
    for (int j0 = 0; j0 < L; j0 += 32) {
        const int j = j0 + lane;
        if (j < L) {
            float x[DMAX];
#pragma unroll
            for (int p = 0; p < DMAX; ++p) x[p] = p < D ? __ldg(c + (size_t)j * D + p) : 0.f;
            const int g = j / w;
            const int nb = kCoherent ? __ldcg(cnt_m + g) : cnt_m[g];
            const float *bx = bx_m + (size_t)g * K * 2 * D;
            float best = TC_INF;
            for (int k = 0; k < nb; ++k) {
                float s = 0.f;
#pragma unroll
                for (int p = 0; p < DMAX; ++p)
                    if (p < D) s = acc_box(x[p], ld_q<kCoherent>(bx + k * 2 * D + p), ld_q<kCoherent>(bx + k * 2 * D + D + p), s);
                best = fminf(best, s);
            }
            acc = __fadd_rd(acc, best);
        }
        const float tot = warp_sum_rd(acc);
        if (tot > prune_threshold(ld_volatile_u64(bsf_m), rho)) return true;
    }
    *bound = warp_sum_rd(acc);
    return false;
}

// |q_i - c| as an interval with directed rounding throughout (two sums, two square
// roots): exact whenever every step is (small-integer series).  Used by the row-sweep
// variants, whose exact rows are few.
template <int DMAX>
__device__ __forceinline__ void exact_interval_rd(const float *__restrict__ qi, const float (&x)[DMAX], int D,
                                                  float *lo, float *hi) {
    float sl = 0.f, sh = 0.f;
#pragma unroll
    for (int p = 0; p < DMAX; ++p) {
        if (p < D) {
            const float y = qi[p];
            const float dl = fmaxf(__fsub_rd(x[p], y), __fsub_rd(y, x[p]));
            const float dh = fmaxf(__fsub_ru(x[p], y), __fsub_ru(y, x[p]));
            sl = __fmaf_rd(dl, dl, sl);
            sh = __fmaf_ru(dh, dh, sh);
        }
    }
    *lo = __fsqrt_rd(sl);
    *hi = __fsqrt_ru(sh);
}

// |q_i - x| as an interval [lo, hi] from one FP32 sum.  s = sum_p (q_p - x_p)^2 with
// round-to-nearest subtractions and fused multiply-adds: s lies within a factor
// (1 +- u)^2 (1 +- g_D) of the exact squared distance S (g_D = D u / (1 - D u), u =
// 2^-24), and r = sqrt(s) correctly rounded within (1 +- u) of sqrt(s), so sqrt(S) lies
// in [r (1 - k), r (1 + k)] with k = (D + 4) u (covering 2u + g_D / 2 + O(u^2)).  The
// factors are applied with directed rounding (klo = 1 - k rounded down, khi = 1 + k
// rounded up), and 2^-70 of absolute slack covers terms that fall into the subnormal
// range (D terms of at most 2^-150 absolute error each; sqrt(64 * 2^-149) < 2^-70).
// One square root per exact cell instead of two directed-rounding ones.
template <int DMAX>
__device__ __forceinline__ void exact_interval(const float *qi, const float (&x)[DMAX], int D, float klo, float khi,
                                               float *lo, float *hi) {
    float sum = 0.f;
#pragma unroll
    for (int p = 0; p < DMAX; ++p) {
        if (p < D) {
            const float d = __fsub_rn(qi[p], x[p]);
            sum = __fmaf_rn(d, d, sum);
        }
    }
    const float r = __fsqrt_rn(sum);
    const float slack = 8.470329472543003e-22f;  // 2^-70
    *lo = fmaxf(__fsub_rd(__fmul_rd(r, klo), slack), 0.f);
    *hi = __fadd_ru(__fmul_ru(r, khi), slack);
}

// The relative widening factors of exact_interval for D dimensions.
__device__ __forceinline__ void exact_interval_factors(int D, float *klo, float *khi) {
    const float k = (float)(D + 4) * 5.9604644775390625e-8f;  // (D + 4) * 2^-24, exact
    *klo = __fsub_rd(1.f, k);
    *khi = __fadd_ru(1.f, k);
}

// LB_TI, TIP_TOP (Section 4).  Lane = candidate point j (column of the cost matrix);
// the rows of its window are i in [i0, i1] = [max(0, j-W), min(L-1, j+W)].  Row i0 is
// exact (the top of the window of row j-W, or row 0, and 0 mod P == 0); rows with
// i mod P == 0 are exact; the others follow Lb = max(Lb - dq_i, dq_i - Ub, 0),
// Ub = Ub + dq_i with dq_i rounded up where it is subtracted from Lb / added to Ub
// and rounded down where Ub is subtracted from it.  bound = sum_j (min_i Lb)^2.
// The lanes of a round take columns of one residue class modulo P (j = r, r+P, ...):
// their window tops j - W share a residue, so at each step of the row recursion either
// every lane's row is exact or none is, and the warp does not run both paths every
// step (with P >= L no row after the top is exact and the columns go in order).  (Two
// columns of the class per lane, as two interleaved chains, measured slower.)  q, dql,
// dqh may point to shared memory (a staged query) or to global memory.  Abandons
// against the live threshold after every round.
template <int DMAX>
__device__ __forceinline__ bool lb_ti_pair(const float *__restrict__ c, const float *q, const float *dql,
                                           const float *dqh, int L, int D, int W, int P,
                                           const unsigned long long *bsf_m, float rho, float *bound) {
    const int lane = threadIdx.x & 31;
    float klo, khi;
    exact_interval_factors(D, &klo, &khi);
    const int nphase = P < L ? P : 1, stride = P < L ? P : 1;
    float acc = 0.f;
    for (int r = 0; r < nphase; ++r) {
        for (int jb = r; jb < L; jb += 32 * stride) {
            const int j = jb + stride * lane;
            if (j < L) {
                float x[DMAX];
#pragma unroll
                for (int p = 0; p < DMAX; ++p) x[p] = p < D ? __ldg(c + (size_t)j * D + p) : 0.f;
                const int i0 = max(0, j - W), i1 = min(L - 1, j + W);
                float lbv, ubv;
                exact_interval<DMAX>(q + (size_t)i0 * D, x, D, klo, khi, &lbv, &ubv);
                float mj = lbv;
                int next_exact = (i0 / P + 1) * P;
                for (int i = i0 + 1; i <= i1; ++i) {
                    if (i == next_exact) {
                        exact_interval<DMAX>(q + (size_t)i * D, x, D, klo, khi, &lbv, &ubv);
                        next_exact += P;
                    } else {
                        const float dl = dql[i], dh = dqh[i];
                        const float nl = fmaxf(fmaxf(__fsub_rd(lbv, dh), __fsub_rd(dl, ubv)), 0.f);
                        ubv = __fadd_ru(ubv, dh);
                        lbv = nl;
                    }
                    mj = fminf(mj, lbv);
                }
                acc = __fmaf_rd(mj, mj, acc);
            }
            const float tot = warp_sum_rd(acc);
            if (tot > prune_threshold(ld_volatile_u64(bsf_m), rho)) return true;
        }
    }
    *bound = warp_sum_rd(acc);
    return false;
}

// |a - b| of two candidate points as an interval (both from global memory).
template <int DMAX>
__device__ __forceinline__ void point_interval(const float *__restrict__ a, const float *__restrict__ b, int D, float *lo,
                                               float *hi) {
    float sl = 0.f, sh = 0.f;
#pragma unroll
    for (int p = 0; p < DMAX; ++p) {
        if (p < D) {
            const float x = __ldg(a + p), y = __ldg(b + p);
            const float dl = fmaxf(__fsub_rd(x, y), __fsub_rd(y, x));
            const float dh = fmaxf(__fsub_ru(x, y), __fsub_ru(y, x));
            sl = __fmaf_rd(dl, dl, sl);
            sh = __fmaf_ru(dh, dh, sh);
        }
    }
    *lo = __fsqrt_rd(sl);
    *hi = __fsqrt_ru(sh);
}

// LB_TI without the exact window top (Section 4.2: the basic LB_TI when P >= L, LB_TIP
// otherwise): the top c_{i+W} of a non-periodic row's window comes from the candidate-
// side triangle with c_{i+W-1} (Eqs. (bt_lb_ir), (bt_ub_ir)), which chains consecutive
// columns of the same row, so the pair is swept row by row instead of one lane per
// column.  The warp holds row i's window by offset k = j - i + W in [0, 2W]: lane l,
// slot s holds k = l + 32 s (NS slots, 32 NS >= 2W + 1).  Between rows the window
// shifts down one offset (shuffles); the column leaving at the bottom adds its minimum
// squared (rounded down).  Per row: i mod P == 0 -> every point exact; otherwise the
// query-side recursion with [dq_lo, dq_hi] for k < 2W, then the top from offset 2W-1's
// (Lb, Ub) and [dc_lo, dc_hi] = |c_{j-1} - c_j| (exact when W = 0: no neighbour in the
// window).  Same rounding directions as lb_ti_pair.  Returns the bound (every lane).
template <int DMAX, int NS>
__device__ __forceinline__ float lb_ti_rows_pair(const float *__restrict__ c, const float *__restrict__ q,
                                                 const float *__restrict__ dql, const float *__restrict__ dqh, int L,
                                                 int D, int W, int P) {
    const int lane = threadIdx.x & 31;
    const float INF = TC_INF;
    float lb[NS], ub[NS], mn[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) { lb[s] = INF; ub[s] = INF; mn[s] = INF; }
    float acc = 0.f;
    const int kt = 2 * W;  // offset of the window top
    for (int i = 0; i < L; ++i) {
        if (i > 0) {
            // the column leaving the window: offset 0 of row i-1, column i-1-W
            if (lane == 0 && i - 1 - W >= 0) acc = __fmaf_rd(mn[0], mn[0], acc);
            float nl[NS], nu[NS], nm[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const float dl = __shfl_down_sync(0xffffffffu, lb[s], 1);
                const float du = __shfl_down_sync(0xffffffffu, ub[s], 1);
                const float dm = __shfl_down_sync(0xffffffffu, mn[s], 1);
                const float wl = __shfl_sync(0xffffffffu, s + 1 < NS ? lb[s + 1 < NS ? s + 1 : s] : INF, 0);
                const float wu = __shfl_sync(0xffffffffu, s + 1 < NS ? ub[s + 1 < NS ? s + 1 : s] : INF, 0);
                const float wm = __shfl_sync(0xffffffffu, s + 1 < NS ? mn[s + 1 < NS ? s + 1 : s] : INF, 0);
                nl[s] = lane == 31 ? wl : dl;
                nu[s] = lane == 31 ? wu : du;
                nm[s] = lane == 31 ? wm : dm;
            }
#pragma unroll
            for (int s = 0; s < NS; ++s) { lb[s] = nl[s]; ub[s] = nu[s]; mn[s] = nm[s]; }
        }
        const bool exact_row = (i % P) == 0;
        const float dl = i > 0 ? __ldg(dql + i) : 0.f, dh = i > 0 ? __ldg(dqh + i) : 0.f;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const int k = lane + 32 * s, j = i - W + k;
            if (k > kt || j < 0 || j >= L) continue;
            if (exact_row || W == 0) {
                float x[DMAX];
#pragma unroll
                for (int p = 0; p < DMAX; ++p) x[p] = p < D ? __ldg(c + (size_t)j * D + p) : 0.f;
                float lo, hi;
                exact_interval_rd<DMAX>(q + (size_t)i * D, x, D, &lo, &hi);
                lb[s] = lo;
                ub[s] = hi;
                mn[s] = k == kt ? lo : fminf(mn[s], lo);
            } else if (k < kt) {
                const float nl = fmaxf(fmaxf(__fsub_rd(lb[s], dh), __fsub_rd(dl, ub[s])), 0.f);
                ub[s] = __fadd_ru(ub[s], dh);
                lb[s] = nl;
                mn[s] = fminf(mn[s], nl);
            }
        }
        if (!exact_row && W > 0 && i + W < L) {
            // the top from its left neighbour in this row (offset kt - 1)
            const int sl = (kt - 1) >> 5, ll = (kt - 1) & 31, st = kt >> 5, lt = kt & 31;
            float nbl = INF, nbu = INF;
#pragma unroll
            for (int s = 0; s < NS; ++s)
                if (s == sl) { nbl = lb[s]; nbu = ub[s]; }
            nbl = __shfl_sync(0xffffffffu, nbl, ll);
            nbu = __shfl_sync(0xffffffffu, nbu, ll);
            if (lane == lt) {
                const int j = i + W;
                float dcl, dch;
                point_interval<DMAX>(c + (size_t)(j - 1) * D, c + (size_t)j * D, D, &dcl, &dch);
                const float tl = fmaxf(fmaxf(__fsub_rd(nbl, dch), __fsub_rd(dcl, nbu)), 0.f);
                const float tu = __fadd_ru(nbu, dch);
#pragma unroll
                for (int s = 0; s < NS; ++s)
                    if (s == st) { lb[s] = tl; ub[s] = tu; mn[s] = tl; }
            }
        }
    }
    // the columns still in the last row's window
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int k = lane + 32 * s, j = L - 1 - W + k;
        if (k <= kt && j >= 0 && j < L) acc = __fmaf_rd(mn[s], mn[s], acc);
    }
    return warp_sum_rd(acc);
}

}  // namespace tc
