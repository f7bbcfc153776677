// batch.cu -- many independent exact DTW-NN searches (uneven L, D, N, W) as one
// captured graph of persistent launches, each taking work items from a device
// queue (not in the paper: a deployment pattern).
//
//   front   items PREP (set, query): envelope, neighbour distances, LB_PC boxes;
//           LBMV (set, query tile, cand tile): one 32 x 128 LB_MV tile;
//           SEED (set, query): the seed candidates (smallest LB_MV) of the query.
//           Queued in that order; LBMV waits for its set's PREP items and SEED for
//           its set's LBMV items on device counters (bounded spins, see below).
//   dtw     the seeds' DTW: warps take entries of one set at a time off the set's
//           cursor, sets in decreasing cost, each set with its own band tile.
//   mid     items (set, query): compaction against the seeded best-so-far, gated
//           LB_PC / LB_TI; the survivors join the set's DTW work list.
//   dtw     the survivors' DTW with early abandoning, as above.
//   refine  items (set, four queries): per warp one query, double-float recompute
//           of the entries FP32 cannot separate from the best, FP64 where
//           double-float cannot either; the answer.
// The DTW runs in launches of its own: one kernel holding the LB_MV stream, the
// refine and the band DP spilled registers inside the DP loop and ran several times
// slower.  In the front launch an item only waits for items with smaller queue
// indices, which running CTAs hold and which never wait for it, so it cannot
// deadlock; each wait gives up after an iteration limit, records
// TCDTW_ERR_TIMEOUT, raises an abort flag that every CTA checks before taking an
// item, and returns.  Every step is the same computation as tcdtw_nn (same bounds,
// margins, refine), so the answers are the same exact nearest neighbours.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "api_internal.h"
#include "batch_internal.cuh"
#include "df.cuh"
#include "dtw_core.cuh"
#include "lb_device.cuh"
#include "lb_kernels.cuh"
#include "lb_rest.cuh"
#include "prep_device.cuh"

namespace tc {

// Grab the next item index of range [begin, end) for the CTA (end when aborted).
__device__ __forceinline__ int grab_item(BatchCtl *ctl, int which, int begin, int end) {
    __shared__ int s_item;
    __syncthreads();
    if (threadIdx.x == 0) s_item = *(volatile int *)&ctl->abort ? end : begin + atomicAdd(&ctl->next[which], 1);
    __syncthreads();
    return s_item;
}

__device__ __forceinline__ int ld_acquire_s32(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 spins until *cnt >= target (bounded); every thread gets the outcome.
__device__ bool batch_wait(const int *cnt, int target, long long limit, BatchCtl *ctl, int where) {
    __shared__ int ok;
    if (threadIdx.x == 0) {
        long long it = 0;
        int v = ld_acquire_s32(cnt);
        while (v < target && it < limit && !*(volatile int *)&ctl->abort) {
            __nanosleep(256);
            ++it;
            v = ld_acquire_s32(cnt);
        }
        ok = v >= target;
        if (!ok) {
            if (it >= limit) set_error(&ctl->status, TCDTW_ERR_TIMEOUT, where);
            atomicExch(&ctl->abort, 1);
        }
    }
    __syncthreads();
    const bool r = ok;
    __syncthreads();
    return r;
}

// Publish the item's writes (all threads done, then a fence) and count it.
__device__ void batch_done(int *cnt) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(cnt, 1);
}

// ------------------------------------------------------------------ PREP
__device__ void prep_item(const BatchSet &S, int q, float *smem, BatchCtl *ctl) {
    const int L = S.L, D = S.D, W = S.W;
    const int64_t E = (int64_t)L * D;
    const float *qm = S.q + (size_t)q * E;
    if (S.check_finite) {
        bool bad = false;
        for (int64_t k = threadIdx.x; k < E; k += blockDim.x) bad |= !isfinite(__ldg(qm + k));
        if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_error(&ctl->status, TCDTW_ERR_NONFINITE, 1);
    }
    // envelope, query-pair interleaved for the LB_MV stream
    for (int64_t k = threadIdx.x; k < S.ldE; k += blockDim.x) {
        float u = TC_INF, l = -TC_INF;
        if (k < E) {
            const int i = (int)(k / D), p = (int)(k % D);
            u = -TC_INF;
            l = TC_INF;
            for (int r = max(0, i - W); r <= min(L - 1, i + W); ++r) {
                const float v = __ldg(qm + (size_t)r * D + p);
                u = fmaxf(u, v);
                l = fminf(l, v);
            }
        }
        const size_t pos = (size_t)(((q >> 1) * S.ldE + k) * 2 + (q & 1));
        S.U[pos] = u;
        S.Lo[pos] = l;
        if (S.samp > 0) {  // the one-query-per-row copy the LB_MV completion reads
            S.Up[(size_t)q * S.ldE + k] = u;
            S.Lp[(size_t)q * S.ldE + k] = l;
        }
    }
    if (S.use_ti) {
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            float lo = 0.f, hi = 0.f;
            if (i > 0) {
                float sl = 0.f, sh = 0.f;
                for (int p = 0; p < D; ++p) {
                    const float x = __ldg(qm + (size_t)(i - 1) * D + p), y = __ldg(qm + (size_t)i * D + p);
                    const float dl = fmaxf(__fsub_rd(x, y), __fsub_rd(y, x)), dh = fmaxf(__fsub_ru(x, y), __fsub_ru(y, x));
                    sl = __fmaf_rd(dl, dl, sl);
                    sh = __fmaf_ru(dh, dh, sh);
                }
                lo = __fsqrt_rd(sl);
                hi = __fsqrt_ru(sh);
            }
            S.dq_lo[(size_t)q * L + i] = lo;
            S.dq_hi[(size_t)q * L + i] = hi;
        }
    }
    if (S.use_pc) {
        const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        unsigned long long *scratch = (unsigned long long *)(smem) + (size_t)warp * (kBatchSmem / 8 / 4);
        for (int g = warp; g < S.Gpc; g += nw)
            pc_boxes_group(qm, L, D, W, S.K, S.Lq, S.w, g, S.np2, scratch,
                           S.boxes + ((size_t)q * S.Gpc + g) * S.K * 2 * D, S.box_counts + (size_t)q * S.Gpc + g);
    }
}

// ------------------------------------------------------------------ compaction
// Ordered compaction of one row by the CTA: entries n with row[n] <= thr, in
// increasing n, to out_idx / out_lb; returns the count on every thread.
__device__ int compact_row(const float *__restrict__ row, int64_t N, float thr, uint32_t *__restrict__ out_idx,
                           float *__restrict__ out_lb) {
    __shared__ int wsum[32];
    __shared__ int running;
    if (threadIdx.x == 0) running = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t n0 = 0; n0 < N; n0 += blockDim.x) {
        const int64_t n = n0 + threadIdx.x;
        const float v = n < N ? row[n] : TC_INF;
        const bool keep = n < N && v < TC_INF && v <= thr;
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int before = running;
        for (int k = 0; k < warp; ++k) before += wsum[k];
        if (keep) {
            const int pos = before + __popc(bal & ((1u << lane) - 1u));
            out_idx[pos] = (uint32_t)n;
            out_lb[pos] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int k = 0; k < nw; ++k) t += wsum[k];
            running += t;
        }
        __syncthreads();
    }
    const int c = running;
    __syncthreads();
    return c;
}

// SEED: the S smallest LB_MV of the query become its seeds (their bounds in the row
// are set to +inf so that compaction skips them); the best-so-far starts at +inf.
__device__ void seed_item(const BatchSet &S, int q) {
    __shared__ uint32_t picked[kSeedSlots];
    seed_topk_row(S.lbm + (size_t)q * S.N, S.N, S.S, picked);
    if (threadIdx.x < kSeedSlots) {
        const uint32_t n = threadIdx.x < (unsigned)S.S ? picked[threadIdx.x] : 0xffffffffu;
        S.seeds[(size_t)q * kSeedSlots + threadIdx.x] = n;
    }
    if (threadIdx.x == 0) {
        int ns = 0;
        for (int k = 0; k < S.S; ++k) ns += picked[k] != 0xffffffffu;
        S.nseed[q] = ns;
        S.bsf[q] = pack_best(TC_INF, 0xffffffffu);
    }
}

__global__ void __launch_bounds__(kBatchThreads) k_batch_front(const BatchSet *__restrict__ sets,
                                                               const BatchItem *__restrict__ items, int begin,
                                                               int end, BatchCtl *ctl, long long spin_limit) {
    extern __shared__ __align__(16) float bsm[];
    for (;;) {
        const int it = grab_item(ctl, 0, begin, end);
        if (it >= end) break;
        const BatchItem item = items[it];
        if (item.kind == kItemStall) {  // waits for a counter nothing increments (self-test)
            batch_wait(&ctl->never, 1, spin_limit, ctl, it);
            continue;
        }
        const BatchSet &S = sets[item.set];
        if (item.kind == kItemPrep) {
            prep_item(S, item.a, bsm, ctl);
            batch_done(S.cnt + kCntPrep);
        } else if (item.kind == kItemMv) {
            if (!batch_wait(S.cnt + kCntPrep, S.M, spin_limit, ctl, it)) continue;
            __threadfence();
            float(*sc)[kMvRows * kMvChunk] = (float(*)[kMvRows * kMvChunk])bsm;
            float(*su)[kBatchQB * kMvChunk] = (float(*)[kBatchQB * kMvChunk])(bsm + 2 * kMvRows * kMvChunk);
            float(*sl)[kBatchQB * kMvChunk] =
                (float(*)[kBatchQB * kMvChunk])(bsm + 2 * kMvRows * kMvChunk + 2 * kBatchQB * kMvChunk);
            lb_mv_tile<kBatchQB>(S.cand, S.N, S.samp > 0 ? S.samp : (S.L * S.D + kMvChunk - 1) / kMvChunk,
                                 S.samp > 0 ? S.sstride : 1, S.L * S.D, (int64_t)S.L * S.D, S.vec4 != 0, S.U, S.Lo, S.ldE, S.M, S.lbm, S.N,
                                 (int64_t)item.b * kMvRows, item.a * kBatchQB, sc, su, sl);
            batch_done(S.cnt + kCntMv);
        } else if (item.kind == kItemSeed) {
            if (!batch_wait(S.cnt + kCntMv, S.n_qtiles * S.n_ctiles, spin_limit, ctl, it)) continue;
            __threadfence();
            seed_item(S, item.a);
        }
    }
}

// ------------------------------------------------------------------ DTW launches
// (the kernels: batch_internal.cuh, instantiated per rows-per-lane in batch_dtw_r*.cu)
cudaError_t launch_batch_dtw(int R, int dm, int grid, cudaStream_t s, const BatchSet *sets, const int *order,
                             int nsets, int phase, BatchCtl *ctl) {
    if (R == 4) return batch_dtw_launch_r4(dm, grid, s, sets, order, nsets, phase, ctl);
    if (R == 8) return batch_dtw_launch_r8(dm, grid, s, sets, order, nsets, phase, ctl);
    if (R == 16) return batch_dtw_launch_r16(dm, grid, s, sets, order, nsets, phase, ctl);
    return cudaErrorInvalidValue;
}

cudaError_t kernel_grid(const void *fn, size_t smem, int *grid) {
    if (smem > 0) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kBatchThreads, smem);
    if (e != cudaSuccess) return e;
    *grid = (occ > 0 ? occ : 1) * num_sms();
    return cudaSuccess;
}

cudaError_t batch_dtw_grid(int R, int dm, int *grid) {
    if (R == 4) return batch_dtw_grid_r4(dm, grid);
    if (R == 8) return batch_dtw_grid_r8(dm, grid);
    if (R == 16) return batch_dtw_grid_r16(dm, grid);
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ mid launch
// Compaction against the seeded best-so-far (seeds are +inf in the row), gated
// tight bounds (one warp per survivor), and the survivors' entries q*N + k appended
// to the set's work list in one reservation.
__device__ void mid_item(const BatchSet &S, int q, BatchCtl *ctl) {
    __shared__ int s_base;
    const int L = S.L, D = S.D;
    const int64_t N = S.N;
    const unsigned long long *bsf = S.bsf + q;
    const float thr = prune_threshold(ld_volatile_u64(bsf), S.rho);
    uint32_t *sv = S.surv + (size_t)q * N;
    float *slb = S.surv_lb + (size_t)q * N;
    const int cnt = compact_row(S.lbm + (size_t)q * N, N, thr, sv, slb);
    if (threadIdx.x == 0) {
        atomicAdd(&ctl->counters[4], (unsigned long long)(N - cnt - S.nseed[q]));
        s_base = atomicAdd(S.cnt + kCntList, cnt);
        S.ncnt[q] = cnt;
    }
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int pass = 0; pass < 2; ++pass) {
        if ((pass == 0 && !S.use_pc) || (pass == 1 && !S.use_ti)) continue;
        unsigned long long pruned = 0;
        for (int e = warp; e < cnt; e += nw) {
            const float cur = slb[e];
            if (!(cur < TC_INF)) continue;
            const unsigned long long key = ld_volatile_u64(bsf);
            if (cur > prune_threshold(key, S.rho)) continue;
            if (!(cur > (pass == 0 ? S.e_pc : S.e_ti) * best_dist(key))) continue;
            const float *c = S.cand + (size_t)sv[e] * L * D;
            float bound = 0.f;
            bool dropped;
            if (pass == 0) {
                const float *bx = S.boxes + (size_t)q * S.Gpc * S.K * 2 * D;
                const int32_t *bc = S.box_counts + (size_t)q * S.Gpc;
                dropped = D <= 8 ? lb_pc_pair<8>(c, bx, bc, L, D, S.K, S.w, bsf, S.rho, &bound)
                                 : lb_pc_pair<16>(c, bx, bc, L, D, S.K, S.w, bsf, S.rho, &bound);
            } else {
                const float *qa = S.q + (size_t)q * L * D;
                const float *dl = S.dq_lo + (size_t)q * L, *dh = S.dq_hi + (size_t)q * L;
                dropped = D <= 8 ? lb_ti_pair<8>(c, qa, dl, dh, L, D, S.W, S.P, bsf, S.rho, &bound)
                                 : lb_ti_pair<16>(c, qa, dl, dh, L, D, S.W, S.P, bsf, S.rho, &bound);
            }
            if (lane == 0) {
                if (dropped) { slb[e] = TC_INF; ++pruned; }
                else slb[e] = fmaxf(cur, bound);
            }
        }
        if (lane == 0 && pruned) atomicAdd(&ctl->counters[5 + pass], pruned);
    }
    __syncthreads();
    const int base = s_base;
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) S.list[base + k] = (uint32_t)(q * N + k);
}

__global__ void __launch_bounds__(kBatchThreads) k_batch_mid(const BatchSet *__restrict__ sets,
                                                             const BatchItem *__restrict__ items, int begin, int end,
                                                             BatchCtl *ctl) {
    for (;;) {
        const int it = grab_item(ctl, 1, begin, end);
        if (it >= end) break;
        const BatchItem item = items[it];
        mid_item(sets[item.set], item.a, ctl);
    }
}

// ------------------------------------------------------------------ LB_MV completion
// Items (set, candidate tile of kBatchRestTile): the completion pass of the abandoning
// LB_MV (lb_rest.cuh), against the best-so-far the seeds left; the pairs whose sample
// sum already exceeds the threshold keep it.
constexpr int kBatchRestTile = kRestTC;
constexpr int kSeed2Threads = 256;

// Second-round seeds of query q (sets whose LB_MV abandons): the S2 smallest bounds of
// the completed row go to the slots after the first round's seeds, marked pending for
// the DTW phase 2 (and set to +inf in the row, so compaction skips them).
__device__ void seed2_item(const BatchSet &S, int q) {
    __shared__ uint32_t picked[kSeedSlots];
    const int na = S.nseed[q];
    const int s2 = min(S.S2, kSeedSlots - na);
    if (s2 <= 0) return;  // (the same for every thread)
    seed_topk_row(S.lbm + (size_t)q * S.N, S.N, s2, picked);
    if (threadIdx.x < (unsigned)s2) {
        const uint32_t n = picked[threadIdx.x];
        S.seeds[(size_t)q * kSeedSlots + na + threadIdx.x] = n;
        S.seed_dtw[(size_t)q * kSeedSlots + na + threadIdx.x] = n != 0xffffffffu ? kSeedPending : TC_INF;
    }
    if (threadIdx.x == 0) {
        int ns = 0;
        for (int k = 0; k < s2; ++k) ns += picked[k] != 0xffffffffu;
        S.nseed[q] = na + ns;
    }
}

__global__ void __launch_bounds__(kSeed2Threads) k_batch_seed2(const BatchSet *__restrict__ sets,
                                                               const BatchItem *__restrict__ items, int begin) {
    const BatchItem item = items[begin + blockIdx.x];
    seed2_item(sets[item.set], item.a);
}

__global__ void __launch_bounds__(kRestCpThreads, 1) k_batch_rest(const BatchSet *__restrict__ sets,
                                                                  const BatchItem *__restrict__ items, int begin,
                                                                  int end, BatchCtl *ctl, uint32_t *lists,
                                                                  int qg_max) {
    extern __shared__ __align__(16) float rs[];
    uint32_t *list = lists + (size_t)blockIdx.x * kBatchRestTile * qg_max;
    unsigned long long terms = 0;
    LbMvRestArgs a;
    memset(&a, 0, sizeof(a));
    for (;;) {
        const int it = grab_item(ctl, 3, begin, end);
        if (it >= end) break;
        const BatchItem item = items[it];
        const BatchSet &S = sets[item.set];
        a.cand = S.cand; a.N = S.N; a.E = S.L * S.D; a.samp = S.samp; a.sstride = S.sstride; a.ldC = a.E; a.Up = S.Up; a.Lp = S.Lp;
        a.ldP = S.ldE; a.Mb = S.M; a.lb = S.lbm; a.ldLb = S.N; a.thresh = nullptr; a.bsf = S.bsf; a.rho = S.rho;
        const int qg = min(S.M, qg_max);
        for (int q0 = 0; q0 < S.M; q0 += qg)
            rest_pass_cp(a, (int64_t)item.a * kBatchRestTile, kBatchRestTile, q0, min(qg, S.M - q0), qg, S.vec4, rs,
                         list, terms);
    }
    a.terms = &ctl->counters[9];
    rest_terms_flush(a, terms);
}

// ------------------------------------------------------------------ refine launch
__device__ __noinline__ double batch_fp64(const BatchSet &S, const float *a, const float *b, const Grp &g,
                                          double *ad) {
    switch (S.Rref) {
#define TC_BR(RV) \
    case RV: return band_pass64<RV>(a, b, S.L, S.D, S.W, g, ad);
        TC_REFINE_RS(TC_BR)
#undef TC_BR
    }
    return __longlong_as_double(0x7ff0000000000000LL);
}

__device__ __noinline__ double batch_df(const BatchSet &S, const float *a, const float *b, const Grp &g) {
    switch (S.Rref) {
#define TC_BR(RV) \
    case RV: return band_pass_df<RV>(a, b, S.L, S.D, S.W, g);
        TC_REFINE_RS(TC_BR)
#undef TC_BR
    }
    return __longlong_as_double(0x7ff0000000000000LL);
}

// Refine of query q by one warp: every entry that FP32 cannot separate from the best
// gets its double-float DTW; only when that still leaves two or more inseparable
// entries (or no finite value) do those get the FP64 recompute.  Entry e < nseed is
// seed e, entry nseed + k is survivor k.
__device__ void refine_warp(const BatchSet &S, int q, double *ad, BatchCtl *ctl) {
    const int lane = threadIdx.x & 31;
    const int L = S.L, D = S.D;
    const int64_t N = S.N;
    const int nseed = __ldcg(S.nseed + q), cnt = __ldcg(S.ncnt + q);
    const int ntot = nseed + cnt;
    const float *qa = S.q + (size_t)q * L * D;
    const uint32_t *sd = S.seeds + (size_t)q * kSeedSlots, *sv = S.surv + (size_t)q * N;
    const float *sdd = S.seed_dtw + (size_t)q * kSeedSlots, *sdt = S.surv_dtw + (size_t)q * N;
    double *d64 = S.d64 + (size_t)q * (N + 8);
    const float tfin = prune_threshold(ld_volatile_u64(S.bsf + q), S.rho_ref);
    const double DINF = __longlong_as_double(0x7ff0000000000000LL);
    Grp g32 = make_grp(32);
    unsigned long long bestdf = 0x7ff0000000000000ull, refined = 0;
    // entries in chunks of 32: a ballot finds the ones to refine, the warp takes them in turn
    for (int e0 = 0; e0 < ntot; e0 += 32) {
        const int e = e0 + lane;
        const float d32 = e < ntot ? (e < nseed ? __ldcg(sdd + e) : __ldcg(sdt + (e - nseed))) : TC_INF;
        const bool want = e < ntot && d32 <= tfin;
        if (e < ntot && !want) d64[e] = DINF;
        unsigned todo = __ballot_sync(0xffffffffu, want);
        while (todo) {
            const int k = __ffs(todo) - 1;
            todo &= todo - 1;
            const int ek = e0 + k;
            const uint32_t cn = ek < nseed ? __ldcg(sd + ek) : __ldcg(sv + (ek - nseed));
            double r = batch_df(S, qa, S.cand + (size_t)cn * L * D, g32);
            r = grp_min(r, g32);
            if (lane == 0) d64[ek] = r;
            const unsigned long long rb = (unsigned long long)__double_as_longlong(r);
            bestdf = rb < bestdf ? rb : bestdf;
            ++refined;
        }
    }
    __syncwarp();
    const double thr_df = __dmul_ru(__longlong_as_double((long long)bestdf), S.kappa);
    int amb = 0;
    unsigned long long best_idx = ~0ull;
    for (int e = lane; e < ntot; e += 32) {
        const double x = d64[e];
        if (x == DINF) continue;
        if (!(x > thr_df)) ++amb;
        if ((unsigned long long)__double_as_longlong(x) == bestdf) {
            const unsigned long long cn = e < nseed ? __ldcg(sd + e) : __ldcg(sv + (e - nseed));
            best_idx = cn < best_idx ? cn : best_idx;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        amb += __shfl_xor_sync(0xffffffffu, amb, o);
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best_idx, o);
        best_idx = ob < best_idx ? ob : best_idx;
    }
    // refine entries marked +inf above were never refined; a refined entry whose
    // value is +inf (overflow) makes the query take the FP64 path
    bool need64 = amb >= 2 || !(__longlong_as_double((long long)bestdf) < DINF);
    unsigned long long best64 = 0x7ff0000000000000ull, refined64 = 0;
    if (need64) {
        best_idx = ~0ull;
        for (int e0 = 0; e0 < ntot; e0 += 32) {
            const int e = e0 + lane;
            bool want = false;
            if (e < ntot) {
                const float d32 = e < nseed ? __ldcg(sdd + e) : __ldcg(sdt + (e - nseed));
                want = d32 <= tfin && !(d64[e] > thr_df);
            }
            unsigned todo = __ballot_sync(0xffffffffu, want);
            while (todo) {
                const int k = __ffs(todo) - 1;
                todo &= todo - 1;
                const int ek = e0 + k;
                const uint32_t cn = ek < nseed ? __ldcg(sd + ek) : __ldcg(sv + (ek - nseed));
                double r = batch_fp64(S, qa, S.cand + (size_t)cn * L * D, g32, ad);
                r = grp_min(r, g32);
                const unsigned long long rb = (unsigned long long)__double_as_longlong(r);
                if (rb < best64 || (rb == best64 && cn < best_idx)) {
                    if (rb < best64) best_idx = cn;
                    best64 = rb;
                    best_idx = cn < best_idx ? cn : best_idx;
                }
                ++refined64;
            }
        }
    }
    if (lane == 0) {
        S.idx[q] = (int64_t)best_idx;
        S.dist[q] = __longlong_as_double((long long)(need64 ? best64 : bestdf));
        atomicAdd(&ctl->counters[7], refined);
        if (refined64) atomicAdd(&ctl->counters[8], refined64);
    }
}

__global__ void __launch_bounds__(kBatchThreads) k_batch_refine(const BatchSet *__restrict__ sets,
                                                                const BatchItem *__restrict__ items, int begin,
                                                                int end, BatchCtl *ctl) {
    extern __shared__ __align__(16) float bsm[];
    constexpr int kAdPerLane = (int)(kBatchSmem / 4 / 32 / sizeof(double));
    for (;;) {
        const int it = grab_item(ctl, 2, begin, end);
        if (it >= end) break;
        const BatchItem item = items[it];
        const BatchSet &S = sets[item.set];
        const int warp = threadIdx.x >> 5;
        const int qw = item.a + warp;
        if (warp < kRefinePerItem && qw < S.M) {
            double *ad = S.Rref * S.D <= kAdPerLane
                             ? (double *)bsm + (size_t)warp * 32 * kAdPerLane + (size_t)(threadIdx.x & 31) * kAdPerLane
                             : nullptr;
            refine_warp(S, qw, ad, ctl);
        }
    }
}

static_assert(2 * kMvRows * kMvChunk * 4 + 4 * kBatchQB * kMvChunk * 4 <= kBatchSmem, "LB_MV buffers");

// ------------------------------------------------------------------ host side
namespace {

// Smallest lane-group size G with G*(R+1) >= 2W+R (no overlap of a lane's virtual
// lanes), or 0.
int batch_G(int R, int W) {
    for (int g = 4; g <= 32; g *= 2)
        if (g * (R + 1) >= 2 * W + R) return g;
    return 0;
}

// The band tile of one set: the single-set tuner's fastest (tile, G) for its (L, D, W)
// -- timed on the set's own candidates, cached per shape for the process (and in the
// TCDTW_TUNE_CACHE file) -- when the batched launches compile that tile; else 8 rows
// per lane with the smallest valid G.
void choose_batch_tile(const tcdtw_dataset &d, int W, cudaStream_t s, int *R, int *G) {
    int tile = -1, g = 0;
    if (autotune_nn_tile(d.cand, d.N, d.L, d.D, W, s, &tile, &g) && tile >= 0 && kTiles[tile].DMAX == d.D &&
        batch_tile_compiled(kTiles[tile].R, d.D) && g * (kTiles[tile].R + 1) >= 2 * W + kTiles[tile].R) {
        *R = kTiles[tile].R;
        *G = g;
        return;
    }
    *R = 8;
    *G = batch_G(8, W);
}

// A workspace arena and a captured graph per batch description.
struct BatchPlan {
    std::vector<tcdtw_dataset> key;
    tcdtw_opts opts;
    void *arena = nullptr;
    BatchSet *d_sets = nullptr;
    BatchItem *d_items = nullptr;
    BatchCtl *d_ctl = nullptr;
    int *d_counts = nullptr, *d_order = nullptr;
    int n_sets = 0;
    // item ranges: front [0, front_end), LB_MV completion [front_end, rest_end), second-
    // round seeds [rest_end, seed2_end), mid [seed2_end, mid_end), refine [mid_end, n_items)
    int front_end = 0, rest_end = 0, seed2_end = 0, mid_end = 0, n_items = 0;
    int grid_front = 0, grid_mid = 0, grid_refine = 0, grid_rest = 0;
    int rest_qg = 0;              // queries per completion pass (0: no set abandons)
    uint32_t *d_rest_lists = nullptr;
    uint64_t dense_terms = 0;     // LB_MV terms of the front's tiles per run
    // DTW launches: per tile class present, its sets d_order[off, off + n) and grid
    struct DtwClass { int R, dm, off, n, grid; };
    std::vector<DtwClass> classes;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
    unsigned long long last_use = 0;
    // the tile classes of a phase are independent (different sets): they run on side
    // streams forked from and joined back to the caller's stream, so that one class's
    // tail (its last, longest pairs on a few warps) overlaps the others' work
    static constexpr int kSide = 4;
    cudaStream_t side[kSide] = {};
    static constexpr int kPhases = 3;  // seeds, survivors, second-round seeds
    cudaEvent_t ev_fork[kPhases] = {}, ev_join[kPhases][kSide] = {};
};
std::vector<BatchPlan *> g_plans;
std::mutex g_plans_mu;
unsigned long long g_plan_clock = 0;

void free_plan(BatchPlan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    for (int k = 0; k < BatchPlan::kSide; ++k) {
        if (p->side[k]) cudaStreamDestroy(p->side[k]);
        for (int ph = 0; ph < BatchPlan::kPhases; ++ph)
            if (p->ev_join[ph][k]) cudaEventDestroy(p->ev_join[ph][k]);
    }
    for (int ph = 0; ph < BatchPlan::kPhases; ++ph)
        if (p->ev_fork[ph]) cudaEventDestroy(p->ev_fork[ph]);
    cudaFree(p->arena);
    delete p;
}

bool same_key(const BatchPlan *p, const tcdtw_dataset *sets, int n, const tcdtw_opts &o) {
    if ((int)p->key.size() != n || memcmp(&p->opts, &o, sizeof(o)) != 0) return false;
    return memcmp(p->key.data(), sets, sizeof(tcdtw_dataset) * n) == 0;
}

bool graph_path_ok(const tcdtw_dataset &d, const tcdtw_opts &o) {
    const int W = d.W > d.L - 1 ? d.L - 1 : d.W;
    return d.D <= kBatchMaxD && batch_G(8, W) > 0 && refine_rows_for(W) > 0 && d.M <= 65535 &&
           o.seed_s <= kSeedSlots && (double)d.M * (double)d.N < 4.29e9;
}

template <typename T>
T *carve(char *&p, size_t n) {
    p = (char *)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    T *r = (T *)p;
    p += sizeof(T) * (n ? n : 1);
    return r;
}
template <typename T>
size_t carve_bytes(size_t n) { return sizeof(T) * (n ? n : 1) + 256; }

int build_plan(const tcdtw_dataset *sets, const std::vector<int> &mk, const tcdtw_opts &o, cudaStream_t s,
               BatchPlan **out) {
    BatchPlan *p = new BatchPlan();
    std::vector<BatchSet> hs;
    std::vector<double> cost;
    size_t bytes = 0;
    for (int k : mk) {
        const tcdtw_dataset &d = sets[k];
        BatchSet b;
        memset(&b, 0, sizeof(b));
        b.cand = d.cand; b.q = d.q; b.idx = d.idx; b.dist = d.dist;
        b.N = d.N; b.L = d.L; b.D = d.D; b.W = d.W > d.L - 1 ? d.L - 1 : d.W; b.K = d.K; b.M = (int)d.M;
        choose_batch_tile(d, b.W, s, &b.R, &b.G);
        b.dcase = d.D;
        b.Rref = refine_rows_for(b.W);
        b.S = (int)(o.seed_s < d.N ? o.seed_s : d.N);
        b.check_finite = o.check_finite != 0;
        b.Lq = o.Lq; b.w = o.w; b.P = o.P; b.e_pc = o.e_pc; b.e_ti = o.e_ti;
        b.use_ti = o.use_ti && !o.no_prune;
        b.use_pc = o.use_pc && !o.no_prune && pc_key_fits(o.Lq, d.D);
        b.Gpc = (d.L + o.w - 1) / o.w;
        if (b.use_pc) {
            int np2 = 0;
            const size_t need = pc_boxes_smem(d.L, d.D, b.W, d.K, o.w, &np2);
            if (need > kBatchSmem / 4) b.use_pc = 0;
            b.np2 = np2;
        }
        b.vec4 = lb_mv_vec4(d.cand, d.L * d.D);
        b.rho_ref = prune_rho(d.L, d.D);
        b.kappa = refine_kappa(d.L, d.D);
        b.rho = o.no_prune ? INFINITY : b.rho_ref;
        b.ldE = ((int64_t)d.L * d.D + 31) / 32 * 32;
        b.n_qtiles = (int)((d.M + kBatchQB - 1) / kBatchQB);
        b.n_ctiles = (int)((d.N + kMvRows - 1) / kMvRows);
        // LB_MV with early abandoning for sets of at least 32 queries (as tcdtw_nn)
        b.samp = (o.mv_abandon && !o.no_prune && d.M >= 32) ? lb_mv_sample(d.L * d.D, &b.sstride) : 0;
        b.S2 = b.samp > 0 ? (int)std::max<int64_t>(0, std::min<int64_t>(std::min(b.S, kSeedSlots - b.S), d.N - b.S)) : 0;
        p->dense_terms += (uint64_t)d.M * d.N * (uint64_t)(b.samp > 0 ? 32 * b.samp : d.L * d.D);
        const size_t Mp = (size_t)(d.M + 1) / 2 * 2, M = (size_t)d.M, N = (size_t)d.N;
        bytes += 2 * carve_bytes<float>(Mp * b.ldE) + 2 * carve_bytes<float>(M * d.L);
        if (b.samp > 0) bytes += 2 * carve_bytes<float>(M * b.ldE);
        if (b.use_pc) bytes += carve_bytes<float>(M * b.Gpc * d.K * 2 * d.D) + carve_bytes<int32_t>(M * b.Gpc);
        bytes += 3 * carve_bytes<float>(M * N) + 2 * carve_bytes<uint32_t>(M * N) + carve_bytes<double>(M * (N + 8));
        bytes += carve_bytes<uint32_t>(M * kSeedSlots) + carve_bytes<float>(M * kSeedSlots);
        bytes += carve_bytes<unsigned long long>(M) + 2 * carve_bytes<int>(M);
        hs.push_back(b);
        cost.push_back((double)N * d.L * d.D * M + (double)M * N * d.L * (2.0 * b.W + 1) * 0.05);
    }
    const int ns = (int)hs.size();
    // items: front (PREP, LBMV, SEED), mid, refine; each kind in decreasing set cost
    std::vector<int> order(ns);
    for (int k = 0; k < ns; ++k) order[k] = k;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    // DTW order: tile classes (R, D) by total cost, the sets of a class by cost
    std::vector<std::pair<int, int>> tiles;  // distinct (R, D)
    std::vector<double> class_cost;
    for (int k = 0; k < ns; ++k) {
        const std::pair<int, int> t{hs[k].R, hs[k].D};
        size_t c = std::find(tiles.begin(), tiles.end(), t) - tiles.begin();
        if (c == tiles.size()) { tiles.push_back(t); class_cost.push_back(0.0); }
        class_cost[c] += cost[k];
    }
    std::vector<int> cls(tiles.size());
    for (size_t c = 0; c < tiles.size(); ++c) cls[c] = (int)c;
    std::sort(cls.begin(), cls.end(), [&](int a, int b) { return class_cost[a] > class_cost[b]; });
    std::vector<int> dtw_order;
    for (int c : cls) {
        BatchPlan::DtwClass dc{tiles[c].first, tiles[c].second, (int)dtw_order.size(), 0, 0};
        for (int k : order)
            if (hs[k].R == dc.R && hs[k].D == dc.dm) dtw_order.push_back(k);
        dc.n = (int)dtw_order.size() - dc.off;
        const cudaError_t e = batch_dtw_grid(dc.R, dc.dm, &dc.grid);
        if (e != cudaSuccess) {
            delete p;
            return cuda_err(e);
        }
        p->classes.push_back(dc);
    }
    std::vector<BatchItem> items;
    for (int k : order)
        for (int m = 0; m < hs[k].M; ++m) items.push_back({kItemPrep, k, m, 0});
    for (int k : order)
        for (int ct = 0; ct < hs[k].n_ctiles; ++ct)
            for (int qt = 0; qt < hs[k].n_qtiles; ++qt) items.push_back({kItemMv, k, qt, ct});
    for (int k : order)
        for (int m = 0; m < hs[k].M; ++m) items.push_back({kItemSeed, k, m, 0});
    p->front_end = (int)items.size();
    for (int k : order)
        if (hs[k].samp > 0) {
            p->rest_qg = std::max(p->rest_qg, std::min(hs[k].M, kRestQG));
            for (int64_t t = 0; t * kBatchRestTile < hs[k].N; ++t) items.push_back({kItemRest, k, (int)t, 0});
        }
    p->rest_end = (int)items.size();
    for (int k : order)
        if (hs[k].S2 > 0)
            for (int m = 0; m < hs[k].M; ++m) items.push_back({kItemSeed2, k, m, 0});
    p->seed2_end = (int)items.size();
    for (int k : order)
        for (int m = 0; m < hs[k].M; ++m) items.push_back({kItemMid, k, m, 0});
    p->mid_end = (int)items.size();
    for (int k : order)
        for (int m = 0; m < hs[k].M; m += kRefinePerItem) items.push_back({kItemRefine, k, m, 0});
    p->n_items = (int)items.size();
    bytes += carve_bytes<BatchSet>(ns) + carve_bytes<BatchItem>(items.size()) + carve_bytes<BatchCtl>(1) +
             carve_bytes<int>((size_t)kCntPerSet * ns) + carve_bytes<int>(ns);
    const int rest_items = p->rest_end - p->front_end;
    p->grid_rest = std::max(1, std::min(rest_items, num_sms()));  // one CTA per SM (shared memory, registers)
    if (p->rest_qg > 0) bytes += carve_bytes<uint32_t>((size_t)p->grid_rest * kBatchRestTile * p->rest_qg);
    if (dev_malloc((void **)&p->arena, bytes) != cudaSuccess) {
        delete p;
        return TCDTW_ERR_NOMEM;
    }
    char *c = (char *)p->arena;
    p->d_sets = carve<BatchSet>(c, ns);
    p->d_items = carve<BatchItem>(c, items.size());
    p->d_ctl = carve<BatchCtl>(c, 1);
    p->d_counts = carve<int>(c, (size_t)kCntPerSet * ns);
    p->d_order = carve<int>(c, ns);
    if (p->rest_qg > 0) p->d_rest_lists = carve<uint32_t>(c, (size_t)p->grid_rest * kBatchRestTile * p->rest_qg);
    for (int k = 0; k < ns; ++k) {
        BatchSet &b = hs[k];
        const size_t Mp = (size_t)(b.M + 1) / 2 * 2, M = (size_t)b.M, N = (size_t)b.N;
        b.U = carve<float>(c, Mp * b.ldE);
        b.Lo = carve<float>(c, Mp * b.ldE);
        b.dq_lo = carve<float>(c, M * b.L);
        b.dq_hi = carve<float>(c, M * b.L);
        if (b.samp > 0) {
            b.Up = carve<float>(c, M * b.ldE);
            b.Lp = carve<float>(c, M * b.ldE);
        }
        if (b.use_pc) {
            b.boxes = carve<float>(c, M * b.Gpc * b.K * 2 * b.D);
            b.box_counts = carve<int32_t>(c, M * b.Gpc);
        }
        b.lbm = carve<float>(c, M * N);
        b.surv_lb = carve<float>(c, M * N);
        b.surv_dtw = carve<float>(c, M * N);
        b.surv = carve<uint32_t>(c, M * N);
        b.list = carve<uint32_t>(c, M * N);
        b.d64 = carve<double>(c, M * (N + 8));
        b.seeds = carve<uint32_t>(c, M * kSeedSlots);
        b.seed_dtw = carve<float>(c, M * kSeedSlots);
        b.bsf = carve<unsigned long long>(c, M);
        b.nseed = carve<int>(c, M);
        b.ncnt = carve<int>(c, M);
        b.cnt = p->d_counts + (size_t)kCntPerSet * k;
    }
    if ((size_t)(c - (char *)p->arena) > bytes) {  // the carving must stay inside the arena
        free_plan(p);
        return TCDTW_ERR_INVALID;
    }
    cudaError_t e = cudaMemcpyAsync(p->d_sets, hs.data(), sizeof(BatchSet) * ns, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_order, dtw_order.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int k = 0; k < BatchPlan::kSide && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&p->side[k], cudaStreamNonBlocking);
        for (int ph = 0; ph < BatchPlan::kPhases && e == cudaSuccess; ++ph)
            e = cudaEventCreateWithFlags(&p->ev_join[ph][k], cudaEventDisableTiming);
    }
    for (int ph = 0; ph < BatchPlan::kPhases && e == cudaSuccess; ++ph)
        e = cudaEventCreateWithFlags(&p->ev_fork[ph], cudaEventDisableTiming);
    if (e == cudaSuccess) e = kernel_grid((const void *)k_batch_front, kBatchSmem, &p->grid_front);
    if (e == cudaSuccess) e = kernel_grid((const void *)k_batch_mid, 0, &p->grid_mid);
    if (e == cudaSuccess && p->rest_qg > 0)
        e = cudaFuncSetAttribute(k_batch_rest, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)rest_cp_smem(kBatchRestTile, p->rest_qg));
    if (e == cudaSuccess) e = kernel_grid((const void *)k_batch_refine, kBatchSmem, &p->grid_refine);
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_err(e);
    }
    p->n_sets = ns;
    p->grid_front = std::max(1, std::min(p->grid_front, p->front_end));
    p->grid_mid = std::max(1, std::min(p->grid_mid, p->mid_end - p->seed2_end));
    p->grid_refine = std::max(1, std::min(p->grid_refine, p->n_items - p->mid_end));
    *out = p;
    return TCDTW_OK;
}

int kernels_per_run(const BatchPlan *p) {
    const int nc = (int)p->classes.size();
    const int seed2 = p->seed2_end > p->rest_end ? 1 + nc : 0;
    return 3 + (p->rest_qg > 0 ? 1 : 0) + seed2 + 2 * nc;
}

// One DTW phase: the classes (largest first) round robin over the side streams, each
// side stream ordered after the work already on s and s after all of them.
cudaError_t run_dtw_classes(BatchPlan *p, cudaStream_t s, int phase) {
    const int nc = (int)p->classes.size();
    if (nc == 1) {
        const auto &c = p->classes[0];
        return launch_batch_dtw(c.R, c.dm, c.grid, s, p->d_sets, p->d_order + c.off, c.n, phase, p->d_ctl);
    }
    const int ns = nc < BatchPlan::kSide ? nc : BatchPlan::kSide;
    cudaError_t e = cudaEventRecord(p->ev_fork[phase], s);
    for (int k = 0; k < ns && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(p->side[k], p->ev_fork[phase], 0);
    for (int i = 0; i < nc && e == cudaSuccess; ++i) {
        const auto &c = p->classes[i];
        e = launch_batch_dtw(c.R, c.dm, c.grid, p->side[i % ns], p->d_sets, p->d_order + c.off, c.n, phase,
                             p->d_ctl);
    }
    for (int k = 0; k < ns && e == cudaSuccess; ++k) {
        e = cudaEventRecord(p->ev_join[phase][k], p->side[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_join[phase][k], 0);
    }
    return e;
}

cudaError_t enqueue_plan(BatchPlan *p, cudaStream_t s, long long spin_limit) {
    cudaError_t e = cudaMemsetAsync(p->d_ctl, 0, sizeof(BatchCtl), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_counts, 0, sizeof(int) * kCntPerSet * p->n_sets, s);
    if (e != cudaSuccess) return e;
    k_batch_front<<<p->grid_front, kBatchThreads, kBatchSmem, s>>>(p->d_sets, p->d_items, 0, p->front_end, p->d_ctl,
                                                                   spin_limit);
    if ((e = run_dtw_classes(p, s, 0)) != cudaSuccess) return e;
    if (p->rest_qg > 0)
        k_batch_rest<<<p->grid_rest, kRestCpThreads, rest_cp_smem(kBatchRestTile, p->rest_qg), s>>>(
            p->d_sets, p->d_items, p->front_end, p->rest_end, p->d_ctl, p->d_rest_lists, p->rest_qg);
    if (p->seed2_end > p->rest_end) {  // second-round seeds from the completed bounds, and their DTW
        k_batch_seed2<<<p->seed2_end - p->rest_end, kSeed2Threads, 0, s>>>(p->d_sets, p->d_items, p->rest_end);
        if ((e = run_dtw_classes(p, s, 2)) != cudaSuccess) return e;
    }
    k_batch_mid<<<p->grid_mid, kBatchThreads, 0, s>>>(p->d_sets, p->d_items, p->seed2_end, p->mid_end, p->d_ctl);
    if ((e = run_dtw_classes(p, s, 1)) != cudaSuccess) return e;
    k_batch_refine<<<p->grid_refine, kBatchThreads, kBatchSmem, s>>>(p->d_sets, p->d_items, p->mid_end, p->n_items,
                                                                     p->d_ctl);
    note_launches(kernels_per_run(p));
    return cudaGetLastError();
}

}  // namespace

}  // namespace tc

using namespace tc;

extern "C" {

int tcdtw_batch_nn(const tcdtw_dataset *sets, int32_t nsets, const tcdtw_opts *opts, tcdtw_stats *stats,
                   void *stream) {
    if (nsets < 0 || (nsets > 0 && !sets)) return TCDTW_ERR_INVALID;
    if (stats) memset(stats, 0, sizeof(*stats));
    if (nsets == 0) return TCDTW_OK;
    tcdtw_opts o;
    if (opts) o = *opts; else tcdtw_default_opts(&o);
    if (o.P < 1 || o.Lq < 1 || o.w < 1 || o.seed_s < 1 || o.seed_s > 8) return TCDTW_ERR_INVALID;
    o.use_rev = 0;  // the candidate-side bound needs per-set candidate envelopes: not batched
    o.ti_top = 1;   // the batched cascade evaluates LB_TI in its TIP_TOP form
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int> mk, other;
    for (int32_t k = 0; k < nsets; ++k) {
        const tcdtw_dataset &d = sets[k];
        if (d.N < 1 || d.L < 1 || d.D < 1 || d.W < 0 || d.K < 1 || d.M < 0) return TCDTW_ERR_INVALID;
        if (!d.cand || (d.M > 0 && (!d.q || !d.idx || !d.dist))) return TCDTW_ERR_INVALID;
        if (d.D > TCDTW_MAX_D) return TCDTW_ERR_UNSUPPORTED;
        if (d.M == 0) continue;
        (graph_path_ok(d, o) ? mk : other).push_back(k);
    }
    uint64_t pairs = 0;
    if (!mk.empty()) {
        std::vector<tcdtw_dataset> key;
        for (int k : mk) key.push_back(sets[k]);
        BatchPlan *plan = nullptr;
        {
            std::lock_guard<std::mutex> lock(g_plans_mu);
            for (BatchPlan *p : g_plans)
                if (same_key(p, key.data(), (int)key.size(), o)) plan = p;
        }
        if (!plan) {
            int rc = build_plan(sets, mk, o, s, &plan);
            if (rc) return rc;
            if (o.check_finite) {
                // candidates are scanned once, when the batch is first seen (as tcdtw_build
                // does); the queries are scanned by every run (PREP items)
                cudaError_t e = cudaMemsetAsync(plan->d_ctl, 0, sizeof(BatchCtl), s);
                for (size_t i = 0; i < mk.size() && e == cudaSuccess; ++i) {
                    const tcdtw_dataset &d = sets[mk[i]];
                    e = launch_check_finite(d.cand, d.N * (int64_t)d.L * d.D, &plan->d_ctl->status, 0, s);
                }
                DevStatus st{0, 0};
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e == cudaSuccess) e = cudaMemcpy(&st, &plan->d_ctl->status, sizeof(st), cudaMemcpyDeviceToHost);
                if (e != cudaSuccess || st.code) {
                    free_plan(plan);
                    return e != cudaSuccess ? cuda_err(e) : st.code;
                }
            }
            plan->key = key;
            plan->opts = o;
            std::lock_guard<std::mutex> lock(g_plans_mu);
            if (g_plans.size() >= 4) {
                auto lru = std::min_element(g_plans.begin(), g_plans.end(),
                                            [](BatchPlan *a, BatchPlan *b) { return a->last_use < b->last_use; });
                free_plan(*lru);
                g_plans.erase(lru);
            }
            g_plans.push_back(plan);
        }
        plan->last_use = ++g_plan_clock;
        cudaError_t e = cudaSuccess;
        if (!o.use_graph) {
            e = enqueue_plan(plan, s, kSpinLimit);
        } else if (plan->launches == 0) {
            e = enqueue_plan(plan, s, kSpinLimit);  // first use runs eagerly
        } else {
            if (!plan->exec) {
                cudaStream_t cs;
                e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t run = enqueue_plan(plan, cs, kSpinLimit);
                    cudaGraph_t graph = nullptr;
                    e = cudaStreamEndCapture(cs, &graph);
                    if (run != cudaSuccess) e = run;
                    if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->exec, graph, 0);
                    if (graph) cudaGraphDestroy(graph);
                    note_launches(-kernels_per_run(plan));  // captured, not launched
                }
                cudaStreamDestroy(cs);
            }
            if (e == cudaSuccess) {
                note_launches(kernels_per_run(plan));
                e = cudaGraphLaunch(plan->exec, s);
            }
        }
        ++plan->launches;
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_err(e);
        BatchCtl ctl;
        e = cudaMemcpy(&ctl, plan->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_err(e);
        if (ctl.status.code) return ctl.status.code;
        if (stats) {
            stats->dtw_started += ctl.counters[0];
            stats->dtw_abandoned += ctl.counters[1];
            stats->cells += ctl.counters[2];
            stats->pruned_mv += ctl.counters[3] + ctl.counters[4];
            stats->pruned_pc += ctl.counters[5];
            stats->pruned_ti += ctl.counters[6];
            stats->refined += ctl.counters[7];
            stats->refined64 += ctl.counters[8];
            stats->mv_terms += plan->dense_terms + ctl.counters[9];
        }
        for (int k : mk) pairs += (uint64_t)sets[k].M * (uint64_t)sets[k].N;
    }
    // shapes outside the graph path's tile family: one index per set
    for (int k : other) {
        const tcdtw_dataset &d = sets[k];
        tcdtw_index *x = nullptr;
        int rc = tcdtw_build(d.cand, d.N, d.L, d.D, d.W, d.K, &o, stream, &x);
        if (rc) return rc;
        tcdtw_stats st;
        rc = tcdtw_nn(x, d.q, d.M, d.idx, d.dist, stats ? &st : nullptr, stream);
        tcdtw_free(x);
        if (rc) return rc;
        if (stats) {
            stats->pruned_mv += st.pruned_mv; stats->pruned_pc += st.pruned_pc; stats->pruned_ti += st.pruned_ti;
            stats->dtw_started += st.dtw_started; stats->dtw_abandoned += st.dtw_abandoned;
            stats->cells += st.cells; stats->refined += st.refined; stats->refined64 += st.refined64;
            stats->mv_terms += st.mv_terms;
        }
        pairs += (uint64_t)d.M * (uint64_t)d.N;
    }
    if (stats) stats->pairs = pairs;
    return TCDTW_OK;
}

int tcdtw_batch_tiles(const tcdtw_dataset *sets, int32_t nsets, const tcdtw_opts *opts, int32_t *R, int32_t *G,
                      void *stream) {
    if (nsets < 0 || (nsets > 0 && (!sets || !R || !G))) return TCDTW_ERR_INVALID;
    tcdtw_opts o;
    if (opts) o = *opts; else tcdtw_default_opts(&o);
    for (int32_t k = 0; k < nsets; ++k) {
        const tcdtw_dataset &d = sets[k];
        if (d.N < 1 || d.L < 1 || d.D < 1 || d.W < 0 || d.K < 1 || d.M < 0 || !d.cand) return TCDTW_ERR_INVALID;
        R[k] = G[k] = 0;
        if (d.M == 0 || !graph_path_ok(d, o)) continue;
        choose_batch_tile(d, d.W > d.L - 1 ? d.L - 1 : d.W, (cudaStream_t)stream, &R[k], &G[k]);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TCDTW_OK : cuda_err(e);
}

// Free every cached batch sequence (graph and workspace); the next tcdtw_batch_nn
// call builds its sequence again.
int tcdtw_batch_release(void) {
    std::lock_guard<std::mutex> lock(g_plans_mu);
    const cudaError_t e = cudaDeviceSynchronize();  // a cached graph may still be running
    for (BatchPlan *p : g_plans) free_plan(p);
    g_plans.clear();
    return e == cudaSuccess ? TCDTW_OK : cuda_err(e);
}

// Self-test of the device-side wait limit: one front launch whose only item
// waits for a counter that nothing increments; the launch must end by itself with
// TCDTW_ERR_TIMEOUT after ~spin_limit sleeps, leaving the context usable.
int tcdtw_batch_selftest_timeout(int64_t spin_limit, void *stream) {
    if (spin_limit < 1) return TCDTW_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    BatchItem item{kItemStall, 0, 0, 0};
    BatchItem *d_item = nullptr;
    BatchCtl *d_ctl = nullptr;
    BatchSet *d_set = nullptr;
    cudaError_t e = dev_malloc((void **)&d_item, sizeof(item));
    if (e == cudaSuccess) e = dev_malloc((void **)&d_set, sizeof(BatchSet));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_set, 0, sizeof(BatchSet), s);
    if (e == cudaSuccess) e = dev_malloc((void **)&d_ctl, sizeof(BatchCtl));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_item, &item, sizeof(item), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ctl, 0, sizeof(BatchCtl), s);
    int grid = 0;
    if (e == cudaSuccess) e = kernel_grid((const void *)k_batch_front, kBatchSmem, &grid);
    if (e == cudaSuccess) {
        k_batch_front<<<1, kBatchThreads, kBatchSmem, s>>>(d_set, d_item, 0, 1, d_ctl, (long long)spin_limit);
        note_launch();
        e = cudaGetLastError();
    }
    BatchCtl ctl;
    memset(&ctl, 0, sizeof(ctl));
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&ctl, d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost);
    cudaFree(d_item);
    cudaFree(d_ctl);
    cudaFree(d_set);
    if (e != cudaSuccess) return cuda_err(e);
    return ctl.status.code;
}

}  // extern "C"
