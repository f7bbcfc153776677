// batch.cu -- many independent exact DTW-NN searches (uneven L, D, N, W) in one
// persistent launch off a device work queue (not in the paper: a deployment pattern).
//
// The launch keeps one CTA (4 warps) per resident slot; each CTA repeatedly takes the
// next item of an ordered queue:
//   PREP   (set, query)               envelope, neighbour distances, LB_PC boxes
//   LBMV   (set, query tile, cand tile) one 32-query x 128-candidate LB_MV tile
//   SEARCH (set, query)               seeds, their DTW, compaction, gated LB_PC/LB_TI,
//                                     DTW of the survivors, FP64 refine, the answer
// Items are queued in that order, so an item only ever waits for items with smaller
// indices; an item is taken only by a running CTA, hence the items it waits for are
// held by running CTAs that do not wait for it: the queue cannot deadlock.  The waits
// (LBMV for all PREP of its set, SEARCH for all LBMV of its set) spin on counters with
// an iteration limit; on expiry the launch records TCDTW_ERR_TIMEOUT, raises an abort
// flag that every CTA checks before taking an item, and returns.  Every step is the
// same computation as tcdtw_nn (same bounds, margins, FP64 refine), so the answers
// are the same exact nearest neighbours.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "api_internal.h"
#include "dtw_core.cuh"
#include "lb_device.cuh"
#include "lb_kernels.cuh"
#include "prep_device.cuh"

namespace tc {

constexpr int kBatchR = 8;          // rows per lane of the batched DTW
constexpr int kBatchMaxD = 12;      // dimensions the megakernel handles (D <= 8 exact, 9..12 padded to 12)
constexpr int kBatchThreads = 128;  // 4 warps per CTA
constexpr int kBatchQB = 32;        // queries per LB_MV tile
constexpr long long kSpinLimit = 4000000;  // ~1 s of 256 ns sleeps
constexpr size_t kBatchSmem = 48 * 1024;   // LB_MV double buffers / DTW staging / box scratch

struct BatchSet {
    const float *cand, *q;
    int64_t *idx;
    double *dist;
    int64_t N;
    int L, D, W, K, M;
    int G, Rref, S;
    int use_pc, use_ti, Lq, w, P, Gpc, np2, vec4, check_finite;
    float e_pc, e_ti, rho, rho_ref;
    int64_t ldE;
    int n_qtiles, n_ctiles;
    float *U, *Lo, *dq_lo, *dq_hi, *boxes;
    int32_t *box_counts;
    float *lbm, *surv_lb, *surv_dtw, *seed_dtw;
    uint32_t *surv;
    double *d64;
    int *prep_done, *mv_done;
};

enum : int { kItemPrep = 0, kItemMv = 1, kItemSearch = 2, kItemStall = 3 };
struct BatchItem {
    int kind, set, a, b;
};

struct BatchCtl {
    int next;
    int abort;
    int never;  // stays 0: the self-test waits on it
    int pad;
    DevStatus status;
    unsigned long long counters[8];  // started, abandoned, cells, pruned at DTW, pruned MV, PC, TI, refined
};

__device__ __forceinline__ int ld_acquire_s32(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 spins until *cnt >= target (bounded); every thread gets the verdict.
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

// ------------------------------------------------------------------ SEARCH pieces
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

// DTW of the candidates list[0..n) against query q, warp lockstep batches (one pair
// per group of S.G lanes), abandoning against and lowering the CTA's best-so-far.
template <int DM>
__device__ __noinline__ void batch_dtw_list(const BatchSet &S, int q, const uint32_t *list, const float *lbl, int n, float *out,
                               unsigned long long *bsf, int *cursor, float *stage, BatchCtl *ctl) {
    Grp g = make_grp(S.G);
    g.mask = 0xffffffffu;
    const int gpw = 32 / S.G;
    const int L = S.L, D = S.D, W = S.W;
    const int nv = (L + kBatchR - 1) / kBatchR;
    const float *qa = S.q + (size_t)q * L * D;
    unsigned long long started = 0, aband = 0, ncells = 0, pruned = 0;
    for (;;) {
        int base = 0;
        if ((threadIdx.x & 31) == 0) base = atomicAdd(cursor, gpw);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n) break;
        const int e = base + (threadIdx.x & 31) / S.G;
        bool live = e < n;
        const uint32_t cn = live ? list[e] : 0u;
        if (live) {
            const float lbe = lbl ? lbl[e] : 0.f;
            const float thr = prune_threshold(ld_volatile_u64(bsf), S.rho);
            if (!(lbe <= thr) || lbe == TC_INF) {
                if (g.lig == 0 && lbe != TC_INF) ++pruned;
                live = false;
            }
        }
        NnHooks h;
        h.bsf = bsf;
        h.rho = S.rho;
        bool ab = false;
        long long cells = 0;
        float r = band_pass<kBatchR, DM>(qa, S.cand + (size_t)cn * L * D, L, D, W, 0, nv, g, h, live, &ab, &cells,
                                         stage);
        r = grp_min(r, g);
        long long cs = cells;
        for (int o = S.G >> 1; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
        if (e < n && g.lig == 0) {
            if (!live) {
                out[e] = TC_INF;
            } else {
                ++started;
                ncells += (unsigned long long)cs;
                if (ab) {
                    ++aband;
                    out[e] = TC_INF;
                } else {
                    out[e] = r;
                    atomicMin(bsf, pack_best(r, cn));
                }
            }
        }
    }
    if (g.lig == 0 && (started | pruned)) {
        atomicAdd(&ctl->counters[0], started);
        atomicAdd(&ctl->counters[1], aband);
        atomicAdd(&ctl->counters[2], ncells);
        atomicAdd(&ctl->counters[3], pruned);
    }
}

__device__ void batch_dtw_dispatch(const BatchSet &S, int q, const uint32_t *list, const float *lbl, int n,
                                   float *out, unsigned long long *bsf, int *cursor, float *stage, BatchCtl *ctl) {
    switch (S.D <= 8 ? S.D : 12) {
#define TC_BD(DMV) \
    case DMV: batch_dtw_list<DMV>(S, q, list, lbl, n, out, bsf, cursor, stage, ctl); break;
        TC_BD(1) TC_BD(2) TC_BD(3) TC_BD(4) TC_BD(5) TC_BD(6) TC_BD(7) TC_BD(8) TC_BD(12)
#undef TC_BD
        default: break;
    }
}

__device__ __noinline__ double batch_fp64(const BatchSet &S, const float *a, const float *b, const Grp &g) {
    switch (S.Rref) {
#define TC_BR(RV) \
    case RV: return band_pass64<RV>(a, b, S.L, S.D, S.W, g);
        TC_REFINE_RS(TC_BR)
#undef TC_BR
    }
    return __longlong_as_double(0x7ff0000000000000LL);
}

__device__ void search_item(const BatchSet &S, int q, float *smem, BatchCtl *ctl) {
    __shared__ uint32_t seeds[8];
    __shared__ float seed_dtw[8];
    __shared__ unsigned long long bsf, best64, best_idx;
    __shared__ int cursor;
    const int L = S.L, D = S.D;
    const int64_t N = S.N;
    float *row = S.lbm + (size_t)q * N;
    float *stage = smem + (size_t)threadIdx.x * kBatchR * kBatchMaxD;
    if (threadIdx.x == 0) {
        bsf = pack_best(TC_INF, 0xffffffffu);
        best64 = 0x7ff0000000000000ull;
        best_idx = ~0ull;
        cursor = 0;
    }
    // seeds and their DTW
    seed_topk_row(row, N, S.S, seeds);
    int nseed = 0;
    for (int k = 0; k < S.S; ++k) nseed += seeds[k] != 0xffffffffu;
    batch_dtw_dispatch(S, q, seeds, nullptr, nseed, seed_dtw, &bsf, &cursor, stage, ctl);
    __syncthreads();
    // compaction against the seeded best-so-far (seeds are +inf in the row now)
    const float thr = prune_threshold(bsf, S.rho);
    uint32_t *sv = S.surv + (size_t)q * N;
    float *slb = S.surv_lb + (size_t)q * N, *sdt = S.surv_dtw + (size_t)q * N;
    const int cnt = compact_row(row, N, thr, sv, slb);
    if (threadIdx.x == 0) atomicAdd(&ctl->counters[4], (unsigned long long)(N - cnt - nseed));
    // gated tight bounds, one warp per survivor
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int pass = 0; pass < 2; ++pass) {
        if ((pass == 0 && !S.use_pc) || (pass == 1 && !S.use_ti)) continue;
        unsigned long long pruned = 0;
        for (int e = warp; e < cnt; e += nw) {
            const float cur = slb[e];
            if (!(cur < TC_INF)) continue;
            const unsigned long long key = ld_volatile_u64(&bsf);
            if (cur > prune_threshold(key, S.rho)) continue;
            if (!(cur > (pass == 0 ? S.e_pc : S.e_ti) * best_dist(key))) continue;
            const float *c = S.cand + (size_t)sv[e] * L * D;
            float bound = 0.f;
            bool dropped;
            if (pass == 0) {
                dropped = D <= 8 ? lb_pc_pair<8, true>(c, S.boxes + (size_t)q * S.Gpc * S.K * 2 * D,
                                                 S.box_counts + (size_t)q * S.Gpc, L, D, S.K, S.w, &bsf, S.rho, &bound)
                                 : lb_pc_pair<16, true>(c, S.boxes + (size_t)q * S.Gpc * S.K * 2 * D,
                                                  S.box_counts + (size_t)q * S.Gpc, L, D, S.K, S.w, &bsf, S.rho, &bound);
            } else {
                const float *qa = S.q + (size_t)q * L * D;
                dropped = D <= 8 ? lb_ti_pair<8, true>(c, qa, S.dq_lo + (size_t)q * L, S.dq_hi + (size_t)q * L, L, D, S.W,
                                                 S.P, &bsf, S.rho, &bound)
                                 : lb_ti_pair<16, true>(c, qa, S.dq_lo + (size_t)q * L, S.dq_hi + (size_t)q * L, L, D, S.W,
                                                  S.P, &bsf, S.rho, &bound);
            }
            if (lane == 0) {
                if (dropped) { slb[e] = TC_INF; ++pruned; }
                else slb[e] = fmaxf(cur, bound);
            }
        }
        if (lane == 0 && pruned) atomicAdd(&ctl->counters[5 + pass], pruned);
        __syncthreads();
    }
    // DTW of the survivors
    if (threadIdx.x == 0) cursor = 0;
    __syncthreads();
    batch_dtw_dispatch(S, q, sv, slb, cnt, sdt, &bsf, &cursor, stage, ctl);
    __syncthreads();
    // FP64 refine of every candidate within the rounding margin of the best
    const float tfin = prune_threshold(bsf, S.rho_ref);
    Grp g32 = make_grp(32);
    const float *qa = S.q + (size_t)q * L * D;
    double *d64 = S.d64 + (size_t)q * (N + 8);
    const int ntot = nseed + cnt;
    for (int e = warp; e < ntot; e += nw) {
        const float d32 = e < nseed ? seed_dtw[e] : sdt[e - nseed];
        const uint32_t cn = e < nseed ? seeds[e] : sv[e - nseed];
        double r = __longlong_as_double(0x7ff0000000000000LL);
        if (d32 <= tfin) {
            r = batch_fp64(S, qa, S.cand + (size_t)cn * L * D, g32);
            r = grp_min(r, g32);
            if (lane == 0) {
                atomicMin(&best64, (unsigned long long)__double_as_longlong(r));
                atomicAdd(&ctl->counters[7], 1ull);
            }
        }
        if (lane == 0) d64[e] = r;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ntot; e += blockDim.x) {
        if ((unsigned long long)__double_as_longlong(d64[e]) == best64) {
            const uint32_t cn = e < nseed ? seeds[e] : sv[e - nseed];
            atomicMin(&best_idx, (unsigned long long)cn);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        S.idx[q] = (int64_t)best_idx;
        S.dist[q] = __longlong_as_double((long long)best64);
    }
    __syncthreads();
}

// ------------------------------------------------------------------ the persistent kernel
__global__ void __launch_bounds__(kBatchThreads, 3) k_batch(const BatchSet *__restrict__ sets,
                                                         const BatchItem *__restrict__ items, int n_items,
                                                         BatchCtl *ctl, long long spin_limit) {
    extern __shared__ __align__(16) float bsm[];
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = *(volatile int *)&ctl->abort ? n_items : atomicAdd(&ctl->next, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const BatchItem item = items[it];
        const BatchSet &S = sets[item.set];
        if (item.kind == kItemPrep) {
            prep_item(S, item.a, bsm, ctl);
            batch_done(S.prep_done);
        } else if (item.kind == kItemMv) {
            if (!batch_wait(S.prep_done, S.M, spin_limit, ctl, it)) continue;
            __threadfence();
            float(*sc)[kMvRows * kMvChunk] = (float(*)[kMvRows * kMvChunk])bsm;
            float(*su)[kBatchQB * kMvChunk] = (float(*)[kBatchQB * kMvChunk])(bsm + 2 * kMvRows * kMvChunk);
            float(*sl)[kBatchQB * kMvChunk] =
                (float(*)[kBatchQB * kMvChunk])(bsm + 2 * kMvRows * kMvChunk + 2 * kBatchQB * kMvChunk);
            lb_mv_tile<kBatchQB>(S.cand, S.N, S.L * S.D, S.vec4 != 0, S.U, S.Lo, S.ldE, S.M, S.lbm, S.N,
                                 (int64_t)item.b * kMvRows, item.a * kBatchQB, sc, su, sl);
            batch_done(S.mv_done);
        } else if (item.kind == kItemSearch) {
            if (!batch_wait(S.mv_done, S.n_qtiles * S.n_ctiles, spin_limit, ctl, it)) continue;
            __threadfence();
            search_item(S, item.a, bsm, ctl);
        } else {  // kItemStall: waits for a counter nothing increments (self-test)
            batch_wait(&ctl->never, 1, spin_limit, ctl, it);
        }
    }
}

static_assert(2 * kMvRows * kMvChunk * 4 + 4 * kBatchQB * kMvChunk * 4 <= kBatchSmem, "LB_MV buffers");
static_assert(kBatchThreads * kBatchR * kBatchMaxD * 4 <= kBatchSmem, "DTW staging");

// ------------------------------------------------------------------ host side
namespace {

int batch_G(int W) {
    for (int g = 4; g <= 32; g *= 2)
        if (g * (kBatchR + 1) >= 2 * W + kBatchR) return g;
    return 0;
}

// A workspace arena and a captured graph per batch description.
struct BatchPlan {
    std::vector<tcdtw_dataset> key;
    tcdtw_opts opts;
    void *arena = nullptr;
    BatchSet *d_sets = nullptr;
    BatchItem *d_items = nullptr;
    BatchCtl *d_ctl = nullptr;
    int *d_counts = nullptr;
    int n_items = 0, n_sets = 0, grid = 0;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
    unsigned long long last_use = 0;
};
std::vector<BatchPlan *> g_plans;
std::mutex g_plans_mu;
unsigned long long g_plan_clock = 0;

void free_plan(BatchPlan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    cudaFree(p->arena);
    delete p;
}

bool same_key(const BatchPlan *p, const tcdtw_dataset *sets, int n, const tcdtw_opts &o) {
    if ((int)p->key.size() != n || memcmp(&p->opts, &o, sizeof(o)) != 0) return false;
    return memcmp(p->key.data(), sets, sizeof(tcdtw_dataset) * n) == 0;
}

bool megakernel_ok(const tcdtw_dataset &d, const tcdtw_opts &o) {
    const int W = d.W > d.L - 1 ? d.L - 1 : d.W;
    return d.D <= kBatchMaxD && batch_G(W) > 0 && refine_rows_for(W) > 0 && d.M <= 65535 && o.seed_s <= 8;
}

template <typename T>
T *carve(char *&p, size_t n) {
    p = (char *)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    T *r = (T *)p;
    p += sizeof(T) * (n ? n : 1);
    return r;
}

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
        b.G = batch_G(b.W);
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
        b.rho = o.no_prune ? INFINITY : b.rho_ref;
        b.ldE = ((int64_t)d.L * d.D + 31) / 32 * 32;
        b.n_qtiles = (int)((d.M + kBatchQB - 1) / kBatchQB);
        b.n_ctiles = (int)((d.N + kMvRows - 1) / kMvRows);
        const int64_t Mp = (d.M + 1) / 2 * 2, M = d.M, N = d.N;
        bytes += 2 * (sizeof(float) * Mp * b.ldE + 256);
        bytes += 2 * (sizeof(float) * M * d.L + 256);
        if (b.use_pc) bytes += sizeof(float) * M * b.Gpc * d.K * 2 * d.D + sizeof(int32_t) * M * b.Gpc + 512;
        bytes += 3 * (sizeof(float) * M * N + 256) + sizeof(uint32_t) * M * N + 256;
        bytes += sizeof(double) * M * (N + 8) + 256;
        hs.push_back(b);
        cost.push_back((double)N * d.L * d.D * M + (double)M * N * d.L * (2.0 * b.W + 1) * 0.05);
    }
    const int ns = (int)hs.size();
    bytes += sizeof(BatchSet) * ns + sizeof(BatchItem) * 4 + sizeof(BatchCtl) + sizeof(int) * 2 * ns + 4096;
    // items: PREP, LBMV, SEARCH, each kind in decreasing set cost
    std::vector<int> order(ns);
    for (int k = 0; k < ns; ++k) order[k] = k;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<BatchItem> items;
    for (int k : order)
        for (int m = 0; m < hs[k].M; ++m) items.push_back({kItemPrep, k, m, 0});
    for (int k : order)
        for (int ct = 0; ct < hs[k].n_ctiles; ++ct)
            for (int qt = 0; qt < hs[k].n_qtiles; ++qt) items.push_back({kItemMv, k, qt, ct});
    for (int k : order)
        for (int m = 0; m < hs[k].M; ++m) items.push_back({kItemSearch, k, m, 0});
    bytes += sizeof(BatchItem) * items.size();
    if (cudaMalloc(&p->arena, bytes) != cudaSuccess) {
        delete p;
        return TCDTW_ERR_NOMEM;
    }
    char *c = (char *)p->arena;
    p->d_sets = carve<BatchSet>(c, ns);
    p->d_items = carve<BatchItem>(c, items.size());
    p->d_ctl = carve<BatchCtl>(c, 1);
    p->d_counts = carve<int>(c, 2 * ns);
    for (int k = 0; k < ns; ++k) {
        BatchSet &b = hs[k];
        const int64_t Mp = (b.M + 1) / 2 * 2, M = b.M, N = b.N;
        b.U = carve<float>(c, Mp * b.ldE);
        b.Lo = carve<float>(c, Mp * b.ldE);
        b.dq_lo = carve<float>(c, M * b.L);
        b.dq_hi = carve<float>(c, M * b.L);
        if (b.use_pc) {
            b.boxes = carve<float>(c, M * b.Gpc * b.K * 2 * b.D);
            b.box_counts = carve<int32_t>(c, M * b.Gpc);
        }
        b.lbm = carve<float>(c, M * N);
        b.surv_lb = carve<float>(c, M * N);
        b.surv_dtw = carve<float>(c, M * N);
        b.seed_dtw = nullptr;
        b.surv = carve<uint32_t>(c, M * N);
        b.d64 = carve<double>(c, M * (N + 8));
        b.prep_done = p->d_counts + 2 * k;
        b.mv_done = p->d_counts + 2 * k + 1;
    }
    cudaError_t e = cudaMemcpyAsync(p->d_sets, hs.data(), sizeof(BatchSet) * ns, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem);
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch, kBatchThreads, kBatchSmem);
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_err(e);
    }
    p->n_items = (int)items.size();
    p->n_sets = ns;
    p->grid = (occ > 0 ? occ : 1) * num_sms();
    if (p->grid > p->n_items) p->grid = p->n_items;
    *out = p;
    return TCDTW_OK;
}

cudaError_t enqueue_plan(BatchPlan *p, cudaStream_t s, long long spin_limit) {
    cudaError_t e = cudaMemsetAsync(p->d_ctl, 0, sizeof(BatchCtl), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_counts, 0, sizeof(int) * 2 * p->n_sets, s);
    if (e != cudaSuccess) return e;
    k_batch<<<p->grid, kBatchThreads, kBatchSmem, s>>>(p->d_sets, p->d_items, p->n_items, p->d_ctl, spin_limit);
    note_launch();
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
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int> mk, other;
    for (int32_t k = 0; k < nsets; ++k) {
        const tcdtw_dataset &d = sets[k];
        if (d.N < 1 || d.L < 1 || d.D < 1 || d.W < 0 || d.K < 1 || d.M < 0) return TCDTW_ERR_INVALID;
        if (!d.cand || (d.M > 0 && (!d.q || !d.idx || !d.dist))) return TCDTW_ERR_INVALID;
        if (d.D > TCDTW_MAX_D) return TCDTW_ERR_UNSUPPORTED;
        if (d.M == 0) continue;
        (megakernel_ok(d, o) ? mk : other).push_back(k);
    }
    uint64_t pairs = 0;
    if (!mk.empty()) {
        // candidates of the megakernel sets: non-finite scan (the queries are checked in PREP)
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
                    note_launches(-1);  // captured, not launched
                }
                cudaStreamDestroy(cs);
            }
            if (e == cudaSuccess) {
                note_launches(1);
                e = cudaGraphLaunch(plan->exec, s);
            }
        }
        ++plan->launches;
        if (e == cudaSuccess && o.check_finite) {
            for (int k : mk) {
                const tcdtw_dataset &d = sets[k];
                e = launch_check_finite(d.cand, d.N * (int64_t)d.L * d.D, &plan->d_ctl->status, 0, s);
                if (e != cudaSuccess) break;
            }
        }
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
        }
        for (int k : mk) pairs += (uint64_t)sets[k].M * (uint64_t)sets[k].N;
    }
    // shapes outside the megakernel's tile family: one index per set
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
            stats->cells += st.cells; stats->refined += st.refined;
        }
        pairs += (uint64_t)d.M * (uint64_t)d.N;
    }
    if (stats) stats->pairs = pairs;
    return TCDTW_OK;
}

// Self-test of the device-side wait limit: one persistent launch whose only item
// waits for a counter that nothing increments; the launch must end by itself with
// TCDTW_ERR_TIMEOUT after ~spin_limit sleeps, leaving the context usable.
int tcdtw_batch_selftest_timeout(int64_t spin_limit, void *stream) {
    if (spin_limit < 1) return TCDTW_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    BatchItem item{kItemStall, 0, 0, 0};
    BatchItem *d_item = nullptr;
    BatchCtl *d_ctl = nullptr;
    BatchSet *d_set = nullptr;
    cudaError_t e = cudaMalloc(&d_item, sizeof(item));
    if (e == cudaSuccess) e = cudaMalloc(&d_set, sizeof(BatchSet));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_set, 0, sizeof(BatchSet), s);
    if (e == cudaSuccess) e = cudaMalloc(&d_ctl, sizeof(BatchCtl));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_item, &item, sizeof(item), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ctl, 0, sizeof(BatchCtl), s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem);
    if (e == cudaSuccess) {
        k_batch<<<1, kBatchThreads, kBatchSmem, s>>>(d_set, d_item, 1, d_ctl, (long long)spin_limit);
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
