// api_nn.cu -- C ABI of the exact DTW-NN search (Def. 1; the search loop of
// Sections 6-7 laid out as a GPU pipeline) and of its individual stages.
//
// Per block of Mb queries, everything stays on the device:
//   1  envelopes, neighbour distances, LB_PC boxes          (prep.cu)
//   2  LB_MV of every (query, candidate) pair              (lb.cu, HBM/L2 stream)
//   3  seeds: per query the seed_s smallest LB_MV, their DTW lowers best-so-far
//   4  compaction of pairs with LB_MV <= threshold         (ordered, flat list)
//   5  gated LB_PC / LB_TI on the survivors (e*bsf < LB_MV < bsf, Section 6)
//   6  banded DTW of the survivors, abandoning against the live best-so-far
//   7  candidates whose FP32 DTW is within the rounding margin of the best are
//      recomputed in FP64; the FP64 minimum (smallest index on ties) is the answer.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include <nvtx3/nvToolsExt.h>
#include <mutex>
#include <new>
#include <vector>

#include "api_internal.h"
#include "common.cuh"
#include "dtw_tiles.cuh"
#include "lb_kernels.cuh"

using namespace tc;

namespace tc {

// Pruning factor rho = (1+g32)/(1-g32) * (1+g64)/(1-g64) with g = n*u/(1-n*u),
// n = 2L+D+2 roundings along a warping path (cell cost and DP additions), u the
// unit roundoff.  Rounded up to float.
float prune_rho(int L, int D) {
    const double n = 2.0 * L + D + 2.0;
    const double u32 = ldexp(1.0, -24), u64 = ldexp(1.0, -53);
    const double g32 = n * u32 / (1.0 - n * u32), g64 = n * u64 / (1.0 - n * u64);
    const double rho = (1.0 + g32) / (1.0 - g32) * (1.0 + g64) / (1.0 - g64);
    float r = (float)rho;
    if ((double)r < rho) r = nextafterf(r, INFINITY);
    return r;
}

// Separation factor of the double-float refine: a candidate whose double-float DTW
// exceeds the best one's times kappa has a larger FP64 DTW.  kappa =
// (1+g64)(1+G)/((1-g64)(1-G)), where G bounds the relative error of the double-float
// DP (cell costs (3D+2)(D+3)u^2/(1-(3D+2)u), u = 2^-24; at most 2L double-word
// additions of relative error 4u^2 along a path; the final rounding to double) and
// g64 = n u64/(1 - n u64), n = 2L+D+2, bounds the FP64 evaluation's error.  Both
// bounds are doubled for safety; rounded up.
double refine_kappa(int L, int D) {
    const double u = ldexp(1.0, -24), u64 = ldexp(1.0, -53);
    const double k = 3.0 * D + 2.0;
    const double e_cost = k * (D + 3.0) * u * u / (1.0 - k * u);
    const double G = 2.0 * ((1.0 + e_cost) * pow(1.0 + 4.0 * u * u, 2.0 * L) - 1.0 + 2.0 * u64);
    const double n = 2.0 * L + D + 2.0;
    const double g64 = 2.0 * (n * u64 / (1.0 - n * u64));
    const double kappa = (1.0 + g64) * (1.0 + G) / ((1.0 - g64) * (1.0 - G));
    return nextafter(nextafter(kappa, INFINITY), INFINITY);
}

bool pc_key_fits(int Lq, int D) {
    // Lq^D must fit below 2^63 (mixed-radix cell key)
    long double v = 1;
    for (int p = 0; p < D; ++p) {
        v *= Lq;
        if (v > 9.2e18L) return false;
    }
    return true;
}

// ------------------------------------------------------------------ autotuner
// Times every valid (tile, G) of the D bucket on a sample of real pairs (candidate k
// against candidate k+1, full band, no abandoning) and keeps the fastest.  Results
// are cached per (L, D, W) for the life of the process.
struct TuneKey {
    int L, D, W;
    bool operator==(const TuneKey &o) const { return L == o.L && D == o.D && W == o.W; }
};
struct TuneVal {
    int tile, G;
};
static std::vector<std::pair<TuneKey, TuneVal>> g_tune_cache;
static std::mutex g_tune_mu;  // indexes may be built from several host threads

// Persistent tuner cache: with the environment variable TCDTW_TUNE_CACHE naming a file,
// results are read from it on first use and appended to it after each new tuning, one
// line "tcdtw-tune <tile-table signature> <device name> L D W tile G" per shape; lines of
// another device or another build's tile table are ignored.
static bool g_tune_file_read = false;

static unsigned tile_table_signature() {
    unsigned h = 2166136261u;  // FNV-1a over the compiled tiles
    for (int t = 0; t < kNumTiles; ++t) {
        h = (h ^ (unsigned)kTiles[t].R) * 16777619u;
        h = (h ^ (unsigned)kTiles[t].DMAX) * 16777619u;
    }
    return h;
}

static void device_tag(char *out, size_t n) {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        snprintf(out, n, "unknown");
        return;
    }
    snprintf(out, n, "%s", prop.name);
    for (char *c = out; *c; ++c)
        if (*c == ' ' || *c == '\t') *c = '_';
}

static void tune_file_load_locked() {
    if (g_tune_file_read) return;
    g_tune_file_read = true;
    const char *path = getenv("TCDTW_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char tag[256], line[512], ftag[256];
    device_tag(tag, sizeof(tag));
    const unsigned sig = tile_table_signature();
    while (fgets(line, sizeof(line), f)) {
        unsigned fsig = 0;
        int L, D, W, tile, G;
        if (sscanf(line, "tcdtw-tune %x %255s %d %d %d %d %d", &fsig, ftag, &L, &D, &W, &tile, &G) != 7) continue;
        if (fsig != sig || strcmp(ftag, tag) != 0 || tile < 0 || tile >= kNumTiles) continue;
        if (kTiles[tile].DMAX != dmax_for(D) || !tile_valid(tile, G, W)) continue;
        const TuneKey key{L, D, W};
        bool have = false;
        for (auto &kv : g_tune_cache) have = have || kv.first == key;
        if (!have) g_tune_cache.push_back({key, TuneVal{tile, G}});
    }
    fclose(f);
}

static void tune_file_append(const TuneKey &k, const TuneVal &v) {
    const char *path = getenv("TCDTW_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    char tag[256];
    device_tag(tag, sizeof(tag));
    fprintf(f, "tcdtw-tune %x %s %d %d %d %d %d\n", tile_table_signature(), tag, k.L, k.D, k.W, v.tile, v.G);
    fclose(f);
}

bool autotune_nn_tile(const float *cand, int64_t N, int L, int D, int W, cudaStream_t s, int *tile, int *G) {
    const TuneKey key{L, D, W};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tune_file_load_locked();
        for (auto &kv : g_tune_cache)
            if (kv.first == key) { *tile = kv.second.tile; *G = kv.second.G; return true; }
    }
    const int dm = dmax_for(D);
    if (dm < 0) return false;
    // enough pairs to fill every SM even with 4-lane groups (8 pairs per warp), but
    // at most ~4e9 band cells; runs of 64 pairs share a "query" (candidate m), as the
    // survivor lists of a search do.
    const double band = (double)L * (2 * W + 1) - (double)W * (W + 1);
    int64_t P = (int64_t)(4.0e9 / band);
    if (P > 65536) P = 65536;
    if (P < 16384) P = 16384;
    int64_t Mq = N < 4096 ? N : 4096;
    while (Mq > 1 && (double)Mq * (double)N >= 4.29e9) Mq >>= 1;
    uint32_t *pairs = nullptr;
    unsigned long long *bsf = nullptr;
    float *dtw = nullptr;
    int *cursor = nullptr;
    bool ok = dev_malloc((void **)&pairs, sizeof(uint32_t) * P) == cudaSuccess &&
              dev_malloc((void **)&bsf, sizeof(unsigned long long) * Mq) == cudaSuccess &&
              dev_malloc((void **)&dtw, sizeof(float) * P) == cudaSuccess && dev_malloc((void **)&cursor, sizeof(int)) == cudaSuccess;
    std::vector<uint32_t> h(P);
    for (int64_t i = 0; i < P; ++i) {
        const int64_t m = (i / 64) % Mq, n = (i * 7919 + 13) % N;
        h[i] = (uint32_t)(m * N + n);
    }
    ok = ok && cudaMemcpyAsync(pairs, h.data(), sizeof(uint32_t) * P, cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && launch_init_block(Mq, bsf, nullptr, nullptr, nullptr, nullptr, nullptr, s) == cudaSuccess;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ok = ok && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    float best = 1e30f;
    bool found = false;
    for (int t = 0; ok && t < kNumTiles; ++t) {
        if (kTiles[t].DMAX != dm) continue;
        for (int g = 4; g <= 32 && ok; g *= 2) {
            if (!tile_valid(t, g, W)) continue;
            DtwNnArgs dn;
            dn.Q = cand; dn.C = cand; dn.L = L; dn.D = D; dn.W = W; dn.G = g; dn.N = N; dn.pairs = pairs;
            dn.lb = nullptr; dn.count = nullptr; dn.n_static = (int)P; dn.cursor = cursor; dn.bsf = bsf;
            dn.rho = INFINITY; dn.dtw = dtw; dn.counters = nullptr;
            int blocks = dtw_occupancy(t, 1, g) * num_sms();
            if (blocks < 1) blocks = num_sms();
            float ms_best = 1e30f;
            for (int rep = 0; rep < 3 && ok; ++rep) {
                ok = cudaMemsetAsync(cursor, 0, sizeof(int), s) == cudaSuccess;
                ok = ok && cudaEventRecord(e0, s) == cudaSuccess;
                ok = ok && dtw_nn_launch(t, blocks, s, dn) == cudaSuccess;
                ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
                float ms = 0.f;
                ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
                if (ok && rep > 0 && ms < ms_best) ms_best = ms;  // rep 0 warms up
            }
            if (ok && ms_best < best) { best = ms_best; *tile = t; *G = g; found = true; }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(pairs); cudaFree(bsf); cudaFree(dtw); cudaFree(cursor);
    if (found) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache.push_back({key, TuneVal{*tile, *G}});
        tune_file_append(key, TuneVal{*tile, *G});
    }
    return found;
}

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    return dev_malloc((void **)p, n * sizeof(T));
}

enum Counter {
    kStarted = 0, kAbandoned, kCells, kPrunedDtw, kPrunedMv, kPrunedPc, kPrunedTi, kRefined, kRefined64, kPrunedRev,
    kMvTerms, kNumCounters
};
enum Scalar { kSurvTotal = 0, kCursorSeed, kCursorSurv, kRefineCount, kRefine64Count, kCursorSeed2, kNumScalars };
constexpr int kFewQueries = 4;  // query blocks at most this big run their survivors on the seed tile

}  // namespace tc

struct tcdtw_index {
    const float *cand = nullptr;
    int64_t N = 0;
    int L = 0, D = 0, W = 0, K = 0;
    tcdtw_opts opts;
    int Mb = 0, Mb_pad = 0, S = 0, G_pc = 0;
    int64_t ldE = 0;
    float rho = 1.f;         // pruning / abandoning factor (+inf with no_prune)
    float rho_ref = 1.f;     // refine factor (always the rounding margin)
    double kappa = 1.0;      // double-float separation factor of the refine (refine_kappa)
    int tile = 0, G = 32, R_ref = 1, sms = 1;
    int blocks_nn = 1, blocks_ref = 1;
    // the seeds' DTW (a few pairs per query, nothing to abandon against at first):
    // the tile of the same point width with the fewest rows per lane and the
    // smallest valid lane group, so that its few pairs spread over more warps
    int tile_seed = 0, G_seed = 32, blocks_seed = 1;
    bool selected = false;   // TC-DTW bound choice made (opts.select)
    // workspaces
    float *U = nullptr, *Lo = nullptr, *dq_lo = nullptr, *dq_hi = nullptr, *boxes = nullptr, *lbm = nullptr;
    int32_t *box_counts = nullptr;
    uint32_t *seeds = nullptr, *surv = nullptr, *refine = nullptr, *refine64 = nullptr;
    float *seed_dtw = nullptr, *surv_lb = nullptr, *surv_dtw = nullptr;
    double *refine_d64 = nullptr, *refine64_d64 = nullptr;
    int32_t *amb = nullptr;
    int32_t *row_counts = nullptr, *row_offsets = nullptr, *scalars = nullptr;
    unsigned long long *bsf = nullptr, *best64 = nullptr, *best_idx = nullptr, *counters = nullptr;
    unsigned long long *bestdf = nullptr, *best_idx_df = nullptr;
    DevStatus *status = nullptr;
    float *Uc = nullptr, *Lc = nullptr;  // candidate envelopes [N][L*D] (use_rev)
    float2 *ref_tab = nullptr;   // global cost tables of the double-float refine (long bands)
    int ref_slots = 0;
    // LB_MV with early abandoning (opts.mv_abandon): the sampled chunks (count, 0: off, and
    // stride), second-round seeds per query, the envelope one query per row, the
    // completion kernel's pair lists
    int mv_samp = 0, mv_stride = 1, S2 = 0;
    float *Up = nullptr, *Lp = nullptr;
    uint32_t *rest_list = nullptr;
    int64_t rest_list_entries = 0;
    float *mv_ws = nullptr;      // partial sums of split LB_MV tiles
    int64_t mv_ws_floats = 0;
    int32_t *mv_cnt = nullptr;   // their per-tile arrival counters (kept zero)
    int64_t refine_cap = 0;
    // per-stage CUDA-event profile (tcdtw_set_profiling)
    bool profile = false;
    std::vector<cudaEvent_t> events;   // (TCDTW_NUM_STAGES + 1) marks per block
    int marks_used = 0;
    double stage_ms[TCDTW_NUM_STAGES] = {0};
    int64_t stage_blocks = 0;
    // CUDA graphs of the per-call kernel sequence of single-block calls, keyed by the
    // number of queries: the graph reads the queries from qbuf and writes the answers
    // to idx_buf / dist_buf, and each call copies in and out around it on its stream,
    // so replay does not depend on where the caller's buffers are
    float *qbuf = nullptr;
    int64_t *idx_buf = nullptr;
    double *dist_buf = nullptr;
    struct GraphEntry {
        int64_t M;
        int seen;                      // eager calls made with this key
        cudaGraphExec_t exec;          // null until captured
        unsigned long long last_use;
        int marks;                     // profiling event marks recorded by the graph
        bool profiled;                 // captured with profiling on
        int kernels;                   // kernel launches captured in the graph
    };
    std::vector<GraphEntry> graphs;
    unsigned long long graph_clock = 0;
    cudaStream_t cap_stream = nullptr;
    bool capturing = false;
};

namespace {

void free_index(tcdtw_index *x) {
    if (!x) return;
    for (cudaEvent_t ev : x->events) cudaEventDestroy(ev);
    for (auto &g : x->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (x->cap_stream) cudaStreamDestroy(x->cap_stream);
    void *ptrs[] = {x->U, x->Lo, x->Up, x->Lp, x->rest_list, x->dq_lo, x->dq_hi, x->boxes, x->lbm,
                    x->box_counts, x->seeds, x->surv, x->refine, x->seed_dtw, x->surv_lb, x->surv_dtw, x->refine_d64, x->row_counts,
                    x->row_offsets, x->scalars, x->bsf, x->best64, x->best_idx, x->counters, x->status,
                    x->refine64, x->refine64_d64, x->amb, x->bestdf, x->best_idx_df, x->mv_ws, x->mv_cnt,
                    x->Uc, x->Lc, x->qbuf, x->idx_buf, x->dist_buf, x->ref_tab};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete x;
}

int validate_shape(int64_t N, int L, int D, int W, int K) {
    if (N < 1 || L < 1 || D < 1 || W < 0 || K < 1) return TCDTW_ERR_INVALID;
    if (D > TCDTW_MAX_D) return TCDTW_ERR_UNSUPPORTED;
    return TCDTW_OK;
}

#define TC_TRY(expr)                                  \
    do {                                              \
        cudaError_t e_ = (expr);                      \
        if (e_ != cudaSuccess) return cuda_err(e_);   \
    } while (0)

int alloc_index(tcdtw_index *x) {
    const int64_t Mb = x->Mb, N = x->N;
    const int L = x->L, D = x->D;
    TC_TRY(dalloc(&x->U, (size_t)x->Mb_pad * x->ldE));
    TC_TRY(dalloc(&x->Lo, (size_t)x->Mb_pad * x->ldE));
    TC_TRY(dalloc(&x->dq_lo, (size_t)Mb * L));
    TC_TRY(dalloc(&x->dq_hi, (size_t)Mb * L));
    if (x->opts.use_pc) {
        TC_TRY(dalloc(&x->boxes, (size_t)Mb * x->G_pc * x->K * 2 * D));
        TC_TRY(dalloc(&x->box_counts, (size_t)Mb * x->G_pc));
    }
    TC_TRY(dalloc(&x->lbm, (size_t)Mb * N));
    TC_TRY(dalloc(&x->seeds, (size_t)Mb * (x->S + x->S2)));
    TC_TRY(dalloc(&x->seed_dtw, (size_t)Mb * (x->S + x->S2)));
    if (x->mv_samp > 0) {
        TC_TRY(dalloc(&x->Up, (size_t)Mb * x->ldE));
        TC_TRY(dalloc(&x->Lp, (size_t)Mb * x->ldE));
        x->rest_list_entries = lb_mv_rest_list_entries(N, x->Mb, x->sms);
        TC_TRY(dalloc(&x->rest_list, (size_t)x->rest_list_entries));
    }
    TC_TRY(dalloc(&x->surv, (size_t)Mb * N));
    TC_TRY(dalloc(&x->surv_lb, (size_t)Mb * N));
    TC_TRY(dalloc(&x->surv_dtw, (size_t)Mb * N));
    x->refine_cap = Mb * (N + x->S + x->S2);
    TC_TRY(dalloc(&x->refine, (size_t)x->refine_cap));
    TC_TRY(dalloc(&x->refine_d64, (size_t)x->refine_cap));
    TC_TRY(dalloc(&x->refine64, (size_t)x->refine_cap));
    TC_TRY(dalloc(&x->refine64_d64, (size_t)x->refine_cap));
    TC_TRY(dalloc(&x->amb, (size_t)Mb));
    TC_TRY(dalloc(&x->bestdf, (size_t)Mb));
    TC_TRY(dalloc(&x->best_idx_df, (size_t)Mb));
    TC_TRY(dalloc(&x->row_counts, (size_t)Mb));
    TC_TRY(dalloc(&x->row_offsets, (size_t)Mb));
    TC_TRY(dalloc(&x->scalars, (size_t)kNumScalars));
    TC_TRY(dalloc(&x->bsf, (size_t)Mb));
    TC_TRY(dalloc(&x->best64, (size_t)Mb));
    TC_TRY(dalloc(&x->best_idx, (size_t)Mb));
    TC_TRY(dalloc(&x->counters, (size_t)kNumCounters));
    TC_TRY(dalloc(&x->status, 1));
    TC_TRY(cudaMemset(x->status, 0, sizeof(DevStatus)));
    x->mv_ws_floats = std::min<int64_t>(kMvWsFloats, 64 * Mb * N);
    TC_TRY(dalloc(&x->mv_ws, (size_t)x->mv_ws_floats));
    TC_TRY(dalloc(&x->mv_cnt, (size_t)kMvTileCounters));
    TC_TRY(cudaMemset(x->mv_cnt, 0, sizeof(int32_t) * kMvTileCounters));
    TC_TRY(cudaMemset(x->counters, 0, sizeof(unsigned long long) * kNumCounters));
    if (!refine_df_table_fits_smem(L, D, x->W)) {
        // two table slots per SM (bounded to ~1.1 GB), each L*(2W+1) double-float costs:
        // a block of up to 256 queries refines its ~one entry per query in one round
        const size_t slot = refine_gtab_slot_bytes(L, x->W);
        int64_t slots = (int64_t)(1.1e9 / (double)slot);
        if (slots > 2 * x->sms) slots = 2 * x->sms;
        if (slots < 1) slots = 1;
        x->ref_slots = (int)slots;
        TC_TRY(dalloc(&x->ref_tab, (size_t)slots * slot / sizeof(float2)));
    }
    if (x->opts.use_graph) {
        TC_TRY(dalloc(&x->qbuf, (size_t)Mb * L * D));
        TC_TRY(dalloc(&x->idx_buf, (size_t)Mb));
        TC_TRY(dalloc(&x->dist_buf, (size_t)Mb));
    }
    return TCDTW_OK;
}

// Stage boundary k of the current block (profiling only).
// With profiling on, every stage is also an NVTX range on the calling thread (seen by
// Nsight Systems when it is attached; the calls do nothing otherwise).
const char *const kStageRange[TCDTW_NUM_STAGES] = {"tcdtw check",   "tcdtw prep",    "tcdtw lb_mv",
                                                   "tcdtw seed",    "tcdtw lb_rest", "tcdtw seed2",
                                                   "tcdtw compact", "tcdtw cascade", "tcdtw dtw",
                                                   "tcdtw refine"};

cudaError_t mark(tcdtw_index *x, int k, cudaStream_t s) {
    if (!x->profile) return cudaSuccess;
    if (k > 0) nvtxRangePop();
    if (k < TCDTW_NUM_STAGES) nvtxRangePushA(kStageRange[k]);
    const size_t slot = (size_t)x->marks_used;
    if (slot >= x->events.size()) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return e;
        x->events.push_back(ev);
    }
    (void)k;
    ++x->marks_used;
    // while capturing, an external record becomes a timing node of the graph
    if (x->capturing) return cudaEventRecordWithFlags(x->events[slot], s, cudaEventRecordExternal);
    return cudaEventRecord(x->events[slot], s);
}

#define TC_MARK(k)                                            \
    do {                                                      \
        if ((e = mark(x, (k), s)) != cudaSuccess) return e;   \
    } while (0)

// One block of Mb_cur queries.  All launches on stream s; no host synchronisation.
// Whether a block of Mb_cur queries runs LB_MV with early abandoning.  Below 32 queries
// the dense stream is bound by one pass over the candidates, which the completion pass
// repeats for any tile with a live pair, and the second seed round adds a DTW sweep of
// latency: the plain stream is faster there.
constexpr int kAbandonMinQueries = 32;
bool block_abandons(const tcdtw_index *x, int Mb_cur) { return x->mv_samp > 0 && Mb_cur >= kAbandonMinQueries; }

// Seed entries of a block (both rounds).
int64_t block_seeds(const tcdtw_index *x, int Mb_cur) {
    return (int64_t)Mb_cur * (x->S + (block_abandons(x, Mb_cur) ? x->S2 : 0));
}

cudaError_t run_block(tcdtw_index *x, const float *q, int Mb_cur, int64_t *idx_out, double *dist_out,
                      cudaStream_t s) {
    const int L = x->L, D = x->D, W = x->W;
    const int64_t N = x->N;
    const int E = L * D;
    cudaError_t e;
    TC_MARK(0);
    if (x->opts.check_finite) {
        e = launch_check_finite(q, (int64_t)Mb_cur * E, x->status, 1, s);
        if (e != cudaSuccess) return e;
    }
    TC_MARK(1);
    e = cudaMemsetAsync(x->scalars, 0, sizeof(int32_t) * kNumScalars, s);
    if (e != cudaSuccess) return e;
    if ((e = launch_init_block(Mb_cur, x->bsf, x->best64, x->best_idx, x->bestdf, x->best_idx_df, x->amb, s)) !=
        cudaSuccess)
        return e;
    const bool ab = block_abandons(x, Mb_cur) && !x->opts.no_prune;
    // 1. query-side preparation
    e = ab ? launch_envelope_pairs_plain(q, Mb_cur, L, D, W, x->U, x->Lo, x->Up, x->Lp, (int)x->ldE, s)
           : launch_envelope_pairs(q, Mb_cur, L, D, W, x->U, x->Lo, (int)x->ldE, s);
    if (e != cudaSuccess) return e;
    if (x->opts.use_ti && (e = launch_query_dq(q, Mb_cur, L, D, x->dq_lo, x->dq_hi, s)) != cudaSuccess) return e;
    if (x->opts.use_pc &&
        (e = launch_pc_boxes(q, Mb_cur, L, D, W, x->K, x->opts.Lq, x->opts.w, x->boxes, x->box_counts, s)) !=
            cudaSuccess)
        return e;
    // 2. LB_MV of all pairs
    TC_MARK(2);
    if (x->opts.no_prune) {
        if ((e = cudaMemsetAsync(x->lbm, 0, sizeof(float) * (size_t)Mb_cur * N, s)) != cudaSuccess) return e;
    } else {
        LbMvArgs mv;
        mv.cand = x->cand; mv.N = N; mv.E = E; mv.U = x->U; mv.Lo = x->Lo; mv.ldE = x->ldE; mv.Mb = Mb_cur;
        mv.lb = x->lbm; mv.ldLb = N; mv.sms = x->sms; mv.status = x->status;
        mv.ws = x->mv_ws; mv.ws_floats = x->mv_ws_floats; mv.tile_cnt = x->mv_cnt; mv.tile_cnt_cap = kMvTileCounters;
        if (ab) {  // with abandoning: the sampled chunks of every pair first
            mv.E = x->mv_samp * 32;
            mv.cstride = x->mv_stride;
            mv.Erow = E;
            mv.ldC = E;
        }
        if ((e = launch_lb_mv(mv, s)) != cudaSuccess) return e;
    }
    // 3. seeds and their DTW
    TC_MARK(3);
    if ((e = launch_seed_topk(x->lbm, Mb_cur, N, N, x->S, x->seeds, s)) != cudaSuccess) return e;
    DtwNnArgs dn;
    dn.Q = q; dn.C = x->cand; dn.L = L; dn.D = D; dn.W = W; dn.G = x->G_seed; dn.N = N;
    dn.pairs = x->seeds; dn.lb = nullptr; dn.count = nullptr; dn.n_static = Mb_cur * x->S;
    dn.cursor = x->scalars + kCursorSeed; dn.bsf = x->bsf; dn.rho = x->rho; dn.dtw = x->seed_dtw;
    dn.counters = x->counters;
    if ((e = dtw_nn_launch(x->tile_seed, x->blocks_seed, s, dn)) != cudaSuccess) return e;
    TC_MARK(4);
    if (ab) {
        // the pairs still at or under the seeded threshold complete their LB_MV (the
        // others keep the sample sum, a lower bound above the threshold) ...
        LbMvRestArgs ra;
        ra.cand = x->cand; ra.N = N; ra.E = E; ra.samp = x->mv_samp; ra.sstride = x->mv_stride; ra.ldC = E; ra.Up = x->Up; ra.Lp = x->Lp;
        ra.ldP = x->ldE; ra.Mb = Mb_cur; ra.lb = x->lbm; ra.ldLb = N; ra.thresh = nullptr; ra.bsf = x->bsf;
        ra.rho = x->rho; ra.list = x->rest_list; ra.list_entries = x->rest_list_entries; ra.sms = x->sms;
        ra.terms = x->counters + kMvTerms; ra.status = x->status;
        if ((e = launch_lb_mv_rest(ra, s)) != cudaSuccess) return e;
    }
    TC_MARK(5);
    if (ab) {
        // ... and a second round of seeds, the smallest completed bounds, starts the best-
        // so-far closer to the answer (their DTW abandons against the first round's)
        if (x->S2 > 0) {
            uint32_t *seeds2 = x->seeds + (size_t)Mb_cur * x->S;
            if ((e = launch_seed_topk(x->lbm, Mb_cur, N, N, x->S2, seeds2, s)) != cudaSuccess) return e;
            dn.pairs = seeds2; dn.n_static = Mb_cur * x->S2; dn.cursor = x->scalars + kCursorSeed2;
            dn.dtw = x->seed_dtw + (size_t)Mb_cur * x->S;
            if ((e = dtw_nn_launch(x->tile_seed, x->blocks_seed, s, dn)) != cudaSuccess) return e;
        }
    }
    dn.G = x->G;
    // 4. compaction against the seeded best-so-far
    TC_MARK(6);
    CompactArgs ca;
    memset(&ca, 0, sizeof(ca));
    ca.lb = x->lbm; ca.M = Mb_cur; ca.N = N; ca.ldLb = N; ca.thresh = nullptr; ca.bsf = x->bsf; ca.rho = x->rho;
    ca.counts = x->row_counts; ca.offsets = x->row_offsets; ca.total = x->scalars + kSurvTotal;
    ca.pairs = x->surv; ca.lbs = x->surv_lb; ca.pruned = x->counters + kPrunedMv;
    if ((e = launch_compact(ca, s)) != cudaSuccess) return e;
    // 5. gated tight bounds
    TC_MARK(7);
    PairListArgs pl;
    pl.Q = q; pl.C = x->cand; pl.L = L; pl.D = D; pl.W = W; pl.pairs = x->surv;
    pl.count = x->scalars + kSurvTotal; pl.n_static = 0; pl.N = N; pl.lb = x->surv_lb;
    const int64_t hint = (int64_t)Mb_cur * 64;
    if (x->opts.use_rev &&
        (e = launch_lb_rev_list(pl, x->Uc, x->Lc, x->bsf, x->rho, x->counters + kPrunedRev, hint, x->sms, s)) !=
            cudaSuccess)
        return e;
    if (x->opts.use_pc &&
        (e = launch_lb_pc_list(pl, x->boxes, x->box_counts, x->K, x->opts.w, x->bsf, x->rho, x->opts.e_pc,
                               x->counters + kPrunedPc, hint, x->sms, s)) != cudaSuccess)
        return e;
    if (x->opts.use_ti) {
        e = x->opts.ti_top ? launch_lb_ti_list(pl, x->dq_lo, x->dq_hi, x->opts.P, x->bsf, x->rho, x->opts.e_ti,
                                               x->counters + kPrunedTi, hint, x->sms, s)
                           : launch_lb_ti_rows_list(pl, x->dq_lo, x->dq_hi, x->opts.P, x->bsf, x->rho,
                                                    x->opts.e_ti, x->counters + kPrunedTi, hint, x->sms, s);
        if (e != cudaSuccess) return e;
    }
    // 6. DTW of the survivors
    TC_MARK(8);
    dn.pairs = x->surv; dn.lb = x->surv_lb; dn.count = x->scalars + kSurvTotal; dn.n_static = 0;
    dn.cursor = x->scalars + kCursorSurv; dn.dtw = x->surv_dtw;
    // a block of a few queries leaves too few survivors to fill the GPU: each pair's
    // sweep latency decides, and the seed tile (fewest rows per lane) is shorter per pair
    // than the autotuned throughput tile
    const bool few = Mb_cur <= kFewQueries;
    dn.G = few ? x->G_seed : x->G;
    if ((e = dtw_nn_launch(few ? x->tile_seed : x->tile, few ? x->blocks_seed : x->blocks_nn, s, dn)) != cudaSuccess)
        return e;
    // 7. refine near-ties in FP64 and select
    TC_MARK(9);
    if ((e = launch_refine_select(x->seeds, x->seed_dtw, nullptr, block_seeds(x, Mb_cur), N, x->bsf, x->rho_ref,
                                  x->refine, x->scalars + kRefineCount, x->refine_cap, x->sms, s)) != cudaSuccess)
        return e;
    if ((e = launch_refine_select(x->surv, x->surv_dtw, x->scalars + kSurvTotal, 0, N, x->bsf, x->rho_ref, x->refine,
                                  x->scalars + kRefineCount, x->refine_cap, x->sms, s)) != cudaSuccess)
        return e;
    // double-float recompute of the refine list; FP64 only for queries whose entries it
    // cannot separate
    DtwRefineArgs rf;
    rf.Q = q; rf.C = x->cand; rf.L = L; rf.D = D; rf.W = W; rf.N = N;
    rf.pairs = x->refine; rf.count = x->scalars + kRefineCount; rf.d64 = x->refine_d64; rf.best64 = x->bestdf;
    e = x->ref_tab ? dtw_refine_df_gtab_launch(x->R_ref, x->ref_slots, s, rf, x->ref_tab)
                   : dtw_refine_df_launch(x->R_ref, x->blocks_ref, s, rf);
    if (e != cudaSuccess) return e;
    if ((e = launch_refine_amb(x->refine, x->refine_d64, x->scalars + kRefineCount, N, x->bestdf, x->kappa, x->amb,
                               x->best_idx_df, x->sms, s)) != cudaSuccess)
        return e;
    if ((e = launch_refine_need64(x->refine, x->refine_d64, x->scalars + kRefineCount, N, x->bestdf, x->kappa,
                                  x->amb, x->refine64, x->scalars + kRefine64Count, x->refine_cap, x->sms, s)) !=
        cudaSuccess)
        return e;
    DtwRefineArgs r64 = rf;
    r64.pairs = x->refine64; r64.count = x->scalars + kRefine64Count; r64.d64 = x->refine64_d64;
    r64.best64 = x->best64;
    if ((e = dtw_refine_launch(x->R_ref, x->blocks_ref, s, r64)) != cudaSuccess) return e;
    if ((e = launch_refine_pick(x->refine64, x->refine64_d64, x->scalars + kRefine64Count, N, x->best64, x->best_idx,
                                x->sms, s)) != cudaSuccess)
        return e;
    if ((e = launch_count_add(x->counters + kRefined, x->scalars + kRefineCount, s)) != cudaSuccess) return e;
    if ((e = launch_count_add(x->counters + kRefined64, x->scalars + kRefine64Count, s)) != cudaSuccess) return e;
    if ((e = launch_finalize(Mb_cur, x->bestdf, x->best_idx_df, x->amb, x->best64, x->best_idx, idx_out, dist_out,
                             s)) != cudaSuccess)
        return e;
    TC_MARK(10);
    return cudaSuccess;
}

// TC-DTW's data-adaptive choice (Section 6; parameter ranges of Section 7.1): on the
// first call, time the pipeline on up to 32 of its queries with LB_MV alone, LB_TI
// (e_ti in {0.05, 0.1, 0.2}) and LB_PC (e_pc in {0.1, 0.5}, Lq in {2, 3}), each within
// what the caller enabled, and keep the fastest.  Every choice gives the same answer
// (the bounds only decide which DTWs are skipped); the paper picks between its two
// bounds on a few sample series the same way, by trying them.
cudaError_t select_cascade(tcdtw_index *x, const float *q, int64_t M, cudaStream_t s) {
    x->selected = true;
    tcdtw_opts &o = x->opts;
    if (!o.select || o.no_prune || (!o.use_pc && !o.use_ti)) return cudaSuccess;
    const tcdtw_opts given = o;
    const int n = (int)std::min<int64_t>(M, std::min<int64_t>(x->Mb, 32));
    struct Cfg { int pc, ti, Lq; float e_pc, e_ti; };
    std::vector<Cfg> cfgs = {{0, 0, o.Lq, o.e_pc, o.e_ti}};
    if (o.use_ti)
        for (float e : {0.05f, 0.1f, 0.2f}) cfgs.push_back({0, 1, o.Lq, o.e_pc, e});
    if (o.use_pc)
        for (int lq : {2, 3})
            if (pc_key_fits(lq, x->D))
                for (float e : {0.1f, 0.5f}) cfgs.push_back({1, 0, lq, e, o.e_ti});
    int64_t *sidx = nullptr;
    double *sdist = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = dev_malloc((void **)&sidx, sizeof(int64_t) * n);
    if (e == cudaSuccess) e = dev_malloc((void **)&sdist, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const bool prof = x->profile;
    x->profile = false;
    float best_ms = INFINITY;
    Cfg best = cfgs[0];
    for (size_t c = 0; c < cfgs.size() && e == cudaSuccess; ++c) {
        o.use_pc = cfgs[c].pc;
        o.use_ti = cfgs[c].ti;
        o.Lq = cfgs[c].Lq;
        o.e_pc = cfgs[c].e_pc;
        o.e_ti = cfgs[c].e_ti;
        float ms = 0.f;
        e = run_block(x, q, n, sidx, sdist, s);  // warm (tables, caches)
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = run_block(x, q, n, sidx, sdist, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best_ms) { best_ms = ms; best = cfgs[c]; }
    }
    x->profile = prof;
    o.use_pc = best.pc;
    o.use_ti = best.ti;
    o.Lq = best.Lq;
    o.e_pc = best.e_pc;
    o.e_ti = best.e_ti;
    if (e != cudaSuccess) {  // keep the given bounds; the next call chooses again
        o = given;
        x->selected = false;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sidx);
    cudaFree(sdist);
    return e;
}

// All query blocks of one call.  With use_graph, a call of at most one block runs on
// the index's own query and answer buffers (copied in and out on s, outside the graph)
// and a query count seen once before is captured into a CUDA graph (on an internal
// stream) and replayed on s; the first call of a count runs eagerly so that any
// one-time setup (function attributes, lazy module loading) happens outside capture.
// Calls of several blocks run eagerly (each block is a long search already).
cudaError_t run_all_blocks(tcdtw_index *x, const float *q, int64_t M, int64_t *idx, double *dist, cudaStream_t s) {
    const int64_t E = (int64_t)x->L * x->D;
    auto eager = [&](const float *qq, int64_t *ii, double *dd, cudaStream_t st) -> cudaError_t {
        for (int64_t m0 = 0; m0 < M; m0 += x->Mb) {
            const int Mb_cur = (int)((M - m0) < x->Mb ? (M - m0) : x->Mb);
            cudaError_t e = run_block(x, qq + m0 * E, Mb_cur, ii + m0, dd + m0, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    if (!x->opts.use_graph || M > x->Mb || !x->qbuf) return eager(q, idx, dist, s);
    cudaError_t e = cudaMemcpyAsync(x->qbuf, q, sizeof(float) * (size_t)(M * E), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    auto copy_out = [&]() -> cudaError_t {
        cudaError_t e2 = cudaMemcpyAsync(idx, x->idx_buf, sizeof(int64_t) * (size_t)M, cudaMemcpyDeviceToDevice, s);
        if (e2 != cudaSuccess) return e2;
        return cudaMemcpyAsync(dist, x->dist_buf, sizeof(double) * (size_t)M, cudaMemcpyDeviceToDevice, s);
    };
    tcdtw_index::GraphEntry *ent = nullptr;
    for (auto &g : x->graphs)
        if (g.M == M && g.profiled == x->profile) ent = &g;
    if (!ent) {
        if (x->graphs.size() >= 8) {  // drop the least recently used key
            size_t lru = 0;
            for (size_t k = 1; k < x->graphs.size(); ++k)
                if (x->graphs[k].last_use < x->graphs[lru].last_use) lru = k;
            if (x->graphs[lru].exec) cudaGraphExecDestroy(x->graphs[lru].exec);
            x->graphs.erase(x->graphs.begin() + lru);
        }
        x->graphs.push_back({M, 0, nullptr, 0, 0, x->profile, 0});
        ent = &x->graphs.back();
    }
    ent->last_use = ++x->graph_clock;
    if (!ent->exec && ent->seen == 0) {
        ent->seen = 1;
        if ((e = eager(x->qbuf, x->idx_buf, x->dist_buf, s)) != cudaSuccess) return e;
        return copy_out();
    }
    if (!ent->exec) {
        if (!x->cap_stream && (e = cudaStreamCreateWithFlags(&x->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return e;
        // order the capture stream after the caller's prior work on s
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        if ((e = cudaStreamBeginCapture(x->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
        x->marks_used = 0;
        x->capturing = true;
        const uint64_t k0 = tcdtw_kernel_launches();
        cudaError_t run = eager(x->qbuf, x->idx_buf, x->dist_buf, x->cap_stream);
        ent->kernels = (int)(tcdtw_kernel_launches() - k0);
        note_launches(-(int64_t)ent->kernels);  // captured, not launched yet
        x->capturing = false;
        ent->marks = x->marks_used;
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(x->cap_stream, &graph);
        if (run != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return run; }
        if (e != cudaSuccess) return e;
        e = cudaGraphInstantiate(&ent->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { ent->exec = nullptr; return e; }
    }
    x->marks_used = ent->marks;  // the graph records these profiling events
    note_launches(ent->kernels);   // kernels the replay launches
    if ((e = cudaGraphLaunch(ent->exec, s)) != cudaSuccess) return e;
    return copy_out();
}

}  // namespace

extern "C" {

int tcdtw_build(const float *cand, int64_t N, int32_t L, int32_t D, int32_t W, int32_t K, const tcdtw_opts *opts,
                void *stream, tcdtw_index **out) {
    if (!out) return TCDTW_ERR_INVALID;
    *out = nullptr;
    if (!cand) return TCDTW_ERR_INVALID;
    int rc = validate_shape(N, L, D, W, K);
    if (rc) return rc;
    tcdtw_opts o;
    if (opts) o = *opts; else tcdtw_default_opts(&o);
    if (o.P < 1 || o.Lq < 1 || o.w < 1 || o.seed_s < 1 || o.seed_s > 8 || o.qblock < 0) return TCDTW_ERR_INVALID;
    // LB_PC only changes speed: skip it when the cell keys (Lq^D) do not fit 63 bits
    if (o.use_pc && !pc_key_fits(o.Lq, D)) o.use_pc = 0;
    if (W > L - 1) W = L - 1;
    if (o.use_ti && !o.ti_top && !lb_ti_rows_supported(W)) return TCDTW_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    tcdtw_index *x = new (std::nothrow) tcdtw_index();
    if (!x) return TCDTW_ERR_NOMEM;
    x->cand = cand; x->N = N; x->L = L; x->D = D; x->W = W; x->K = K; x->opts = o;
    x->S = (int)(o.seed_s < N ? o.seed_s : N);
    // LB_MV with early abandoning: a spread sample of every pair, then the live pairs' rest
    x->mv_samp = (o.mv_abandon && !o.no_prune) ? lb_mv_sample(L * D, &x->mv_stride) : 0;
    x->S2 = x->mv_samp > 0 ? (int)std::min<int64_t>(x->S, N - x->S) : 0;
    x->sms = num_sms();
    x->G_pc = (L + o.w - 1) / o.w;
    x->ldE = ((int64_t)L * D + 31) / 32 * 32;
    x->rho_ref = prune_rho(L, D);
    x->kappa = refine_kappa(L, D);
    x->rho = o.no_prune ? INFINITY : x->rho_ref;
    if (o.no_prune) { x->opts.use_pc = 0; x->opts.use_ti = 0; x->opts.use_rev = 0; }
    // query block: bounded by the u32 pair ids and by ~4 GB of workspace
    int64_t Mb = o.qblock > 0 ? o.qblock : 256;
    const double per_q = (double)N * 20.0 + (double)x->ldE * 8.0 + (o.use_pc ? (double)x->G_pc * K * 2 * D * 4.0 : 0);
    while (Mb > 1 && per_q * Mb > 4.0e9) Mb >>= 1;
    while (Mb > 1 && (double)Mb * (double)N >= 4.29e9) Mb >>= 1;
    x->Mb = (int)Mb;
    x->Mb_pad = (int)((Mb + 31) / 32 * 32);
    if (o.tile >= 0) {
        if (o.tile >= kNumTiles || kTiles[o.tile].DMAX < D) { free_index(x); return TCDTW_ERR_INVALID; }
        x->tile = o.tile;
        x->G = 0;
        for (int g = 4; g <= 32; g *= 2)
            if (tile_valid(o.tile, g, W)) { x->G = g; break; }
        if (!x->G) { free_index(x); return TCDTW_ERR_INVALID; }
    } else if (!autotune_nn_tile(cand, N, L, D, W, s, &x->tile, &x->G) &&
               !choose_tile((int64_t)x->Mb * 64, L, D, W, 0, &x->tile, &x->G)) {
        free_index(x);
        return TCDTW_ERR_UNSUPPORTED;
    }
    x->R_ref = refine_rows_for(W);
    if (x->R_ref == 0) { free_index(x); return TCDTW_ERR_UNSUPPORTED; }
    x->blocks_nn = dtw_occupancy(x->tile, 1, x->G) * x->sms;
    if (x->blocks_nn < 1) x->blocks_nn = x->sms;
    x->tile_seed = x->tile;
    x->G_seed = x->G;
    for (int t = 0; t < kNumTiles; ++t) {
        if (kTiles[t].DMAX != kTiles[x->tile].DMAX || kTiles[t].R >= kTiles[x->tile_seed].R) continue;
        for (int g = 4; g <= 32; g *= 2)
            if (tile_valid(t, g, W)) {
                x->tile_seed = t;
                x->G_seed = g;
                break;
            }
    }
    x->blocks_seed = dtw_occupancy(x->tile_seed, 1, x->G_seed) * x->sms;
    if (x->blocks_seed < 1) x->blocks_seed = x->sms;
    x->blocks_ref = x->sms * 8;  // one-warp blocks
    rc = alloc_index(x);
    if (rc) { free_index(x); return rc; }
    if (o.check_finite) {
        cudaError_t e = launch_check_finite(cand, N * (int64_t)L * D, x->status, 0, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { free_index(x); return cuda_err(e); }
        DevStatus st;
        if (cudaMemcpy(&st, x->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) {
            free_index(x);
            return TCDTW_ERR_CUDA;
        }
        if (st.code) { free_index(x); return st.code; }
    }
    if (x->opts.use_rev) {
        // candidate-side envelopes for the reverse LB_MV, once per index
        const int64_t E = (int64_t)L * D;
        if (E > INT32_MAX) { free_index(x); return TCDTW_ERR_UNSUPPORTED; }
        rc = dalloc(&x->Uc, (size_t)N * E) == cudaSuccess && dalloc(&x->Lc, (size_t)N * E) == cudaSuccess
                 ? TCDTW_OK
                 : TCDTW_ERR_NOMEM;
        cudaError_t e = cudaSuccess;
        for (int64_t n0 = 0; rc == TCDTW_OK && n0 < N && e == cudaSuccess; n0 += 65535) {
            const int64_t nc = (N - n0) < 65535 ? (N - n0) : 65535;
            e = launch_envelope(cand + n0 * E, nc, L, D, W, x->Uc + n0 * E, x->Lc + n0 * E, (int)E, s);
        }
        if (rc == TCDTW_OK && e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (rc == TCDTW_OK && e != cudaSuccess) rc = cuda_err(e);
        if (rc) { free_index(x); return rc; }
    }
    *out = x;
    return TCDTW_OK;
}

int tcdtw_nn(tcdtw_index *x, const float *q, int64_t M, int64_t *idx, double *dist, tcdtw_stats *stats,
             void *stream) {
    if (!x || M < 0) return TCDTW_ERR_INVALID;
    if (M == 0) {
        if (stats) memset(stats, 0, sizeof(*stats));
        return TCDTW_OK;
    }
    if (!q || !idx || !dist) return TCDTW_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t E = (int64_t)x->L * x->D;
    if (!x->selected) TC_TRY(select_cascade(x, q, M, s));
    const bool sync = stats != nullptr || x->opts.check_finite || x->profile;
    x->marks_used = 0;
    if (sync) {
        TC_TRY(cudaMemsetAsync(x->counters, 0, sizeof(unsigned long long) * kNumCounters, s));
        TC_TRY(cudaMemsetAsync(x->status, 0, sizeof(DevStatus), s));
    }
    TC_TRY(run_all_blocks(x, q, M, idx, dist, s));
    if (!sync) return TCDTW_OK;
    TC_TRY(cudaStreamSynchronize(s));
    if (x->profile) {
        const int per = TCDTW_NUM_STAGES + 1;
        for (int b = 0; b + per <= x->marks_used; b += per) {
            for (int k = 0; k < TCDTW_NUM_STAGES; ++k) {
                float ms = 0.f;
                TC_TRY(cudaEventElapsedTime(&ms, x->events[b + k], x->events[b + k + 1]));
                x->stage_ms[k] += ms;
            }
            ++x->stage_blocks;
        }
    }
    DevStatus st;
    TC_TRY(cudaMemcpy(&st, x->status, sizeof(st), cudaMemcpyDeviceToHost));
    if (st.code) return st.code;
    if (stats) {
        unsigned long long c[kNumCounters];
        TC_TRY(cudaMemcpy(c, x->counters, sizeof(c), cudaMemcpyDeviceToHost));
        uint64_t seeds = 0;
        for (int64_t m0 = 0; m0 < M; m0 += x->Mb)
            seeds += (uint64_t)block_seeds(x, (int)((M - m0) < x->Mb ? (M - m0) : x->Mb));
        stats->pairs = (uint64_t)M * (uint64_t)x->N;
        stats->pruned_mv = c[kPrunedMv] - seeds + c[kPrunedDtw];
        stats->pruned_pc = c[kPrunedPc];
        stats->pruned_ti = c[kPrunedTi];
        stats->pruned_rev = c[kPrunedRev];
        // the dense stream's terms (all of every pair, or the sample of every pair) are
        // counted here; the completion kernel counts its own
        uint64_t dense = 0;
        if (!x->opts.no_prune)
            for (int64_t m0 = 0; m0 < M; m0 += x->Mb) {
                const int mb = (int)((M - m0) < x->Mb ? (M - m0) : x->Mb);
                dense += (uint64_t)mb * (uint64_t)x->N * (uint64_t)(block_abandons(x, mb) ? 32 * x->mv_samp : E);
            }
        stats->mv_terms = dense + c[kMvTerms];
        stats->dtw_started = c[kStarted];
        stats->dtw_abandoned = c[kAbandoned];
        stats->cells = c[kCells];
        stats->refined = c[kRefined];
        stats->refined64 = c[kRefined64];
    }
    return TCDTW_OK;
}

int tcdtw_index_opts(tcdtw_index *x, tcdtw_opts *out) {
    if (!x || !out) return TCDTW_ERR_INVALID;
    *out = x->opts;
    return TCDTW_OK;
}

int tcdtw_index_info(tcdtw_index *x, int32_t *tile, int32_t *G, int32_t *qblock) {
    if (!x) return TCDTW_ERR_INVALID;
    if (tile) *tile = x->tile;
    if (G) *G = x->G;
    if (qblock) *qblock = x->Mb;
    return TCDTW_OK;
}

int tcdtw_set_profiling(tcdtw_index *x, int32_t enable) {
    if (!x) return TCDTW_ERR_INVALID;
    x->profile = enable != 0;
    for (int k = 0; k < TCDTW_NUM_STAGES; ++k) x->stage_ms[k] = 0.0;
    x->stage_blocks = 0;
    return TCDTW_OK;
}

int tcdtw_stage_times(tcdtw_index *x, double *ms, int64_t *blocks) {
    if (!x || !ms) return TCDTW_ERR_INVALID;
    for (int k = 0; k < TCDTW_NUM_STAGES; ++k) ms[k] = x->stage_ms[k];
    if (blocks) *blocks = x->stage_blocks;
    return TCDTW_OK;
}

void tcdtw_free(tcdtw_index *x) {
    if (!x) return;
    cudaDeviceSynchronize();
    free_index(x);
}

// ------------------------------------------------------------------ stage entry points
int tcdtw_envelope(const float *q, int64_t M, int32_t L, int32_t D, int32_t W, float *U, float *Lo, void *stream) {
    if (M < 0 || L < 1 || D < 1 || W < 0) return TCDTW_ERR_INVALID;
    if (M == 0) return TCDTW_OK;
    if (!q || !U || !Lo) return TCDTW_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    for (int64_t m0 = 0; m0 < M; m0 += 65535) {
        const int64_t mc = (M - m0) < 65535 ? (M - m0) : 65535;
        const int64_t off = m0 * L * D;
        TC_TRY(launch_envelope(q + off, mc, L, D, W, U + off, Lo + off, L * D, s));
    }
    return TCDTW_OK;
}

int tcdtw_query_dq(const float *q, int64_t M, int32_t L, int32_t D, float *dq_lo, float *dq_hi, void *stream) {
    if (M < 0 || L < 1 || D < 1) return TCDTW_ERR_INVALID;
    if (M == 0) return TCDTW_OK;
    if (!q || !dq_lo || !dq_hi) return TCDTW_ERR_INVALID;
    return cuda_err(launch_query_dq(q, M, L, D, dq_lo, dq_hi, (cudaStream_t)stream));
}

int tcdtw_pc_boxes(const float *q, int64_t M, int32_t L, int32_t D, int32_t W, int32_t K, int32_t Lq, int32_t w,
                   float *boxes, int32_t *counts, void *stream) {
    if (M < 0 || L < 1 || D < 1 || W < 0 || K < 1 || Lq < 1 || w < 1) return TCDTW_ERR_INVALID;
    if (D > TCDTW_MAX_D) return TCDTW_ERR_UNSUPPORTED;
    if (!pc_key_fits(Lq, D)) return TCDTW_ERR_INVALID;
    if (M == 0) return TCDTW_OK;
    if (!q || !boxes || !counts) return TCDTW_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const int G = (L + w - 1) / w;
    for (int64_t m0 = 0; m0 < M; m0 += 65535) {
        const int64_t mc = (M - m0) < 65535 ? (M - m0) : 65535;
        TC_TRY(launch_pc_boxes(q + m0 * L * D, mc, L, D, W, K, Lq, w, boxes + m0 * G * K * 2 * D, counts + m0 * G,
                               s));
    }
    return TCDTW_OK;
}

int tcdtw_compact(const float *lb, int64_t M, int64_t N, const float *thresh, int32_t *out_idx, int32_t *count,
                  void *stream) {
    if (M < 0 || N < 0) return TCDTW_ERR_INVALID;
    if (M == 0) return TCDTW_OK;
    if (!lb || !thresh || !out_idx || !count) return TCDTW_ERR_INVALID;
    if (N >= (int64_t)1 << 31) return TCDTW_ERR_UNSUPPORTED;
    CompactArgs ca;
    memset(&ca, 0, sizeof(ca));
    ca.lb = lb; ca.M = M; ca.N = N; ca.ldLb = N; ca.thresh = thresh; ca.counts = count; ca.ldOut = N;
    ca.idx_out = out_idx;
    return cuda_err(launch_compact(ca, (cudaStream_t)stream));
}

int tcdtw_lb_mv_abandon(const float *q, int64_t M, const float *c, int64_t N, int32_t L, int32_t D, int32_t W,
                        const float *thresh, float *out, void *stream) {
    if (M < 0 || N < 0 || L < 1 || D < 1 || W < 0) return TCDTW_ERR_INVALID;
    if (D > TCDTW_MAX_D) return TCDTW_ERR_UNSUPPORTED;
    if (M == 0 || N == 0) return TCDTW_OK;
    if (!q || !c || !thresh || !out) return TCDTW_ERR_INVALID;
    if (W > L - 1) W = L - 1;
    if ((double)M * (double)N >= 4.29e9) return TCDTW_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    const int sms = num_sms();
    const int E = L * D;
    int sstride = 1;
    const int samp = lb_mv_sample(E, &sstride);
    const int64_t ldE = ((int64_t)E + 31) / 32 * 32;
    const int64_t Mp = (M + 31) / 32 * 32;
    const int64_t ws_floats = std::min<int64_t>(kMvWsFloats, 64 * M * N);
    const int64_t list_n = samp > 0 ? lb_mv_rest_list_entries(N, (int)std::min<int64_t>(M, kRestQG), sms) : 1;
    float *U = nullptr, *Lo = nullptr, *Up = nullptr, *Lp = nullptr, *ws = nullptr;
    DevStatus *st = nullptr;
    int32_t *cnt = nullptr;
    uint32_t *list = nullptr;
    auto release = [&]() {
        for (void *p : {(void *)U, (void *)Lo, (void *)Up, (void *)Lp, (void *)ws, (void *)st, (void *)cnt,
                        (void *)list})
            cudaFree(p);
    };
    if (dev_malloc((void **)&U, sizeof(float) * Mp * ldE) != cudaSuccess ||
        dev_malloc((void **)&Lo, sizeof(float) * Mp * ldE) != cudaSuccess ||
        dev_malloc((void **)&Up, sizeof(float) * Mp * ldE) != cudaSuccess ||
        dev_malloc((void **)&Lp, sizeof(float) * Mp * ldE) != cudaSuccess ||
        dev_malloc((void **)&st, sizeof(DevStatus)) != cudaSuccess ||
        dev_malloc((void **)&ws, sizeof(float) * ws_floats) != cudaSuccess ||
        dev_malloc((void **)&cnt, sizeof(int32_t) * kMvTileCounters) != cudaSuccess ||
        dev_malloc((void **)&list, sizeof(uint32_t) * list_n) != cudaSuccess) {
        release();
        return TCDTW_ERR_NOMEM;
    }
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * kMvTileCounters, s);
    for (int64_t m0 = 0; m0 < M && e == cudaSuccess; m0 += 65534) {  // even chunks keep the pair layout
        const int64_t mc = (M - m0) < 65534 ? (M - m0) : 65534;
        e = launch_envelope_pairs_plain(q + m0 * E, mc, L, D, W, U + m0 * ldE, Lo + m0 * ldE, Up + m0 * ldE,
                                        Lp + m0 * ldE, (int)ldE, s);
    }
    if (e == cudaSuccess) {  // the sample of every pair (all of it without a sample)
        LbMvArgs mv;
        mv.cand = c; mv.N = N; mv.E = samp > 0 ? 32 * samp : E; mv.cstride = sstride; mv.Erow = E; mv.ldC = E;
        mv.U = U; mv.Lo = Lo; mv.ldE = ldE;
        mv.Mb = (int)M; mv.lb = out; mv.ldLb = N; mv.sms = sms; mv.status = st;
        mv.ws = ws; mv.ws_floats = ws_floats; mv.tile_cnt = cnt; mv.tile_cnt_cap = kMvTileCounters;
        e = launch_lb_mv(mv, s);
    }
    if (e == cudaSuccess && samp > 0) {  // the rest of the pairs still under their threshold
        LbMvRestArgs ra;
        ra.cand = c; ra.N = N; ra.E = E; ra.samp = samp; ra.sstride = sstride; ra.ldC = E; ra.Up = Up; ra.Lp = Lp; ra.ldP = ldE;
        ra.Mb = (int)M; ra.lb = out; ra.ldLb = N; ra.thresh = thresh; ra.bsf = nullptr; ra.rho = 1.f;
        ra.list = list; ra.list_entries = list_n; ra.sms = sms; ra.status = st;
        e = launch_lb_mv_rest(ra, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int rc = cuda_err(e);
    if (rc == TCDTW_OK) {
        DevStatus h;
        rc = cuda_err(cudaMemcpy(&h, st, sizeof(h), cudaMemcpyDeviceToHost));
        if (rc == TCDTW_OK && h.code) rc = h.code;
    }
    release();
    return rc;
}

int tcdtw_lower_bounds(const float *q, int64_t M, const float *c, int64_t N, int32_t L, int32_t D, int32_t W,
                       int32_t K, const tcdtw_opts *opts, int32_t which, float *out, void *stream) {
    if (M < 0 || N < 0 || L < 1 || D < 1 || W < 0 || K < 1) return TCDTW_ERR_INVALID;
    if (which < TCDTW_LB_MV || which > TCDTW_LB_MV_REV) return TCDTW_ERR_INVALID;
    if (D > TCDTW_MAX_D) return TCDTW_ERR_UNSUPPORTED;
    if (M == 0 || N == 0) return TCDTW_OK;
    if (!q || !c || !out) return TCDTW_ERR_INVALID;
    tcdtw_opts o;
    if (opts) o = *opts; else tcdtw_default_opts(&o);
    if (which == TCDTW_LB_PC && !pc_key_fits(o.Lq, D)) return TCDTW_ERR_INVALID;
    if (which == TCDTW_LB_TI && !o.ti_top && !lb_ti_rows_supported(W < L - 1 ? W : L - 1))
        return TCDTW_ERR_UNSUPPORTED;
    if (o.P < 1 || o.Lq < 1 || o.w < 1) return TCDTW_ERR_INVALID;
    if (W > L - 1) W = L - 1;
    if ((double)M * (double)N >= 4.29e9) return TCDTW_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    const int sms = num_sms();
    const int E = L * D;
    int rc = TCDTW_OK;
    if (which == TCDTW_LB_MV) {
        const int64_t ldE = ((int64_t)E + 31) / 32 * 32;
        const int64_t Mp = (M + 31) / 32 * 32;
        float *U = nullptr, *Lo = nullptr;
        DevStatus *st = nullptr;
        float *ws = nullptr;
        int32_t *cnt = nullptr;
        const int64_t ws_floats = std::min<int64_t>(kMvWsFloats, 64 * M * N);
        auto release = [&]() {
            cudaFree(U);
            cudaFree(Lo);
            cudaFree(st);
            cudaFree(ws);
            cudaFree(cnt);
        };
        if (dev_malloc((void **)&U, sizeof(float) * Mp * ldE) != cudaSuccess ||
            dev_malloc((void **)&Lo, sizeof(float) * Mp * ldE) != cudaSuccess ||
            dev_malloc((void **)&st, sizeof(DevStatus)) != cudaSuccess || dev_malloc((void **)&ws, sizeof(float) * ws_floats) != cudaSuccess ||
            dev_malloc((void **)&cnt, sizeof(int32_t) * kMvTileCounters) != cudaSuccess) {
            release();
            return TCDTW_ERR_NOMEM;
        }
        cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * kMvTileCounters, s);
        for (int64_t m0 = 0; m0 < M && e == cudaSuccess; m0 += 65534) {  // even chunks keep the pair layout
            const int64_t mc = (M - m0) < 65534 ? (M - m0) : 65534;
            e = launch_envelope_pairs(q + m0 * E, mc, L, D, W, U + m0 * ldE, Lo + m0 * ldE, (int)ldE, s);
        }
        if (e == cudaSuccess) {
            LbMvArgs mv;
            mv.cand = c; mv.N = N; mv.E = E; mv.U = U; mv.Lo = Lo; mv.ldE = ldE; mv.Mb = (int)M; mv.lb = out;
            mv.ldLb = N; mv.sms = sms; mv.status = st;
            mv.ws = ws; mv.ws_floats = ws_floats; mv.tile_cnt = cnt; mv.tile_cnt_cap = kMvTileCounters;
            e = launch_lb_mv(mv, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        rc = cuda_err(e);
        if (rc == TCDTW_OK) {
            DevStatus h;
            rc = cuda_err(cudaMemcpy(&h, st, sizeof(h), cudaMemcpyDeviceToHost));
            if (rc == TCDTW_OK && h.code) rc = h.code;
        }
        release();
        return rc;
    }
    // LB_PC / LB_TI: every pair listed once, no gate (e = -1), threshold +inf
    const int64_t P = M * N;
    uint32_t *pairs = nullptr;
    unsigned long long *bsf = nullptr;
    float *aux1 = nullptr, *aux2 = nullptr;
    int32_t *cnts = nullptr;
    cudaError_t e = dev_malloc((void **)&pairs, sizeof(uint32_t) * P);
    if (e == cudaSuccess) e = dev_malloc((void **)&bsf, sizeof(unsigned long long) * M);
    if (e == cudaSuccess) e = launch_iota_pairs(pairs, P, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, sizeof(float) * P, s);
    if (e == cudaSuccess) e = launch_init_block(M, bsf, nullptr, nullptr, nullptr, nullptr, nullptr, s);
    PairListArgs pl;
    pl.Q = q; pl.C = c; pl.L = L; pl.D = D; pl.W = W; pl.pairs = pairs; pl.count = nullptr; pl.n_static = P;
    pl.N = N; pl.lb = out;
    const float rho = 1.0f;
    if (which == TCDTW_LB_PC) {
        const int G = (L + o.w - 1) / o.w;
        if (e == cudaSuccess) e = dev_malloc((void **)&aux1, sizeof(float) * M * G * K * 2 * D);
        if (e == cudaSuccess) e = dev_malloc((void **)&cnts, sizeof(int32_t) * M * G);
        for (int64_t m0 = 0; m0 < M && e == cudaSuccess; m0 += 65535) {
            const int64_t mc = (M - m0) < 65535 ? (M - m0) : 65535;
            e = launch_pc_boxes(q + m0 * E, mc, L, D, W, K, o.Lq, o.w, aux1 + m0 * G * K * 2 * D, cnts + m0 * G, s);
        }
        if (e == cudaSuccess) e = launch_lb_pc_list(pl, aux1, cnts, K, o.w, bsf, rho, -1.0f, nullptr, P, sms, s);
    } else if (which == TCDTW_LB_MV_REV) {
        // envelopes of the candidates, then every pair's reverse bound
        if (e == cudaSuccess) e = dev_malloc((void **)&aux1, sizeof(float) * N * E);
        if (e == cudaSuccess) e = dev_malloc((void **)&aux2, sizeof(float) * N * E);
        for (int64_t n0 = 0; n0 < N && e == cudaSuccess; n0 += 65535) {
            const int64_t nc = (N - n0) < 65535 ? (N - n0) : 65535;
            e = launch_envelope(c + n0 * E, nc, L, D, W, aux1 + n0 * E, aux2 + n0 * E, E, s);
        }
        if (e == cudaSuccess) e = launch_lb_rev_list(pl, aux1, aux2, nullptr, rho, nullptr, P, sms, s);
    } else {
        if (e == cudaSuccess) e = dev_malloc((void **)&aux1, sizeof(float) * M * L);
        if (e == cudaSuccess) e = dev_malloc((void **)&aux2, sizeof(float) * M * L);
        if (e == cudaSuccess) e = launch_query_dq(q, M, L, D, aux1, aux2, s);
        if (e == cudaSuccess)
            e = o.ti_top ? launch_lb_ti_list(pl, aux1, aux2, o.P, bsf, rho, -1.0f, nullptr, P, sms, s)
                         : launch_lb_ti_rows_list(pl, aux1, aux2, o.P, bsf, rho, -1.0f, nullptr, P, sms, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    rc = cuda_err(e);
    cudaFree(pairs); cudaFree(bsf); cudaFree(aux1); cudaFree(aux2); cudaFree(cnts);
    return rc;
}

}  // extern "C"
