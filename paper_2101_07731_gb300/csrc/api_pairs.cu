// api_pairs.cu -- C ABI: error strings, options, tile table, and the
// differentiable DTW distance of independent pairs (forward with band-row
// checkpoints, and the path adjoint).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include "api_internal.h"
#include "common.cuh"
#include "dtw_tiles.cuh"

#include <atomic>

namespace tc {

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(int64_t n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

int dmax_bucket_ok(int tile, int D) { return kTiles[tile].DMAX >= D; }

// Smallest DMAX bucket that holds D.
int dmax_for(int D) {
    int best = 1 << 30;
    for (int t = 0; t < kNumTiles; ++t)
        if (kTiles[t].DMAX >= D && kTiles[t].DMAX < best) best = kTiles[t].DMAX;
    return best == (1 << 30) ? -1 : best;
}

bool tile_valid(int tile, int G, int W) {
    const int R = kTiles[tile].R;
    return G * (R + 1) >= 2 * W + R;
}

// Estimated cost of computing P pairs with (tile, G): time steps per pair times
// issue slots per lane-step, times the share of a warp a pair occupies, with a
// floor for too little parallelism (too few warps to fill the SMs).
double tile_cost(int tile, int G, int64_t P, int L, int W) {
    const int R = kTiles[tile].R, DM = kTiles[tile].DMAX;
    const double steps = (double)L + (L + R - 1) / R;
    const double per_step = R * (2.0 * DM + 4.0) + DM + 16.0;
    const double warps = (double)P * G / 32.0;
    const double fill = (double)num_sms() * 8.0;  // warps needed to hide latency
    const double waves = warps < fill ? 1.0 : warps / fill;
    (void)W;
    return steps * per_step * waves * (R * DM > 96 ? 1.5 : 1.0);
}

// Deterministic tile choice: among tiles of the smallest DMAX bucket holding D,
// and G in {4, 8, 16, 32} satisfying the no-overlap rule, minimise tile_cost.
// `need_div` (if > 0) restricts to R dividing it (checkpoint segments).
bool choose_tile(int64_t P, int L, int D, int W, int need_div, int *tile, int *G) {
    const int dm = dmax_for(D);
    if (dm < 0) return false;
    double best = 1e300;
    bool found = false;
    for (int t = 0; t < kNumTiles; ++t) {
        if (kTiles[t].DMAX != dm) continue;
        if (need_div > 0 && need_div % kTiles[t].R != 0) continue;
        for (int g = 4; g <= 32; g *= 2) {
            if (!tile_valid(t, g, W)) continue;
            double c = tile_cost(t, g, P, L, W);
            if (c < best) { best = c; *tile = t; *G = g; found = true; }
        }
    }
    if (!found) {  // try wider DMAX buckets (more registers, still correct)
        for (int t = 0; t < kNumTiles; ++t) {
            if (kTiles[t].DMAX < D) continue;
            if (need_div > 0 && need_div % kTiles[t].R != 0) continue;
            for (int g = 4; g <= 32; g *= 2) {
                if (!tile_valid(t, g, W)) continue;
                double c = tile_cost(t, g, P, L, W) * (double)kTiles[t].DMAX / dm;
                if (c < best) { best = c; *tile = t; *G = g; found = true; }
            }
        }
    }
    return found;
}

int blocks_for(int tile, int which, int64_t groups, int G) {
    int occ = dtw_occupancy(tile, which, G);
    if (occ <= 0) occ = 1;
    const int64_t gpb = 128 / G;
    int64_t need = (groups + gpb - 1) / gpb;
    int64_t cap = (int64_t)occ * num_sms();
    if (need > cap) need = cap;
    return (int)(need < 1 ? 1 : need);
}

// Checkpoint segment height: rows per recomputed segment in the backward pass.
// 48 is divisible by every R of the compiled tiles that can serve it (2, 4, 6, 8,
// 16); smaller when the shared-memory segment (C+1)*(2W+1) floats gets too big.
int ckpt_rows(int L, int W) {
    (void)L;
    const int BW = 2 * W + 1;
    const int cands[] = {48, 24, 16, 8, 4, 2};
    for (int c : cands)
        if ((size_t)(c + 1) * BW * sizeof(float) <= 48 * 1024) return c;
    return 2;
}

int64_t ckpt_floats(int64_t P, int L, int W) {
    const int C = ckpt_rows(L, W);
    const int nck = (L + C - 1) / C - 1;
    return P * (int64_t)nck * (2 * W + 1);
}

// Last CUDA error seen by this thread (name and message), for tcdtw_last_error_detail.
static thread_local char g_last_detail[256];

int cuda_err(cudaError_t e) {
    if (e == cudaSuccess) return TCDTW_OK;
    snprintf(g_last_detail, sizeof(g_last_detail), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return TCDTW_ERR_NOMEM;
    return TCDTW_ERR_CUDA;
}

const char *last_detail() { return g_last_detail; }

// Allocation-failure injection on the host (tcdtw_inject_alloc_failure): how many more
// device allocations may succeed, or -1 for no limit.
static std::atomic<int64_t> g_alloc_allow{-1};

cudaError_t dev_malloc(void **p, size_t bytes) {
    *p = nullptr;
    int64_t a = g_alloc_allow.load();
    while (a >= 0) {
        if (a == 0) return cudaErrorMemoryAllocation;
        if (g_alloc_allow.compare_exchange_weak(a, a - 1)) break;
    }
    return cudaMalloc(p, bytes);
}

}  // namespace tc

using namespace tc;

extern "C" {

void tcdtw_default_opts(tcdtw_opts *o) {
    if (!o) return;
    o->P = 5;
    o->Lq = 2;
    o->w = 6;
    o->e_pc = 0.1f;
    o->e_ti = 0.1f;
    o->use_pc = 1;
    o->use_ti = 1;
    o->seed_s = 4;
    o->qblock = 0;
    o->tile = -1;
    o->check_finite = 1;
    o->no_prune = 0;
    o->use_graph = 1;
    o->select = 1;
    o->use_rev = 0;
    o->ti_top = 1;
    o->mv_abandon = 1;
}

const char *tcdtw_strerror(int code) {
    switch (code) {
        case TCDTW_OK: return "ok";
        case TCDTW_ERR_INVALID: return "invalid argument";
        case TCDTW_ERR_NOMEM: return "out of device memory";
        case TCDTW_ERR_CUDA: return "CUDA error";
        case TCDTW_ERR_TIMEOUT: return "device wait timed out";
        case TCDTW_ERR_NONFINITE: return "non-finite value (NaN or Inf) in an input series";
        case TCDTW_ERR_UNSUPPORTED: return "shape not supported by the compiled kernels";
        default: return "unknown error";
    }
}

int tcdtw_tile_count(void) { return kNumTiles; }

const char *tcdtw_last_error_detail(void) { return last_detail(); }

int tcdtw_inject_alloc_failure(int64_t after) {
    if (after < -1) return TCDTW_ERR_INVALID;
    g_alloc_allow.store(after);
    return TCDTW_OK;
}

uint64_t tcdtw_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int tcdtw_tile_info(int32_t t, int32_t *G, int32_t *R, int32_t *maxD) {
    if (t < 0 || t >= kNumTiles) return TCDTW_ERR_INVALID;
    if (G) *G = 0;  // run-time choice
    if (R) *R = kTiles[t].R;
    if (maxD) *maxD = kTiles[t].DMAX;
    return TCDTW_OK;
}

int tcdtw_dtw_pairs_ckpt_bytes(int64_t P, int32_t L, int32_t D, int32_t W, int64_t *bytes) {
    if (!bytes || P < 0 || L < 1 || D < 1 || W < 0) return TCDTW_ERR_INVALID;
    if (W > L - 1) W = L - 1;
    *bytes = ckpt_floats(P, L, W) * (int64_t)sizeof(float);
    return TCDTW_OK;
}

int tcdtw_dtw_pairs(const float *A, const float *B, int64_t P, int32_t L, int32_t D, int32_t W, float *dist,
                    void *ckpt, int64_t ckpt_bytes, void *stream) {
    if (P < 0 || L < 1 || D < 1 || W < 0) return TCDTW_ERR_INVALID;
    if (P == 0) return TCDTW_OK;
    if (!A || !B || !dist) return TCDTW_ERR_INVALID;
    if (D > TCDTW_MAX_D) return TCDTW_ERR_UNSUPPORTED;
    if (W > L - 1) W = L - 1;
    const int C = ckpt_rows(L, W);
    if (ckpt) {
        if (ckpt_bytes < ckpt_floats(P, L, W) * (int64_t)sizeof(float)) return TCDTW_ERR_INVALID;
    }
    int tile = 0, G = 32;
    if (!choose_tile(P, L, D, W, ckpt ? C : 0, &tile, &G)) return TCDTW_ERR_UNSUPPORTED;
    const int blocks = blocks_for(tile, 0, P, G);
    cudaStream_t s = (cudaStream_t)stream;
    return cuda_err(dtw_pairs_launch(tile, G, blocks, s, A, B, P, L, D, W, dist, (float *)ckpt, C));
}

int tcdtw_dtw_pairs_backward(const float *A, const float *B, const void *ckpt, int64_t ckpt_bytes,
                             const float *grad_dist, int64_t P, int32_t L, int32_t D, int32_t W, float *gA,
                             float *gB, void *stream) {
    if (P < 0 || L < 1 || D < 1 || W < 0) return TCDTW_ERR_INVALID;
    if (P == 0) return TCDTW_OK;
    if (!A || !B || !grad_dist || !gA || !gB) return TCDTW_ERR_INVALID;
    if (D > TCDTW_MAX_D) return TCDTW_ERR_UNSUPPORTED;
    if (W > L - 1) W = L - 1;
    const int C = ckpt_rows(L, W);
    const int64_t need = ckpt_floats(P, L, W) * (int64_t)sizeof(float);
    if (need > 0 && (!ckpt || ckpt_bytes < need)) return TCDTW_ERR_INVALID;
    int tile = 0, G = 32;
    if (!choose_tile(P, L, D, W, C, &tile, &G)) return TCDTW_ERR_UNSUPPORTED;
    if (G < 4) G = 4;
    const size_t per_group = (size_t)(C + 1) * (2 * W + 1) * sizeof(float);
    int gpb = 128 / G;
    while (gpb > 1 && per_group * gpb > 200 * 1024) gpb >>= 1;
    if (per_group * gpb > 220 * 1024) return TCDTW_ERR_UNSUPPORTED;
    // the kernel derives groups per block from blockDim
    const int64_t groups = P;
    int64_t blocks = (groups + gpb - 1) / gpb;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    cudaStream_t s = (cudaStream_t)stream;
    // launch with gpb*G threads per block
    return cuda_err(dtw_backward_launch(tile, G, (int)blocks, per_group * gpb, s, A, B, (const float *)ckpt, C,
                                        grad_dist, P, L, D, W, gA, gB, gpb * G));
}

}  // extern "C"
