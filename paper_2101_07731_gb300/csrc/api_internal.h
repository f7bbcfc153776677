// api_internal.h -- helpers shared by the host-side API translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tc {
int num_sms();
int dmax_for(int D);
bool tile_valid(int tile, int G, int W);
bool choose_tile(int64_t P, int L, int D, int W, int need_div, int *tile, int *G);
int blocks_for(int tile, int which, int64_t groups, int G);
int ckpt_rows(int L, int W);
int64_t ckpt_floats(int64_t P, int L, int W);
int cuda_err(cudaError_t e);
// Every device allocation of the library: cudaMalloc, unless a failure was injected
// with tcdtw_inject_alloc_failure (then cudaErrorMemoryAllocation, nothing allocated).
cudaError_t dev_malloc(void **p, size_t bytes);
const char *last_detail();
float prune_rho(int L, int D);
double refine_kappa(int L, int D);
bool pc_key_fits(int Lq, int D);
// The single-set DTW tuner: the fastest valid (tile, G) for (L, D, W), timed on pairs of
// the given candidates; cached per shape (and in the TCDTW_TUNE_CACHE file when set).
bool autotune_nn_tile(const float *cand, int64_t N, int L, int D, int W, cudaStream_t s, int *tile, int *G);
}  // namespace tc
