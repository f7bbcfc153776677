// common.cuh -- definitions shared by the libtcdtw kernels and the host API.
// (Internal; the public interface is include/tcdtw.h.)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tcdtw.h"

#define TC_INF __int_as_float(0x7f800000)

namespace tc {

constexpr int kWarp = 32;

// ---------------------------------------------------------------- device error flag
// Kernels never trap: they record the first error code here and return.
struct DevStatus {
    int code;    // TCDTW_OK or an error code
    int where;   // kernel-specific detail (e.g. which wait gave up)
};

__device__ __forceinline__ void set_error(DevStatus *st, int code, int where) {
    if (st && atomicCAS(&st->code, 0, code) == 0) st->where = where;
}

// ---------------------------------------------------------------- packed best-so-far
// Per query a 64-bit key (float bits of the FP32 DTW << 32 | candidate index).  For
// non-negative floats the bit pattern orders like the value, so atomicMin keeps the
// smallest distance and, among equal distances, the smallest index.
__device__ __forceinline__ unsigned long long pack_best(float d, uint32_t idx) {
    return ((unsigned long long)__float_as_uint(d) << 32) | idx;
}
__device__ __forceinline__ float best_dist(unsigned long long key) {
    return __uint_as_float((uint32_t)(key >> 32));
}
__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p) {
    return *(const volatile unsigned long long *)p;
}

// Pruning threshold: any candidate whose FP32 DTW exceeds bsf*rho, or whose
// rounded-down lower bound exceeds it, cannot be the exact nearest neighbour
// (rho covers the FP32 DTW rounding error both ways and an FP64 margin).
__device__ __forceinline__ float prune_threshold(unsigned long long key, float rho) {
    return __fmul_ru(best_dist(key), rho);
}

// ---------------------------------------------------------------- three-way min/max
__device__ __forceinline__ float fmin3(float a, float b, float c) { return fminf(fminf(a, b), c); }
__device__ __forceinline__ float fmax3(float a, float b, float c) { return fmaxf(fmaxf(a, b), c); }

// ---------------------------------------------------------------- launch helpers
inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace tc

// ---------------------------------------------------------------- host-side launchers
// Each kernel translation unit exports plain host functions that the API file calls.
namespace tc {

struct Workspace;  // defined in api.cu

// prep.cu
cudaError_t launch_check_finite(const float *x, int64_t n, DevStatus *st, int where, cudaStream_t s);
cudaError_t launch_envelope(const float *q, int64_t M, int L, int D, int W, float *U, float *Lo,
                            int ldE, cudaStream_t s);
cudaError_t launch_query_dq(const float *q, int64_t M, int L, int D, float *dq_lo, float *dq_hi,
                            cudaStream_t s);
cudaError_t launch_pc_boxes(const float *q, int64_t M, int L, int D, int W, int K, int Lq, int w,
                            float *boxes, int32_t *counts, cudaStream_t s);

// lb.cu
struct LbMvArgs {
    const float *cand;    // [N][E]   (E = L*D)
    int64_t N;
    int E;                // elements per series
    const float *U;       // [Mb][ldE] envelope upper (padded with +inf)
    const float *Lo;      // [Mb][ldE] envelope lower (padded with -inf)
    int ldE;              // padded row stride of U/Lo (multiple of 32)
    int Mb;               // queries in the block
    float *lb;            // [Mb][ldLb] output, rounded down
    int64_t ldLb;
};
cudaError_t launch_lb_mv(const LbMvArgs &a, const void *tmap /* CUtensorMap or null */,
                         cudaStream_t s);
bool lb_mv_can_tma(const float *cand, int64_t N, int E);
cudaError_t make_lb_mv_tmap(const float *cand, int64_t N, int E, void *tmap_out /*128B*/);

// Tight bounds for listed pairs (query m, candidate n) -> out[e] (rounded down).
struct PairListArgs {
    const float *Q;       // [Mb][L][D]
    const float *C;       // [N][L][D]
    int L, D, W;
    const uint32_t *pairs;   // entry e: m * N + n
    const int32_t *count;    // device count of entries (or null: use n_static)
    int64_t n_static;
    int64_t N;
    float *lb;               // in/out per entry
};
cudaError_t launch_lb_pc_list(const PairListArgs &a, const float *boxes, const int32_t *counts,
                              int K, int w, int G, const unsigned long long *bsf, float rho,
                              const float *e_gate, float *lb_mv_in, cudaStream_t s);
cudaError_t launch_lb_ti_list(const PairListArgs &a, const float *dq_lo, const float *dq_hi, int P,
                              const unsigned long long *bsf, float rho, const float *e_gate,
                              float *lb_mv_in, cudaStream_t s);

cudaError_t launch_compact_rows(const float *lb, int64_t M, int64_t N, int64_t ldLb,
                                const float *thresh, int32_t *out_idx, int64_t ldOut, int32_t *count,
                                cudaStream_t s);

}  // namespace tc
