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
// rho = +inf disables pruning (the threshold is +inf even when the best is 0).
__device__ __forceinline__ float prune_threshold(unsigned long long key, float rho) {
    return rho == __int_as_float(0x7f800000) ? rho : __fmul_ru(best_dist(key), rho);
}

// ---------------------------------------------------------------- packed FP32 pairs
typedef unsigned long long f2;  // two floats: low word first
__device__ __forceinline__ f2 pk(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// ---------------------------------------------------------------- three-way min/max
__device__ __forceinline__ float fmin3(float a, float b, float c) { return fminf(fminf(a, b), c); }
__device__ __forceinline__ float fmax3(float a, float b, float c) { return fmaxf(fmaxf(a, b), c); }

// ---------------------------------------------------------------- launch helpers
inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Host-side count of kernel launches issued by the library (tcdtw_kernel_launches).
void note_launch();
void note_launches(int64_t n);  // graph replays: kernels in the replayed graph

}  // namespace tc

