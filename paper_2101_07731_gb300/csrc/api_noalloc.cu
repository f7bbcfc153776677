// api_noalloc.cu -- LB_MV of every (query, candidate) pair without any device
// allocation.  tcdtw_lower_bounds(TCDTW_LB_MV) allocates its envelope scratch with
// cudaMalloc on every call; this entry point runs the same two kernels (envelope,
// LB_MV stream) with the scratch taken from a fixed array that is part of the
// loaded library instead, for callers that must not allocate device memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "api_internal.h"
#include "common.cuh"
#include "lb_kernels.cuh"

using namespace tc;

namespace {

// Capacity of each of the two envelope halves (U and Lo), in floats: 4 MiB each,
// 8 MiB in all.  Every device that loads the library keeps this array until exit.
constexpr int64_t kEnvFloats = (int64_t)1 << 20;
static __device__ __align__(256) float g_env_scratch[2 * kEnvFloats];

// Device address of g_env_scratch, resolved once per device with that device current
// (in host code the symbol is only a host-side stand-in, not a device address).
constexpr int kMaxDevices = 64;
static float *g_env_ptr[kMaxDevices];
static std::mutex g_env_mutex;

cudaError_t scratch_of_current_device(float **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_env_mutex);
    if (!g_env_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_env_scratch);
        if (e != cudaSuccess) return e;
        g_env_ptr[dev] = (float *)p;
    }
    *out = g_env_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int tcdtw_lb_mv_noalloc(const float *q, int64_t M, const float *c, int64_t N, int32_t L, int32_t D,
                                   int32_t W, float *out, void *stream) {
    if (M < 0 || N < 0 || L < 1 || D < 1 || W < 0) return TCDTW_ERR_INVALID;
    if (M == 0 || N == 0) return TCDTW_OK;
    if (!q || !c || !out) return TCDTW_ERR_INVALID;
    if (W > L - 1) W = L - 1;
    // the envelope of the M queries in the query-pair interleaved layout of the LB_MV
    // stream: ceil(M/2) pairs x ldE elements x 2 floats per half
    const int64_t ldE = ((int64_t)L * D + 31) / 32 * 32;
    const int64_t need = (M + 1) / 2 * 2 * ldE;
    if (need > kEnvFloats) return TCDTW_ERR_UNSUPPORTED;  // beyond the static scratch
    float *env = nullptr;
    cudaError_t e = scratch_of_current_device(&env);
    if (e != cudaSuccess) return cuda_err(e);
    float *U = env, *Lo = env + kEnvFloats;
    cudaStream_t s = (cudaStream_t)stream;
    e = launch_envelope_pairs(q, M, L, D, W, U, Lo, (int)ldE, s);
    if (e != cudaSuccess) return cuda_err(e);
    LbMvArgs mv;
    mv.cand = c;
    mv.N = N;
    mv.E = L * D;
    mv.U = U;
    mv.Lo = Lo;
    mv.ldE = ldE;
    mv.Mb = (int)M;
    mv.lb = out;
    mv.ldLb = N;
    mv.sms = num_sms();
    return cuda_err(launch_lb_mv(mv, s));
}
