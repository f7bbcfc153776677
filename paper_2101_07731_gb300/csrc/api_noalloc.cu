// api_noalloc.cu -- LB_MV of every (query, candidate) pair without any device
// allocation.  tcdtw_lower_bounds(TCDTW_LB_MV) allocates its envelope scratch with
// cudaMalloc on every call; this entry point runs the same two kernels (envelope,
// LB_MV stream) with the scratch taken from a fixed array that is part of the
// loaded library instead, for callers that must not allocate device memory.
#include <cuda.h>
#include <cudaTypedefs.h>
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

// Device address of g_env_scratch, resolved with the device current (in host code the
// symbol is only a host-side stand-in, not a device address).  It is resolved on the
// first call on a device and again whenever that device's current context differs from
// the one it was resolved in (after cudaDeviceReset the module is loaded anew, possibly
// at another address); resolving allocates nothing.
constexpr int kMaxDevices = 64;
struct ScratchAddr {
    CUcontext ctx;
    float *ptr;
};
static ScratchAddr g_env[kMaxDevices];
static std::mutex g_env_mutex;

typedef PFN_cuCtxGetCurrent_v4000 CtxGetCurrentFn;

CtxGetCurrentFn ctx_get_current_fn() {
    static const CtxGetCurrentFn fn = []() -> CtxGetCurrentFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(p);
    }();
    return fn;
}

cudaError_t scratch_of_current_device(float **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    CtxGetCurrentFn get_ctx = ctx_get_current_fn();
    if (!get_ctx) return cudaErrorInitializationError;
    CUcontext ctx = nullptr;
    if (get_ctx(&ctx) != CUDA_SUCCESS) return cudaErrorInitializationError;
    std::lock_guard<std::mutex> lock(g_env_mutex);
    if (!ctx || !g_env[dev].ptr || g_env[dev].ctx != ctx) {
        // (also makes the device's primary context current if no context was yet)
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_env_scratch);
        if (e != cudaSuccess) return e;
        if (!ctx && get_ctx(&ctx) != CUDA_SUCCESS) return cudaErrorInitializationError;
        g_env[dev].ctx = ctx;
        g_env[dev].ptr = (float *)p;
    }
    *out = g_env[dev].ptr;
    return cudaSuccess;
}

}  // namespace

extern "C" int tcdtw_lb_mv_noalloc(const float *q, int64_t M, const float *c, int64_t N, int32_t L, int32_t D,
                                   int32_t W, float *out, void *stream) {
    // the same argument checks, in the same order, as tcdtw_lower_bounds(TCDTW_LB_MV)
    if (M < 0 || N < 0 || L < 1 || D < 1 || W < 0) return TCDTW_ERR_INVALID;
    if (D > TCDTW_MAX_D) return TCDTW_ERR_UNSUPPORTED;
    if (M == 0 || N == 0) return TCDTW_OK;
    if (!q || !c || !out) return TCDTW_ERR_INVALID;
    if (W > L - 1) W = L - 1;
    if ((double)M * (double)N >= 4.29e9) return TCDTW_ERR_UNSUPPORTED;
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
