// tma.cuh -- device helpers for bulk-tensor (TMA) pipelines: mbarriers with bounded
// waits, 2-D tensor copies into shared memory; and the host-side tensor-map encoder.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tc {

// 2-D FP32 tensor map: rows of `width` floats `pitch` bytes apart, box [box_h][box_w]
// (lb_tma.cu); false when the driver entry point is missing or the encoder refuses.
bool encode_2d(CUtensorMap *m, const float *ptr, uint64_t width, uint64_t height, uint64_t pitch, uint32_t box_w,
               uint32_t box_h, CUtensorMapSwizzle swz);
typedef PFN_cuTensorMapEncodeTiled_v12000 EncodeFn;
EncodeFn encode_fn();

namespace {

constexpr uint64_t kWaitNs = 2000000000ull;  // a bounded wait gives up after ~2 s by default
constexpr uint32_t kWaitIters = 1u << 28;    // and after this many polls in any case

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of parity `parity` of the barrier; false when it gives up
// (time or poll limit, or *abort set by another thread of the CTA; abort may be null).
__device__ __noinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity, const volatile int *abort,
                                            uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1; it < kWaitIters; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63) == 0 && ((abort && *abort) || global_ns() - t0 > limit_ns)) return false;
    }
    return false;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int *abort,
                                          uint64_t limit_ns) {
    return mbar_try(bar, parity) || mbar_wait_slow(bar, parity, abort, limit_ns);
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

}  // namespace
}  // namespace tc
