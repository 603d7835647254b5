// Asynchronous-copy glue shared by the pipelined kernels: mbarrier
// initialisation, transaction counts and bounded waits, and the 1-D bulk
// copy of the Tensor Memory Accelerator (cp.async.bulk, global -> shared,
// completing on an mbarrier).  Every wait gives up after a bounded number of
// clock cycles and reports it, so that no kernel can spin forever.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr long long VP_WAIT_CYCLES = 1LL << 32;   // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait on the phase of the given parity; false when it gave up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit = VP_WAIT_CYCLES) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
// global -> shared bulk copy of `bytes` (a multiple of 16; both addresses
// 16-byte aligned) whose completion counts against the mbarrier's
// transaction count
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

}  // namespace
