// tma.cuh -- bulk asynchronous copies (the Tensor Memory Accelerator's
// non-tensor form, cp.async.bulk) into shared memory, completed on an
// mbarrier with a transaction count, and bounded waits on that barrier.
//
// Use pattern (one barrier per shared buffer, initialised with an arrival
// count of 1): one thread announces the bytes a round will deliver with
// arrive_expect_tx (that is the round's single arrival); any threads issue
// the copies; every consumer waits for the round's phase parity.  Copies
// may complete before the announcement: the transaction count may go
// negative in between, and the phase cannot complete while the arrival is
// still pending.
#pragma once

#include "hm_internal.cuh"

namespace hm {

// polls of mbarrier.try_wait (each may suspend the thread for a
// hardware-defined interval, then sleeps 32 ns) before a wait gives up:
// bounded at tens of milliseconds, far beyond any copy's completion
constexpr int kMbarSpinLimit = 1 << 16;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// make barrier initialisation visible to the async proxy (bulk copies)
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// wait for the phase with the given parity to complete; false on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int i = 0; i < kMbarSpinLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        __nanosleep(32);
    }
    return false;
}

// global -> shared bulk copy of `bytes` (multiple of 16; both addresses
// 16-byte aligned), completing `bytes` transactions on `bar`
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace hm
