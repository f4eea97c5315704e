// Bulk asynchronous global -> shared copies (cp.async.bulk, the Blackwell tensor-memory
// accelerator's untiled form) completed on shared-memory mbarriers, with bounded waits.
// Every wait gives up after a fixed number of polls or ~1 s of SM clock, so a copy that
// never lands ends the kernel with an error status instead of a hang.
#pragma once

#include <stdint.h>

namespace cel {

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// one arrival (the issuing thread) completes a phase once the expected bytes land
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// make barrier initialisation visible to the async proxy
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier shared-memory accesses before later async-proxy writes
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global src to
// shared dst, announcing them on bar first.  Called by one thread.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

constexpr int MBAR_MAX_POLLS = 1 << 22;
constexpr long long MBAR_MAX_CYCLES = 2000000000LL;   // ~1 s at 2 GHz

// Wait for the phase with the given parity to complete; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    const long long t0 = clock64();
    for (int i = 0; i < MBAR_MAX_POLLS; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > MBAR_MAX_CYCLES) return false;
    }
    return false;
}

}  // namespace cel
