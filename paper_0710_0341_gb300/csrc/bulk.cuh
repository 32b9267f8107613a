// Bulk global -> shared copies completed on an mbarrier (sm_90 and later:
// cp.async.bulk with mbarrier::complete_tx), in inline PTX.
//
// A copy needs 16-byte aligned source and destination addresses and a size
// that is a multiple of 16 bytes; the callers check this. The destination is
// this CTA's own shared memory (a CTA launched without a cluster is a cluster
// of one), so no multicast is involved.
//
// Waits are bounded: mbar_wait gives up after max_polls polls and returns
// false, so that a copy that never completes ends in an error status instead
// of a hung kernel.
#pragma once
#include <cstdint>

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// count arrivals complete a phase (together with the expected transaction bytes)
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// initialised barriers become visible to the asynchronous (bulk copy) proxy
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// order this thread's earlier shared-memory accesses before later bulk copies
// into the same bytes (reads of a stage before it is refilled)
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// one arrival that also announces `bytes` of copies to come in this phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// wait for the phase of parity `parity` to complete; false after max_polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long max_polls) {
    for (long long it = 0; it < max_polls; it++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
