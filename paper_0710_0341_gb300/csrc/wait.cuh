// Bounded device-side waits.
//
// Every spin-wait in this library polls a counter with an iteration limit:
// when the limit runs out the waiting CTA stores OVL_ETIMEOUT in a status
// word that the host reads after the kernel, every other waiter sees that
// status and leaves too, and the kernel returns normally, so the CUDA
// context stays usable.
#pragma once
#include "ovl_common.cuh"

// Barrier of `members` CTAs on `bar` (zero before the launch), generation
// `gen` per CTA. Returns false if it (or another member) timed out.
__device__ __forceinline__ bool group_wait(unsigned* bar, int* status, unsigned& gen, int members,
                                           long long max_polls) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        gen++;
        const unsigned target = gen * (unsigned)members;
        __threadfence();
        atomicAdd(bar, 1u);
        long long it = 0;
        int good = 1;
        while (true) {
            unsigned v = *((volatile unsigned*)bar);
            if (v >= target) break;
            if (*((volatile int*)status) == OVL_ETIMEOUT) {
                good = 0;
                break;
            }
            if (++it > max_polls) {
                atomicExch(status, OVL_ETIMEOUT);
                good = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}
