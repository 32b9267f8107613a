// Self-test of the bounded device waits (failure detection without a fault).
#include "wait.cuh"

namespace {
// one CTA waits at a barrier that expects two members: nothing ever arrives
__global__ void k_wait_selftest(unsigned* bar, int* status, long long max_polls) {
    unsigned gen = 0;
    if (!group_wait(bar, status, gen, 2, max_polls)) return;
    if (threadIdx.x == 0) atomicExch(status, -1);  // unreachable unless the barrier is broken
}
}  // namespace

extern "C" int ovl_wait_selftest(ovl_lattice lat, long long max_polls, int* status) {
    if (!lat || !status || max_polls < 1 || max_polls > (1ll << 24))
        return ovl_fail(lat, OVL_EINVAL, "ovl_wait_selftest: bad argument");
    // two ints in the lattice's status words: barrier counter and status
    int* w = lat->d_status + 32;
    OVL_CUDA_TRY(lat, cudaMemsetAsync(w, 0, 2 * sizeof(int), lat->stream));
    k_wait_selftest<<<1, 64, 0, lat->stream>>>((unsigned*)w, w + 1, max_polls);
    OVL_LAUNCH_CHECK(lat);
    OVL_CUDA_TRY(lat, cudaMemcpyAsync(status, w + 1, sizeof(int), cudaMemcpyDeviceToHost, lat->stream));
    OVL_CUDA_TRY(lat, cudaStreamSynchronize(lat->stream));
    return OVL_OK;
}
