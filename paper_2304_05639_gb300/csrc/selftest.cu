// Self-test of the bounded-wait failure path: one block arms an mbarrier for
// 16 bytes that no copy ever delivers, waits with a short clock limit, and
// reports the timeout through the context's device status word, exactly as a
// streaming kernel does when a copy never lands.  Nothing faults or traps.
#include "lenia_internal.cuh"
#include "ptx_util.cuh"

namespace lenia {

__global__ void k_selftest_wait(long long limit, int* status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        mbar_arrive_expect_tx(&bar, 16);         // never completed: no copy is issued
        if (!mbar_wait_bounded(&bar, 0, limit)) atomicExch(status, kStatusWaitTimeout);
    }
}

cudaError_t launch_selftest_wait(long long limit_cycles, int* status, cudaStream_t s)
{
    k_selftest_wait<<<1, 32, 0, s>>>(limit_cycles, status);
    return cudaGetLastError();
}

}  // namespace lenia
