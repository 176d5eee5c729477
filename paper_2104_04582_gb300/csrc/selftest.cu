// selftest.cu -- a kernel whose bounded wait always expires, to exercise the device error latch
// without a fault (few_selftest_wait_expiry).
#include "fewsum_internal.h"
#include "async.cuh"

namespace fewsum {

// Self-test of the bounded waits and the error latch: one thread waits on an mbarrier that
// nothing arrives on and no copy targets, gives up after limit_ns, and latches the timeout bit
// exactly as the summation and reduced-basis kernels do when a wait expires.
__global__ void k_wait_selftest(unsigned *err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        if (!mbar_wait_limit(&bar, 0u, limit_ns)) atomicOr(err, ERRBIT_TIMEOUT);
    }
}

cudaError_t launch_wait_selftest(unsigned *err, unsigned limit_us, cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(err, 1000ull * limit_us);
    return cudaGetLastError();
}

}  // namespace fewsum
