// Self-test of failure detection: one block waits, with the bounded wait the
// FFT passes use for their tensor copies (%globaltimer, 2 s), on an
// mbarrier that nothing ever arrives at.  The wait gives up, the block
// records the error in the flag the passes use, and the host reads it as it
// reads an expired wait of a pass.  No fault, trap or unbounded wait.
#include "pm_launch.h"
#include "pm_passes.cuh"

namespace {

__global__ void k_wait_expiry(int *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        pmk::mbar_init(&bar, 1);   // one arrival expected; none comes
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !pmk::mbar_wait(&bar, 0)) atomicExch(err, 1);
}

}  // namespace

cudaError_t pm_launch_wait_expiry(int *err, cudaStream_t st) {
    k_wait_expiry<<<1, 32, 0, st>>>(err);
    return cudaGetLastError();
}
