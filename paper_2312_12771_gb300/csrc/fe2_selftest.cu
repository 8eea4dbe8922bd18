// Self-test of the bounded device waits used by the TMA and tensor-core
// kernels: an mbarrier that nothing ever arrives on.  The wait gives up after
// ~2^31 cycles and the kernel reports FE2_ERR_TIMEOUT; the context stays usable.
#include "fe2_internal.cuh"
#include "fe2_ptx.cuh"

namespace fe2 {

namespace {

__global__ void k_selftest_wait(int* status) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int to;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) to = mbar_wait_bounded(&bar, 0) ? 0 : 1;
    __syncthreads();
    if (threadIdx.x == 0) *status = to ? FE2_ERR_TIMEOUT : FE2_OK;
}

}  // namespace

cudaError_t launch_selftest_wait(int* status, cudaStream_t s) {
    k_selftest_wait<<<1, 32, 0, s>>>(status);
    return cudaGetLastError();
}

}  // namespace fe2
