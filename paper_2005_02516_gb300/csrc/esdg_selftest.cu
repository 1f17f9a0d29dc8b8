// Self-test of the bounded device-side wait (failure detection without a GPU
// fault): one warp arms an mbarrier phase that expects bytes no copy will
// deliver and waits on it through mbar_wait_bounded, the same wait the stage
// kernels use on their bulk copies.  The wait gives up after its cycle limit
// (about a second), sets STATUS_TIMEOUT in the status word and the kernel
// returns; nothing is in flight, so the context stays usable.
#include <cuda_runtime.h>

#include "esdg.h"
#include "esdg_stage2.cuh"

namespace esdg {

__global__ void k_wait_selftest(int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    fence_mbar_init();
    __syncwarp();
    // one arrival with 16 bytes still expected: the phase cannot complete
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16);
    __syncwarp();
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bar, 0, status))) return;
    // (not reached: the phase never completes)
    if (threadIdx.x == 0) atomicOr(status, 8);
}

}  // namespace esdg

extern "C" int esdg_selftest_wait_timeout(void* stream) {
    using namespace esdg;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int* d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return ESDG_ENOMEM;
    int h = 0;
    int rc = ESDG_OK;
    if (cudaMemsetAsync(d, 0, sizeof(int), s) != cudaSuccess) rc = ESDG_ECUDA;
    if (!rc) {
        k_wait_selftest<<<1, 32, 0, s>>>(d);
        if (cudaGetLastError() != cudaSuccess) rc = ESDG_ECUDA;
    }
    if (!rc && cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = ESDG_ECUDA;
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = ESDG_ECUDA;
    cudaFree(d);
    if (rc) return rc;
    if (h == STATUS_TIMEOUT) return ESDG_ETIMEOUT;
    return h == 0 ? ESDG_OK : ESDG_ECUDA;
}
