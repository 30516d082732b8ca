// selftest.cu -- failure detection of the bounded device waits, exercised without a fault.
//
// The filter kernels wait on mbarriers for bulk copies; every such wait gives up after a
// poll limit, records kStatusTimeout in a device status word and lets the kernel finish,
// so the host sees SMC2_E_TIMEOUT and the context stays usable.  This entry point runs one
// block whose warps wait on a barrier that nothing completes, with a caller-chosen poll
// limit, and reports what the status word says.
#include <cuda_runtime.h>

#include <string>

#include "../../include/smc2.h"
#include "ring.cuh"
#include "runtime.h"

namespace {

__global__ void wait_nothing_kernel(uint32_t polls, int* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        smc2::mbar_init(&bar, 1);  // one arrival completes the phase; none comes
        smc2::mbar_fence_init();
    }
    __syncthreads();
    if (!smc2::mbar_wait(&bar, 0u, polls)) atomicOr(status, smc2::kStatusTimeout);
}

}  // namespace

extern "C" int smc2_selftest_bounded_wait(int polls, int* timed_out) {
    using namespace smc2;
    if (polls < 1 || !timed_out) return fail(SMC2_E_INVAL, "polls must be >= 1 and timed_out not NULL");
    int* status = nullptr;
    if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SMC2_E_NOMEM, "status allocation failed");
    }
    int host = 0;
    cudaError_t e = cudaMemset(status, 0, sizeof(int));
    if (e == cudaSuccess) {
        wait_nothing_kernel<<<1, 64>>>((uint32_t)polls, status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&host, status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(status);
    if (e != cudaSuccess) return fail(SMC2_E_CUDA, std::string("self-test: ") + cudaGetErrorString(e));
    count_launches(1);
    *timed_out = (host & kStatusTimeout) ? 1 : 0;
    return SMC2_OK;
}
