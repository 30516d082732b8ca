// selftest.cu -- failure detection of the bounded device waits, exercised without a fault.
//
// The filter kernels wait on mbarriers for bulk copies; every such wait gives up after a
// poll limit, records kStatusTimeout in a device status word and lets the kernel finish,
// so the host sees SMC2_E_TIMEOUT and the context stays usable.  This entry point runs one
// block whose warps wait on a barrier that nothing completes, with a caller-chosen poll
// limit, and reports what the status word says.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/smc2.h"
#include "philox.cuh"
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

// One thread per (key, counter) pair: the filter kernels' own key expansion, Philox rounds,
// uniform map and Box-Muller pair (philox.cuh), written out for comparison.
__global__ void crn_words_kernel(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key, int n,
                                 uint32_t* __restrict__ words, float* __restrict__ u, float* __restrict__ z) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const smc2::PhiloxKey k = smc2::philox_key(key[4 * i], key[4 * i + 1], key[4 * i + 2], key[4 * i + 3]);
        const uint4 w = smc2::philox4x32_10(make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]), k);
        if (words) {
            words[4 * i] = w.x;
            words[4 * i + 1] = w.y;
            words[4 * i + 2] = w.z;
            words[4 * i + 3] = w.w;
        }
        if (u) {
            u[4 * i] = smc2::u01_open(w.x);
            u[4 * i + 1] = smc2::u01_open(w.y);
            u[4 * i + 2] = smc2::u01_open(w.z);
            u[4 * i + 3] = smc2::u01_open(w.w);
        }
        if (z) {
            smc2::box_muller(w.x, w.y, z[4 * i], z[4 * i + 1]);
            smc2::box_muller(w.z, w.w, z[4 * i + 2], z[4 * i + 3]);
        }
    }
}

}  // namespace

extern "C" int smc2_selftest_crn(const uint32_t* ctr_dev, const uint32_t* key_dev, int n, uint32_t* words_dev,
                                 float* u_dev, float* z_dev, void* stream) {
    using namespace smc2;
    if (n < 0 || (n > 0 && (!ctr_dev || !key_dev))) return fail(SMC2_E_INVAL, "n < 0 or NULL inputs");
    if (n == 0) return SMC2_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int blocks = (int)std::min<long>((n + 255) / 256, 4096);
    crn_words_kernel<<<blocks, 256, 0, st>>>(ctr_dev, key_dev, n, words_dev, u_dev, z_dev);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(SMC2_E_CUDA, std::string("CRN self-test: ") + cudaGetErrorString(e));
    count_launches(1);
    return SMC2_OK;
}

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
