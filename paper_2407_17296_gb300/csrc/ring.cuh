// ring.cuh -- a shared-memory ring of trajectory slices filled by bulk asynchronous copies.
//
// The adjoint reads one slice of stored particle states (M x d_x floats, rows padded to a
// multiple of 4) per reversed step.  Thread 0 issues cp.async.bulk copies of the next R
// slices into R shared-memory slots; each slot has a "full" mbarrier (completed by the
// copy's transaction count) and an "empty" mbarrier (one arrival per warp once the warp is
// done with the slot).  Consumers wait on "full", the producer waits on "empty" before
// refilling a slot.  Every wait is bounded: on expiry the thread records kStatusTimeout in
// the caller's status word and carries on without the data, so the kernel always
// terminates and the host sees the failure.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "pf_args.h"

namespace smc2 {

constexpr int kStatusTimeout = 1;
constexpr uint32_t kWaitLimit = 1u << 22;  // try_wait polls (each may suspend briefly)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make barrier initialisation visible to the asynchronous proxy (then __syncthreads)
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ bool mbar_try_wait_u32(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for the phase with the given parity to complete; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kWaitLimit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// The same for a barrier given by its shared-memory address.
__device__ __forceinline__ bool mbar_wait_u32(uint32_t bar, uint32_t parity, uint32_t limit = kWaitLimit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait_u32(bar, parity)) return true;
    return false;
}

// global -> shared bulk copy completing `bytes` transactions on `bar` (16-byte aligned
// addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// shared -> global bulk copy in the issuing thread's bulk async-group (16-byte aligned
// addresses, size a multiple of 16); commit, then wait until at most N groups still read their
// source (wait_read) or at most N are incomplete (wait)
__device__ __forceinline__ void bulk_copy_s2g(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
template <int N>
__device__ __forceinline__ void bulk_wait() {
    asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// order this thread's earlier generic-proxy global writes before later async-proxy reads
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

// order this thread's earlier generic-proxy shared-memory writes before later async-proxy
// accesses of the same memory (e.g. a bulk copy that overwrites a slot it wrote into)
__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int R, int DX>
struct SliceRing {
    float* slots;        // R slots of padded_particles(M) * DX floats
    uint64_t* full;      // R "full" barriers, then R "empty" barriers
    int M;               // particles (slot rows, padded to a multiple of 4)
    uint32_t full_phase = 0;   // per-slot parity bits of the next "full" phase to wait for
    uint32_t empty_phase = 0;  // producer only: parity bits for "empty" waits (start "free")
    uint32_t filled = 0;       // producer only: slots that have ever been filled

    __device__ float* slot(uint32_t g) const { return slots + (size_t)(g % R) * padded_particles(M) * DX; }

    // The same operations by slot index s (= g % R, which the sweep advances step by step),
    // with the slot size and the barriers' shared-memory address computed once by the caller.
    __device__ float* slot_at(uint32_t s, uint32_t slot_elems) const { return slots + s * slot_elems; }
    __device__ void acquire_slot(uint32_t s, uint32_t full_u32, int* status) {
        if (!mbar_wait_u32(full_u32 + 8u * s, (full_phase >> s) & 1u)) atomicOr(status, kStatusTimeout);
        full_phase ^= 1u << s;
    }
    __device__ void release_slot(uint32_t s, uint32_t full_u32) const {
        __syncwarp();
        if ((threadIdx.x & 31) == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(full_u32 + 8u * (R + s)) : "memory");
    }

    // thread 0 only: copy slice src into the slot of slice g once every warp has released it
    __device__ void produce(uint32_t g, const float* src, int* status) {
        const uint32_t s = g % R;
        if (filled & (1u << s)) {
            if (!mbar_wait(&full[R + s], (empty_phase >> s) & 1u)) atomicOr(status, kStatusTimeout);
            empty_phase ^= 1u << s;
        }
        filled |= 1u << s;
        const uint32_t bytes = (uint32_t)(sizeof(float) * padded_particles(M) * DX);
        mbar_arrive_expect_tx(&full[s], bytes);
        bulk_copy_g2s(slot(g), src, bytes, &full[s]);
    }

    // every thread: wait until slice g has landed
    __device__ void acquire(uint32_t g, int* status) {
        const uint32_t s = g % R;
        if (!mbar_wait(&full[s], (full_phase >> s) & 1u)) atomicOr(status, kStatusTimeout);
        full_phase ^= 1u << s;
    }

    // every thread: this warp is done with slice g
    __device__ void release(uint32_t g) {
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(&full[R + g % R]);
    }
};

}  // namespace smc2
