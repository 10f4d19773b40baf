// qew_tma.cuh -- one-dimensional bulk copies between global and shared memory through the
// Tensor Memory Accelerator (cp.async.bulk, sm_90+), with an mbarrier for load completion.
//
// Every wait is bounded: a wait that gives up returns false, and the caller records an error
// and skips the data instead of spinning forever.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qew {

// Spin limit of an mbarrier wait: far beyond any copy's latency (each try_wait already
// suspends for a hardware-chosen time slice), small enough that a lost copy ends the kernel.
constexpr int kMbarSpinLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make the initialised barrier visible to the async proxy (the TMA unit completes it).
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bulk copy global -> shared; completes `bytes` transactions on `bar`.  src and dst 16-byte
// aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bulk copy shared -> global in the current bulk group.  Same alignment rules.
__device__ __forceinline__ void tma_store_1d(void* dst, const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_store_commit()
{
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until all committed bulk stores of this thread have completed.
__device__ __forceinline__ void tma_store_wait_all()
{
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Wait until all committed bulk stores of this thread have finished reading their shared-memory
// sources (the global writes may still be in flight).
__device__ __forceinline__ void tma_store_wait_read_all()
{
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Bounded wait for phase `phase` of `bar`; false if `limit` polls did not see it complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, int limit = kMbarSpinLimit)
{
    const uint32_t addr = smem_u32(bar);
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(phase)
            : "memory");
        if (done)
            return true;
    }
    return false;
}

}  // namespace qew
