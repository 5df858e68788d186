// Inline-PTX helpers for sm_103a: mbarrier-tracked bulk (TMA engine) copies global -> shared,
// bounded waits, and the library's device-side status word.
#pragma once
#include <cstdint>

namespace cdmimo {

// Device-side status word (CDMIMO_DEV_* bits) of this translation unit's kernels.  Each of the
// library's translation units is its own device module with its own word (internal linkage);
// cdmimo_device_status() reads and clears all of them (launch.h: module_status).
static __device__ unsigned int g_dev_status = 0u;

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before later async-proxy
// (bulk copy) accesses, and makes an mbarrier initialization visible to the async proxy.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned) from global memory to
// this CTA's shared memory; completion is signalled as transaction bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Asks the TMA engine to bring [src, src + bytes) into L2 (no registers, no completion to wait for).
// src 16-byte aligned, bytes a multiple of 16; otherwise nothing is issued.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes)
{
    if ((reinterpret_cast<uintptr_t>(src) & 15u) != 0u || (bytes & 15u) != 0u || bytes == 0u) return;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for phase `parity` of `bar` to complete, for at most `limit_ns` nanoseconds.  Returns
// false (and sets CDMIMO_DEV_TIMEOUT in the status word) if the wait gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns = 2000000000ull)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) {
            atomicOr(&g_dev_status, 0x1u);
            return false;
        }
        __nanosleep(64);
    }
}

}  // namespace cdmimo
