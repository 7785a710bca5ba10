// mm_async.cuh -- asynchronous global-to-shared copies (bulk copies completed on an mbarrier, and
// 4-byte cp.async) with waits that give up after a time limit instead of spinning forever.
#pragma once

#include <cstdint>

namespace mm {

// A wait that has not completed after this many SM clocks (about one second at 2 GHz) gives up;
// the caller records a device fault and leaves.
constexpr long long kWaitLimitClocks = 2000000000LL;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// One-time set-up of a barrier by one thread: `count` arrivals complete a phase. The fence makes the
// initialised barrier visible to the bulk-copy unit before any copy names it.
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Arrive once on bar and announce `bytes` of copies that will complete on it.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Arrive once on bar (no copies announced).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from global to this CTA's
// shared memory, counted on bar when it lands.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Wait for the phase of bar with the given parity to complete; false after kWaitLimitClocks.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > kWaitLimitClocks) return false;
    return true;
}

// 4-byte asynchronous copy global -> shared; src_bytes 0 writes a zero instead of reading src
// (src must still be a valid address).
__device__ __forceinline__ void cp_async4(void *dst, const void *src, unsigned src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
// 16-byte asynchronous copy global -> shared (both addresses 16-byte aligned); bytes past src_bytes
// (0, 4, 8, 12 or 16) are written as zeros.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, unsigned src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Wait until at most N of this thread's committed groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

}  // namespace mm
