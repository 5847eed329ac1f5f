// tma.cuh -- tensor-memory-accelerator (TMA) bulk copies into shared memory
// with an mbarrier completion, as inline PTX for sm_103a.
//
// Protocol used by the RAS sweep: thread 0 initialises one mbarrier (arrival
// count 1), makes the initialisation visible to the async proxy, and after a
// CTA barrier arrives on it announcing the total number of bytes the copies
// will deliver, then issues the copies; every thread waits for phase 0.  The
// wait is bounded: after TMA_WAIT_TRIES polls (by default; about one second)
// it gives up and reports it, so that a copy that never lands cannot hang
// the GPU.
#pragma once

#include <cuda.h>  // CUtensorMap

namespace qdd {

// Each poll may suspend the thread until the phase completes, for at most
// TMA_SUSPEND_NS (so waiting warps take no issue slots from the other CTA of
// the SM); TMA_WAIT_TRIES polls bound a wait to about one second.
constexpr unsigned TMA_SUSPEND_NS = 500000;
constexpr long TMA_WAIT_TRIES = 2000;

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(TMA_SUSPEND_NS)
        : "memory");
    return ok != 0;
}

// Polls phase `parity` of the barrier at most `tries` times; returns whether
// it completed.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity, long tries)
{
    for (long i = 0; i < tries; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// One tiled 5-D tensor copy global -> shared memory (this CTA), completing
// on the barrier.  dst must be 128-byte aligned; c0 * 4 bytes (the innermost
// coordinate of a 32-bit-element map) must be a multiple of 16.
__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, unsigned long long *bar, int c0, int c1,
                                            int c2, int c3, int c4)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6, "
        "%7}], [%2];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(c4)
        : "memory");
}

}  // namespace qdd
