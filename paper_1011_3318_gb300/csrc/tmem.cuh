// tmem.cuh -- the SM's tensor memory (TMEM) as per-thread private storage,
// through tcgen05 inline PTX for sm_103a.
//
// TMEM is 128 lanes x 512 columns of 32-bit cells per SM, allocated by
// columns to a CTA (a power of two, at least 32).  With the 32x32b access
// shape, thread i of warp w reads and writes lane 32 (w % 4) + i, so each
// thread of a 128-thread CTA owns one lane: a store/load of N columns moves N
// 32-bit values between the thread's registers and its lane.  The RAS sweep
// keeps there what only the owning thread reads, freeing shared memory.
//
// Protocol: one full warp allocates (the address lands in shared memory) and,
// at the end, frees the columns; tcgen05 fences around the CTA barriers
// order the allocation, the accesses and the release.  A CTA must free its
// columns on every path that allocated them.
#pragma once

#include "tma.cuh"  // smem_addr

namespace qdd {

// By all 32 threads of one warp: allocates ncols columns, writing the TMEM
// address (lane 0, first column) to *dst, and gives up the right to allocate
// again (without that, the next CTAs' allocations on the SM waited: a sweep
// of 128-site domains ran at half speed).
__device__ __forceinline__ void tm_alloc(unsigned *dst, unsigned ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// By all 32 threads of one warp, after every access of the CTA.
__device__ __forceinline__ void tm_dealloc(unsigned taddr, unsigned ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// The address of this thread's lane at column col of an allocation at base
// (the warp's quarter of the 128 lanes in bits 31:16).
__device__ __forceinline__ unsigned tm_lane_addr(unsigned base, unsigned col)
{
    return base + (((threadIdx.x >> 5) & 3u) << 21) + col;
}

// Columns addr .. addr+7 of this thread's lane <- v (by a whole warp).
__device__ __forceinline__ void tm_st8(unsigned addr, const float *v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(addr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}

// v <- columns addr .. addr+23 of this thread's lane (by a whole warp), in
// one round trip: the earlier stores of the thread complete first, then both
// loads are issued and waited for together.
__device__ __forceinline__ void tm_ld24(unsigned addr, float *v)
{
    unsigned r[24];
    asm volatile(
        "tcgen05.wait::st.sync.aligned;\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%24];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%25];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
        : "r"(addr), "r"(addr + 16)
        : "memory");
#pragma unroll
    for (int k = 0; k < 24; k++) v[k] = __uint_as_float(r[k]);
}

}  // namespace qdd
