// Tensor Memory (TMEM) as per-thread storage: inline PTX for sm_100-family tcgen05.
//
// TMEM is 128 lanes x 512 columns of 32-bit cells per SM.  A warp reaches the 32 lanes of its
// quadrant (lanes 32 * (warp % 4) .. + 31): with the 32x32b shape, thread i of the warp reads and
// writes lane 32 * (warp % 4) + i, so each thread owns a row of cells that no other thread of the
// CTA touches.  The decoder keeps each check thread's outgoing messages there: the next round's
// old-message reads then leave the shared-memory pipe.
//
// Address: bits 31..16 lane, bits 15..0 column.  tcgen05.ld / tcgen05.st are asynchronous:
// registers loaded by tcgen05.ld are read only after tcgen05.wait::ld (the wait below takes the
// registers as operands, so the compiler cannot move their uses above it), and TMEM cells stored
// by tcgen05.st are read back only after tcgen05.wait::st.  All tcgen05 instructions here are
// warp-collective (.sync.aligned): the whole warp executes them, converged.
#pragma once

#include <cstdint>

namespace sagms {

// Allocate `ncols` columns (a power of two, 32..512) for the CTA; the whole warp `w` calls it
// and the base address lands in shared memory at `slot`.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(slot));
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Release the CTA's columns: the warp that allocated them, after every access has completed
// and a CTA barrier bracketed by tmem_fence_before / tmem_fence_after.
__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Load 16 + 4 consecutive columns of the thread's lane into r[0..19], then wait for them.
__device__ __forceinline__ void tmem_ld20(uint32_t taddr, uint32_t (&r)[20]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19])
                 : "r"(taddr + 16u)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19])
                 :
                 : "memory");
}

// Store r[0..19] to 16 + 4 consecutive columns of the thread's lane.
__device__ __forceinline__ void tmem_st20(uint32_t taddr, const uint32_t (&r)[20]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr + 16u), "r"(r[16]),
                 "r"(r[17]), "r"(r[18]), "r"(r[19])
                 : "memory");
}

// Store x, y to 2 consecutive columns.
__device__ __forceinline__ void tmem_st2(uint32_t taddr, uint32_t x, uint32_t y) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr), "r"(x), "r"(y) : "memory");
}

// Load 2 consecutive columns of the thread's lane into x, y, then wait for them.
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, uint32_t& x, uint32_t& y) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(x), "=r"(y) : "r"(taddr) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(x), "+r"(y) : : "memory");
}

}  // namespace sagms
