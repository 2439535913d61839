// Packed 16-bit helpers for the SGM kernels (two cells per 32-bit register).
//
// Every value the recurrence handles stays below 2^15 (costs and path costs
// are at most 255, penalties at most 255, the "infinite" neighbour is 0x3FFF
// plus a penalty), so a plain 32-bit add or subtract of two packed pairs never
// carries or borrows across the halves and equals two independent 16-bit
// operations.  min.u16x2 and the three-input __vimin3_u16x2 are native
// instructions on sm_103a.
#pragma once

#include <stdint.h>

namespace simsense {

__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// three-input minimum per half (a DPX instruction on this GPU: one issue slot)
__device__ __forceinline__ uint32_t vmin3(uint32_t a, uint32_t b, uint32_t c) { return __vimin3_u16x2(a, b, c); }

__device__ __forceinline__ uint32_t vmax2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// bytes b0, b1 of w -> (b0, b1) as a packed pair
__device__ __forceinline__ uint32_t lo_bytes(uint32_t w) { return __byte_perm(w, 0, 0x4140); }
// bytes b2, b3 of w -> (b2, b3)
__device__ __forceinline__ uint32_t hi_bytes(uint32_t w) { return __byte_perm(w, 0, 0x4342); }
// (hi half of a, lo half of b): the pair shifted by one cell across a and b
__device__ __forceinline__ uint32_t shift_pair(uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x5432); }
// low bytes of two pairs -> four bytes (a.lo, a.hi, b.lo, b.hi)
__device__ __forceinline__ uint32_t pack_bytes(uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x6420); }
// minimum of the two halves of a pair
__device__ __forceinline__ uint32_t hmin(uint32_t a) { return min(a & 0xffffu, a >> 16); }

}  // namespace simsense
