// Bit-level helpers shared by the key kernels (host- and device-callable so
// the host can unit-test them).
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define XYZ_HD __host__ __device__ __forceinline__
#else
#define XYZ_HD inline
#endif

namespace xyz {

// In-register transpose of a 32 x 32 bit matrix: on entry bit c of A[m] is
// element (m, c); on exit bit m of A[c] is that element.  Five rounds swap
// the off-diagonal blocks of size 16, 8, 4, 2, 1 (the recursive block
// transposition of Warren, "Hacker's Delight", ch. 7-3, written for
// least-significant-bit-first indexing).
XYZ_HD void transpose32(uint32_t (&A)[32])
{
#define XYZ_TR_ROUND(J, MASK)                                          \
    _Pragma("unroll") for (int k = 0; k < 32; ++k)                     \
    {                                                                  \
        if ((k & (J)) == 0) {                                          \
            uint32_t t = ((A[k] >> (J)) ^ A[k + (J)]) & (MASK);        \
            A[k] ^= t << (J);                                          \
            A[k + (J)] ^= t;                                           \
        }                                                              \
    }
#ifdef __CUDA_ARCH__
    // rounds 16 and 8 move whole half-words and bytes: one byte permutation
    // per output word instead of the shift/xor/mask sequence (same result)
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const uint32_t a = A[k], b = A[k + 16];
        A[k] = __byte_perm(a, b, 0x5410);        // low halves of a, b
        A[k + 16] = __byte_perm(a, b, 0x7632);   // high halves of a, b
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        if ((k & 8) == 0) {
            const uint32_t a = A[k], b = A[k + 8];
            A[k] = __byte_perm(a, b, 0x6240);        // even bytes of a, b interleaved
            A[k + 8] = __byte_perm(a, b, 0x7351);    // odd bytes
        }
    }
#else
    XYZ_TR_ROUND(16, 0x0000FFFFu)
    XYZ_TR_ROUND(8, 0x00FF00FFu)
#endif
    XYZ_TR_ROUND(4, 0x0F0F0F0Fu)
    XYZ_TR_ROUND(2, 0x33333333u)
    XYZ_TR_ROUND(1, 0x55555555u)
#undef XYZ_TR_ROUND
}

// Bijective 32-bit mixer (the MurmurHash3 finaliser, Appleby): spreads the
// group keys uniformly over partitions; equal keys stay equal.
XYZ_HD uint32_t mix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

}  // namespace xyz
