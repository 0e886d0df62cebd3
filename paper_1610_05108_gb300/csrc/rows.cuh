// Row draws of a run (the row draw of Algorithm 2 with the counter-based stream):
// draw t of a search with seed s uses u = splitmix64 output t (the finaliser
// of Steele, Lea & Flood applied to s + (t + 1) * 0x9E3779B97F4A7C15).
//   uniform rows (binary Y):      row = floor(u * n / 2^64);
//   weighted rows (real Y, Section 3.1): with integer weights q_i and
//   cdf[i] = q_0 + ... + q_i (total = cdf[n-1]), r = floor(u * total / 2^64)
//   and the row is the least i with cdf[i] > r, i.e. P(i) = q_i / total.
// With equal weights both give the same row.
#pragma once

#include <stdint.h>

namespace xyz {

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int64_t draw_row(uint64_t seed, uint64_t t, int64_t n,
                                            const uint64_t *__restrict__ cdf, uint64_t total)
{
    const uint64_t u = mix64(seed + (t + 1ULL) * 0x9E3779B97F4A7C15ULL);
    if (!cdf)
        return (int64_t)__umul64hi(u, (uint64_t)n);
    const uint64_t r = __umul64hi(u, total);        // r < total = cdf[n - 1]
    int64_t lo = 0, hi = n - 1;                      // least i with cdf[i] > r
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(cdf + mid) > r)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

}  // namespace xyz
