// Real-valued response (Section 3.1, continuous Y with binary X).
//
// The search samples row i with probability |Y_i| / ||Y||_1, forms Z from
// the signs of Y, and weighs each agreeing row by |Y_i|.  The weights are
// used in fixed point: with max |Y_i| = f 2^e (f in [0.5, 1)),
// q_i = floor(|Y_i| 2^(24 - e) + 1/2), an integer in [0, 2^24] (every step
// below is exact, so the result does not depend on the order of any sum).
// Prepared once per response:
//   yb      sign bits (1 for Y_i < 0; padding rows 1, so they never agree),
//   planes  per 32-row word, 25 bit planes of the q of its rows,
//   cdf     inclusive prefix sums of q (the weighted row draw, rows.cuh),
//   total   Q = sum q.
#include <math.h>

#include "rows.cuh"
#include "xyz_internal.cuh"

namespace xyz {
namespace {

constexpr int WT_THREADS = 256;

// max |Y_i| as the bits of a non-negative double (ordered like the value);
// bad != 0 when some entry is not finite
__global__ void maxabs_kernel(const double *__restrict__ Y, int64_t n,
                              unsigned long long *__restrict__ maxbits, int *__restrict__ bad)
{
    unsigned long long m = 0;
    int b = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double y = Y[i];
        if (!isfinite(y)) {
            b = 1;
            continue;
        }
        const unsigned long long v = (unsigned long long)__double_as_longlong(fabs(y));
        m = v > m ? v : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
        b |= __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (m)
            atomicMax(maxbits, m);
        if (b)
            atomicOr(bad, 1);
    }
}

// One warp per 32-row word: fixed-point weights, sign bits and bit planes.
__global__ void quantize_kernel(const double *__restrict__ Y, int64_t n, int64_t Wp,
                                const unsigned long long *__restrict__ maxbits,
                                uint64_t *__restrict__ q, uint32_t *__restrict__ yb,
                                uint32_t *__restrict__ planes)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= Wp)
        return;                                   // whole warp leaves together
    int e = 0;
    frexp(__longlong_as_double((long long)*maxbits), &e);
    const int64_t i = 32 * w + lane;
    uint64_t qv = 0;
    uint32_t neg = 1;                             // padding rows: never agree
    if (i < n) {
        const double y = Y[i];
        qv = isfinite(y) ? (uint64_t)floor(ldexp(fabs(y), 24 - e) + 0.5) : 0u;   // rejected later
        neg = y < 0.0 ? 1u : 0u;
        q[i] = qv;
    }
    const uint32_t sb = __ballot_sync(0xffffffffu, neg);
    uint32_t mine = 0;                            // lane b keeps plane b
#pragma unroll
    for (int b = 0; b < XYZ_WPLANES; ++b) {
        const uint32_t pb = __ballot_sync(0xffffffffu, (uint32_t)(qv >> b) & 1u);
        if (lane == b)
            mine = pb;
    }
    if (lane == 0)
        yb[w] = sb;
    if (lane < XYZ_WPLANES)
        planes[w * XYZ_WPLANES + lane] = mine;
}

// exclusive prefix sums -> inclusive
__global__ void inclusive_kernel(uint64_t *__restrict__ cdf, const uint64_t *__restrict__ q, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        cdf[i] += q[i];
}

// Weighted strengths of the output pairs: one warp per pair recomputes the
// weight sum S of its agreeing rows; strength = (2 S - Q) / Q, or
// (2 S - Q) * scale when scale is set (the Lasso check reports r^T w / n).
__global__ void weighted_strength_kernel(const uint32_t *__restrict__ Xc, int64_t Wp,
                                         const uint32_t *__restrict__ yb,
                                         const uint32_t *__restrict__ planes, uint64_t Q, double scale,
                                         PairOut *__restrict__ out, const uint32_t *__restrict__ nout)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t N = *nout;
    for (int64_t t = wid; t < N; t += nw) {
        const int64_t j = out[t].j, k = out[t].k;
        int64_t S = 0;
        for (int64_t w = lane; w < Wp; w += 32) {
            const uint32_t g = ~(Xc[j * Wp + w] ^ Xc[k * Wp + w] ^ yb[w]);
            const uint32_t *pl = planes + w * XYZ_WPLANES;
            for (int b = 0; b < XYZ_WPLANES; ++b)
                S += (int64_t)__popc(g & pl[b]) << b;
        }
        for (int o = 16; o > 0; o >>= 1)
            S += __shfl_xor_sync(0xffffffffu, S, o);
        if (lane == 0) {
            const double v = (double)(2 * S - (int64_t)Q);
            out[t].strength = (float)(scale != 0.0 ? v * scale : v / (double)Q);
        }
    }
}

// Flip the response sign bits of the n valid rows (Y -> -Y); padding bits stay 1.
__global__ void flip_kernel(uint32_t *__restrict__ yb, int64_t n, int64_t Wp)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < Wp; w += stride) {
        const int64_t rows = n - 32 * w;
        const uint32_t valid = rows >= 32 ? 0xFFFFFFFFu : (rows > 0 ? ((1u << rows) - 1u) : 0u);
        yb[w] ^= valid;
    }
}

// Sign transform of a real X (Section 3.2): -1 / +1 by sign; an entry that is
// exactly 0 gets a fair coin, the top bit of splitmix64 output t = its
// column-major index from the state coin_seed.  bad != 0 on a NaN.
__global__ void sign_kernel(const float *__restrict__ X, int64_t count, uint64_t coin_seed,
                            int8_t *__restrict__ out, int *__restrict__ bad)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride) {
        const float x = X[t];
        int8_t v;
        if (x < 0.0f)
            v = -1;
        else if (x > 0.0f)
            v = 1;
        else if (x == 0.0f)
            v = (mix64(coin_seed + ((uint64_t)t + 1ULL) * 0x9E3779B97F4A7C15ULL) >> 63) ? (int8_t)-1 : (int8_t)1;
        else {
            v = 1;
            atomicOr(bad, 1);
        }
        out[t] = v;
    }
}

}  // namespace

cudaError_t launch_sign_transform(const float *dX, int64_t count, uint64_t coin_seed, int8_t *out, int *bad,
                                  cudaStream_t s, int64_t *launches)
{
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e != cudaSuccess)
        return e;
    int64_t g = (count + WT_THREADS - 1) / WT_THREADS;
    g = g < 1 ? 1 : (g > 65535 ? 65535 : g);
    sign_kernel<<<(unsigned)g, WT_THREADS, 0, s>>>(dX, count, coin_seed, out, bad);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_flip_signs(const Packed &pk, cudaStream_t s, int64_t *launches)
{
    int64_t g = (pk.Wp + WT_THREADS - 1) / WT_THREADS;
    g = g < 1 ? 1 : (g > 1024 ? 1024 : g);
    flip_kernel<<<(unsigned)g, WT_THREADS, 0, s>>>(pk.yb, pk.n, pk.Wp);
    *launches += 1;
    return cudaGetLastError();
}

size_t weights_scan_bytes(int64_t n) { return scan_temp_bytes(n); }

cudaError_t launch_prepare_weights(const double *dY, int64_t n, int64_t Wp, uint64_t *q, uint32_t *yb,
                                   uint32_t *planes, uint64_t *cdf, uint64_t *total,
                                   unsigned long long *maxbits, int *bad, void *scan_tmp, cudaStream_t s,
                                   int64_t *launches)
{
    cudaError_t e = cudaMemsetAsync(maxbits, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e != cudaSuccess)
        return e;
    int64_t g = (n + WT_THREADS - 1) / WT_THREADS;
    g = g < 1 ? 1 : (g > 4096 ? 4096 : g);
    maxabs_kernel<<<(unsigned)g, WT_THREADS, 0, s>>>(dY, n, maxbits, bad);
    const int64_t qb = (Wp * 32 + WT_THREADS - 1) / WT_THREADS;
    quantize_kernel<<<(unsigned)qb, WT_THREADS, 0, s>>>(dY, n, Wp, maxbits, q, yb, planes);
    *launches += 2;
    e = scan_u64_dev(q, cdf, nullptr, n, total, nullptr, scan_tmp, s, launches);
    if (e != cudaSuccess)
        return e;
    inclusive_kernel<<<(unsigned)g, WT_THREADS, 0, s>>>(cdf, q, n);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_weighted_strengths(const Packed &pk, PairOut *out, const uint32_t *nout, int64_t cap,
                                      cudaStream_t s, int64_t *launches)
{
    if (cap <= 0)
        return cudaSuccess;
    int64_t blocks = (cap * 32 + WT_THREADS - 1) / WT_THREADS;
    blocks = blocks > 4096 ? 4096 : (blocks < 1 ? 1 : blocks);
    weighted_strength_kernel<<<(unsigned)blocks, WT_THREADS, 0, s>>>(pk.Xc, pk.Wp, pk.yb, pk.planes,
                                                                     pk.wtotal, pk.wscale, out, nout);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace xyz
