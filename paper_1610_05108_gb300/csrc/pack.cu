// K1 pack: the "form Z" step of Algorithm 2 (step 1).  Z = Y o X is never
// stored: its bits are X's bits xor Y's bits, so packing X and Y is enough.
// Input int8 +-1, column-major X[j*n + i]; bit(v) = 1 iff v == -1.
// Memory-bound one-off per context: every input byte is read once.
#include "xyz_internal.cuh"

namespace xyz {
namespace {

// One thread per (column j, word w): bits of rows 32w..32w+31 of column j.
// Neighbouring threads take neighbouring words of a column, so a warp reads
// 1 KB of the column contiguously.  Also validates every entry.
__global__ void pack_cols_kernel(const int8_t *__restrict__ X, int64_t n, int64_t p, int64_t Wp,
                                 uint32_t *__restrict__ Xc, int *__restrict__ bad)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p * Wp)
        return;
    int64_t j = t / Wp, w = t - j * Wp;
    const int8_t *col = X + j * n;
    uint32_t word = 0;
    int badv = 0;
    int64_t i0 = w * 32;
#pragma unroll 8
    for (int b = 0; b < 32; ++b) {
        int64_t i = i0 + b;
        if (i < n) {
            int v = col[i];
            word |= (uint32_t)(v == -1) << b;
            badv |= (v != 1 && v != -1);
        }
    }
    Xc[t] = word;
    if (badv)
        atomicOr(bad, 1);
}

// One thread per (row i, word J): bits of columns 32J..32J+31 of row i.
// Threads of a warp take 32 consecutive rows, so for each column the warp
// reads 32 contiguous bytes.
__global__ void pack_rows_kernel(const int8_t *__restrict__ X, int64_t n, int64_t p, int64_t Pp,
                                 uint32_t *__restrict__ Xr)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    for (int64_t J = blockIdx.y; J < Pp; J += gridDim.y) {
        uint32_t word = 0;
        int64_t j0 = J * 32;
#pragma unroll 8
        for (int b = 0; b < 32; ++b) {
            int64_t j = j0 + b;
            if (j < p)
                word |= (uint32_t)(X[j * n + i] == -1) << b;
        }
        Xr[i * Pp + J] = word;
    }
}

// Response bits; positions past n are 1 so they never agree.
__global__ void pack_y_kernel(const int8_t *__restrict__ Y, int64_t n, int64_t Wp,
                              uint32_t *__restrict__ yb, int *__restrict__ bad)
{
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= Wp)
        return;
    uint32_t word = 0;
    int badv = 0;
    for (int b = 0; b < 32; ++b) {
        int64_t i = w * 32 + b;
        if (i < n) {
            int v = Y[i];
            word |= (uint32_t)(v == -1) << b;
            badv |= (v != 1 && v != -1);
        } else {
            word |= 1u << b;
        }
    }
    yb[w] = word;
    if (badv)
        atomicOr(bad, 1);
}

}  // namespace

cudaError_t launch_pack_y(const int8_t *dY, const Packed &pk, int *bad_flag, cudaStream_t s,
                          int64_t *launches)
{
    int threads = 256;
    int64_t blocks = (pk.Wp + threads - 1) / threads;
    pack_y_kernel<<<(unsigned)blocks, threads, 0, s>>>(dY, pk.n, pk.Wp, pk.yb, bad_flag);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_pack(const int8_t *dX, const int8_t *dY, const Packed &pk, int *bad_flag,
                        cudaStream_t s, int64_t *launches)
{
    int threads = 256;
    int64_t total = pk.p * pk.Wp;
    int64_t blocks = (total + threads - 1) / threads;
    pack_cols_kernel<<<(unsigned)blocks, threads, 0, s>>>(dX, pk.n, pk.p, pk.Wp, pk.Xc, bad_flag);
    *launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    dim3 grid((unsigned)((pk.n + threads - 1) / threads), (unsigned)(pk.Pp < 65535 ? pk.Pp : 65535));
    pack_rows_kernel<<<grid, threads, 0, s>>>(dX, pk.n, pk.p, pk.Pp, pk.Xr);
    *launches += 1;
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    return launch_pack_y(dY, pk, bad_flag, s, launches);
}

}  // namespace xyz
