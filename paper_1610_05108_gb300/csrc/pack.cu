// K1 pack: the "form Z" step of Algorithm 2 (step 1).  Z = Y o X is never
// stored: its bits are X's bits xor Y's bits, so packing X and Y is enough.
// Input int8 +-1, column-major X[j*n + i]; bit(v) = 1 iff v == -1.
// Memory-bound one-off per context: every input byte is read once.
#include "xyz_internal.cuh"

namespace xyz {
namespace {

// One CTA per tile of 32 columns (one Xr word) x 1024 rows (32 Xc words):
// the tile's bytes are read once (16-byte loads when every column segment
// is 16-byte aligned) into shared memory, then each packed word is one warp
// ballot of "entry == -1" -- over 32 rows of one column for Xc, over the 32
// columns of one row for Xr.  Entries past n or p read as +1 (bit 0), so
// the padding words come out zero.  X may live in device memory or in
// mapped pinned host memory (then the tile loads are the host transfer).
// Also validates every entry.
constexpr int PK_COLS = 32;
constexpr int PK_ROWS = 1024;
constexpr int PK_PITCH = PK_ROWS + 16;     // bytes per tile column: 16-byte aligned
constexpr int PK_THREADS = 256;
static_assert(PK_COLS * PK_ROWS % (16 * PK_THREADS) == 0, "whole 16-byte pieces per thread");

__global__ void __launch_bounds__(PK_THREADS)
    pack_tile_kernel(const int8_t *__restrict__ X, int64_t n, int64_t p, int64_t Wp, int64_t Pp,
                     int64_t nchunks, int vec16, uint32_t *__restrict__ Xc, uint32_t *__restrict__ Xr,
                     int *__restrict__ bad)
{
    __shared__ __align__(16) uint8_t tile[PK_COLS][PK_PITCH];
    const unsigned FULL = 0xffffffffu;
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    constexpr int NW = PK_THREADS / 32;
    const int64_t J = blockIdx.x;                   // columns 32 J .. 32 J + 31
    int badv = 0;
    for (int64_t chunk = blockIdx.y; chunk < nchunks; chunk += gridDim.y) {
        const int64_t i0 = chunk * PK_ROWS;
        const int64_t rows = n - i0 >= PK_ROWS ? PK_ROWS : (n > i0 ? n - i0 : 0);
        if (vec16) {
            // n is a multiple of 16 and X 16-byte aligned: each column's
            // segment is whole 16-byte pieces
            constexpr int PER_COL = PK_ROWS / 16;
            constexpr int PER_T = PK_COLS * PER_COL / PK_THREADS;     // 8 pieces per thread
            uint4 v[PER_T];
#pragma unroll
            for (int k = 0; k < PER_T; ++k) {                          // all loads in flight
                const int q = t + k * PK_THREADS;
                const int c = q / PER_COL, r16 = q - c * PER_COL;
                const int64_t j = 32 * J + c;
                v[k] = make_uint4(0x01010101u, 0x01010101u, 0x01010101u, 0x01010101u);
                if (j < p && 16 * r16 < rows)
                    v[k] = *reinterpret_cast<const uint4 *>(X + j * n + i0 + 16 * r16);
            }
#pragma unroll
            for (int k = 0; k < PER_T; ++k) {
                const int q = t + k * PK_THREADS;
                const int c = q / PER_COL, r16 = q - c * PER_COL;
                *reinterpret_cast<uint4 *>(&tile[c][16 * r16]) = v[k];
            }
        } else {
            for (int q = t; q < PK_COLS * PK_ROWS; q += PK_THREADS) {
                const int c = q / PK_ROWS, r = q - c * PK_ROWS;
                const int64_t j = 32 * J + c;
                tile[c][r] = (j < p && r < rows) ? (uint8_t)X[j * n + i0 + r] : (uint8_t)1;
            }
        }
        __syncthreads();
        // Xc: warp wp packs columns wp, wp + 8, ...; lane w keeps word w
        for (int c = wp; c < PK_COLS; c += NW) {
            uint32_t mine = 0;
#pragma unroll 4
            for (int w = 0; w < PK_ROWS / 32; ++w) {
                const uint8_t b = tile[c][32 * w + lane];
                badv |= (b != 0x01u && b != 0xFFu);
                const uint32_t word = __ballot_sync(FULL, b == 0xFFu);
                if (lane == w)
                    mine = word;
            }
            const int64_t j = 32 * J + c, wg = i0 / 32 + lane;
            if (j < p && wg < Wp)
                Xc[j * Wp + wg] = mine;
        }
        // Xr: warp wp packs rows wp * 32 .. + 31, then wp * 32 + 256 ...; lane
        // c reads column c, lane r keeps the word of row r
        for (int r0 = 32 * wp; r0 < PK_ROWS; r0 += 32 * NW) {
            uint32_t mine = 0;
#pragma unroll 4
            for (int rr = 0; rr < 32; ++rr) {
                const uint32_t word = __ballot_sync(FULL, tile[lane][r0 + rr] == 0xFFu);
                if (lane == rr)
                    mine = word;
            }
            const int64_t i = i0 + r0 + lane;
            if (i < n)
                Xr[i * Pp + J] = mine;
        }
        __syncthreads();                            // the tile is reused
    }
    if (__any_sync(FULL, badv) && lane == 0)
        atomicOr(bad, 1);
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
    const int64_t nchunks = (32 * pk.Wp + PK_ROWS - 1) / PK_ROWS;   // every Xc word, padding included
    const int vec16 = (pk.n % 16 == 0 && ((uintptr_t)dX & 15) == 0) ? 1 : 0;
    if (pk.Pp > 0x7FFFFFFFLL)
        return cudaErrorInvalidValue;
    dim3 grid((unsigned)pk.Pp, (unsigned)(nchunks < 65535 ? nchunks : 65535));
    pack_tile_kernel<<<grid, PK_THREADS, 0, s>>>(dX, pk.n, pk.p, pk.Wp, pk.Pp, nchunks, vec16, pk.Xc, pk.Xr,
                                                 bad_flag);
    *launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    return launch_pack_y(dY, pk, bad_flag, s, launches);
}

}  // namespace xyz
