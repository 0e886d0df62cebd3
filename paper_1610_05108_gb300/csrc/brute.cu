// Exhaustive screen of all p(p-1)/2 pairs (eq. 1 evaluated for every pair):
// the comparator the xyz search is measured against, and the M = 0 case of
// Algorithm 2 (every column has the same empty key, so every pair is a
// candidate).
//
// a_jk = sum_w popc(~(z_j[w] ^ x_k[w])) with z_j = Xc_j ^ yb (bit of Z_ij is
// bit(X_ij) xor bit(Y_i)); padding bits never agree (Xc padding 0, yb
// padding 1).  One CTA of 256 threads scores a 128 x 128 tile of (j, k)
// (tiles on or above the diagonal only), each thread an 8 x 8 block held in
// registers.  The packed words of both column tiles stream through shared
// memory in chunks of 32 words, stored word-major so that a thread reads its
// eight columns of one word with two 16-byte loads.  Passing pairs (j < k,
// a >= a_min) are appended as records (j << kbits | k, a) for the sort and
// unique kernels that order the union of a search.
#include "xyz_internal.cuh"

namespace xyz {
namespace {

constexpr int BF_T = 128;          // columns per tile side
constexpr int BF_K = 32;           // words per chunk
constexpr int BF_LD = BF_T + 4;    // shared row pitch: 16-byte rows, 4-way store conflicts at most
constexpr int BF_THREADS = 256;

__global__ void __launch_bounds__(BF_THREADS, 2)
    brute_kernel(const uint32_t *__restrict__ Xc, int64_t Wp, int64_t W, const uint32_t *__restrict__ yb,
                 int64_t p, int64_t ntiles, int64_t amin, int kbits, uint64_t *__restrict__ rec_keys,
                 uint32_t *__restrict__ rec_agree, uint32_t *__restrict__ nrec, uint32_t rec_cap)
{
    __shared__ __align__(16) uint32_t zs[BF_K][BF_LD];
    __shared__ __align__(16) uint32_t xs[BF_K][BF_LD];
    // tile (bj, bk), bj <= bk, from the linear block index (row-major upper
    // triangle: row bj holds ntiles - bj tiles)
    int64_t rem = blockIdx.x;
    int64_t bj = 0;
    while (rem >= ntiles - bj) {
        rem -= ntiles - bj;
        ++bj;
    }
    const int64_t bk = bj + rem;
    const int t = threadIdx.x;
    const int tx = t & 15, ty = t >> 4;
    const int64_t j0 = bj * BF_T, k0 = bk * BF_T;

    uint32_t acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b)
            acc[a][b] = 0;

    const int lw = t & 31;          // word within the chunk this thread loads
    const int lc = t >> 5;          // first column it loads (then every 8th)
    for (int64_t w0 = 0; w0 < W; w0 += BF_K) {
        const int64_t w = w0 + lw;
        const bool inw = w < W;
        const uint32_t yw = inw ? yb[w] : 0u;
#pragma unroll 4
        for (int i = 0; i < BF_T / 8; ++i) {
            const int col = lc + 8 * i;
            const int64_t cj = j0 + col, ck = k0 + col;
            // words past W: z = 0, x = ~0, so ~(z ^ x) = 0 adds nothing
            zs[lw][col] = (inw && cj < p) ? (Xc[cj * Wp + w] ^ yw) : 0u;
            xs[lw][col] = (inw && ck < p) ? Xc[ck * Wp + w] : (inw ? 0u : 0xFFFFFFFFu);
        }
        __syncthreads();
#pragma unroll 2
        for (int ww = 0; ww < BF_K; ++ww) {
            const uint4 z0 = *reinterpret_cast<const uint4 *>(&zs[ww][ty * 8]);
            const uint4 z1 = *reinterpret_cast<const uint4 *>(&zs[ww][ty * 8 + 4]);
            const uint4 x0 = *reinterpret_cast<const uint4 *>(&xs[ww][tx * 8]);
            const uint4 x1 = *reinterpret_cast<const uint4 *>(&xs[ww][tx * 8 + 4]);
            const uint32_t zj[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
            const uint32_t xk[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b)
                    acc[a][b] += __popc(~(zj[a] ^ xk[b]));
        }
        __syncthreads();
    }

    // passing pairs j < k < p, warp-aggregated appends
    const unsigned FULL = 0xffffffffu;
    const int lane = t & 31;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int64_t j = j0 + ty * 8 + a;
        uint32_t keep = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int64_t k = k0 + tx * 8 + b;
            if (j < k && k < p && (int64_t)acc[a][b] >= amin)
                keep |= 1u << b;
        }
        const uint32_t cnt = __popc(keep);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o)
                incl += y;
        }
        const uint32_t wtot = __shfl_sync(FULL, incl, 31);
        if (wtot == 0)
            continue;
        uint32_t base = 0;
        if (lane == 31)
            base = atomicAdd(nrec, wtot);
        base = __shfl_sync(FULL, base, 31);
        uint32_t o = base + incl - cnt;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            if ((keep >> b) & 1u) {
                if (o < rec_cap) {
                    const uint64_t k = (uint64_t)(k0 + tx * 8 + b);
                    rec_keys[o] = ((uint64_t)j << kbits) | k;
                    rec_agree[o] = acc[a][b];
                }
                ++o;
            }
        }
    }
}

}  // namespace

int64_t brute_tiles(int64_t p)
{
    const int64_t nt = (p + BF_T - 1) / BF_T;
    return nt * (nt + 1) / 2;
}

cudaError_t launch_brute(const Packed &pk, int64_t amin, int kbits, uint64_t *rec_keys,
                         uint32_t *rec_agree, uint32_t *nrec, uint32_t rec_cap, cudaStream_t s,
                         int64_t *launches)
{
    const int64_t nt = (pk.p + BF_T - 1) / BF_T;
    const int64_t blocks = nt * (nt + 1) / 2;
    if (blocks > 0x7FFFFFFFLL)
        return cudaErrorInvalidValue;
    brute_kernel<<<(unsigned)blocks, BF_THREADS, 0, s>>>(pk.Xc, pk.Wp, pk.W, pk.yb, pk.p, nt, amin, kbits,
                                                        rec_keys, rec_agree, nrec, rec_cap);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace xyz
