// K2 keybuild: the projection step of Algorithm 2 for a group of runs.
//
// Run l draws M rows s_0..s_{M-1} (eq. projR, subsampling with replacement)
// from the splitmix64 counter stream, and column j gets the key
//     kx_j = sum_m bit(X_{s_m j}) 2^m,   bit(v) = 1 iff v = -1.
// The Z-key of column k is kz_k = kx_k xor c with c = sum_m bit(Y_{s_m}) 2^m,
// because bit(Y_s X_sk) = bit(Y_s) xor bit(X_sk).  Equal real projections
// x_j = z_k (F = U[0,1]) happen exactly when kx_j = kz_k.
//
// Canonical key.  With c != 0, (j, k) is a candidate iff kx_j = kx_k xor c,
// i.e. iff j and k share h = min(kx, kx xor c) and lie on different sides
// (kx = h or kx = h xor c).  h always has bit t = msb(c) clear, so dropping
// that bit and appending the side as the lowest bit gives an M-bit key
// whose equal-prefix groups are exactly the candidate groups, with side A
// entries sorted before side B.  With c == 0 every column collides only with
// columns of the same kx, so the key is kx itself.  The run index within
// the launch group sits above the M key bits, so one sort groups all runs.
//
// One warp handles 8 row words (256 columns) of one run.  Lane m loads the
// 32 bytes of row s_m (and s_{m+32} when M > 32) with two 16-byte loads; a
// warp ballot per bit position transposes the M x 32 bit tile so that lane b
// ends up with the key of column 32w + b.  Stores are coalesced.
#include "rows.cuh"
#include "xyz_internal.cuh"

namespace xyz {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int KB_WARPS = 8;

__device__ __forceinline__ uint32_t transpose_take(uint32_t word, int lane)
{
    uint32_t key = 0;
#pragma unroll
    for (int b = 0; b < 32; ++b) {
        uint32_t bal = __ballot_sync(FULL, (word >> b) & 1u);
        key = (lane == b) ? bal : key;
    }
    return key;
}

template <typename K>
__global__ void __launch_bounds__(KB_WARPS * 32)
    keybuild_kernel(const uint32_t *__restrict__ Xr, int64_t Pp, int64_t P,
                    const uint32_t *__restrict__ yb, int64_t n, int64_t p, int M, uint64_t seed,
                    int64_t l0, int rbits, K *__restrict__ keys, uint32_t *__restrict__ vals,
                    uint8_t *__restrict__ cnz, uint64_t *__restrict__ raw_kx,
                    uint64_t *__restrict__ raw_c, const uint64_t *__restrict__ cdf, uint64_t wtot)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int r = blockIdx.y;
    const int64_t run = l0 + r;
    const int64_t g = (int64_t)blockIdx.x * KB_WARPS + warp;   // 8-word group
    const int64_t w0 = g * 8;

    // rows of this run and the response key c
    int64_t s_lo = 0, s_hi = 0;
    uint32_t yb_lo = 0, yb_hi = 0;
    if (lane < M) {
        s_lo = draw_row(seed, (uint64_t)run * (uint64_t)M + (uint64_t)lane, n, cdf, wtot);
        yb_lo = (yb[s_lo >> 5] >> (s_lo & 31)) & 1u;
    }
    if (lane + 32 < M) {
        s_hi = draw_row(seed, (uint64_t)run * (uint64_t)M + (uint64_t)(lane + 32), n, cdf, wtot);
        yb_hi = (yb[s_hi >> 5] >> (s_hi & 31)) & 1u;
    }
    const uint64_t c = ((uint64_t)__ballot_sync(FULL, yb_hi) << 32) | __ballot_sync(FULL, yb_lo);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (cnz)
            cnz[r] = (c != 0);
        if (raw_c)
            raw_c[0] = c;
    }
    if (w0 >= P)
        return;   // whole warp leaves together

    uint32_t lo[8], hi[8];
    if (lane < M) {
        const uint4 *src = reinterpret_cast<const uint4 *>(Xr + s_lo * Pp + w0);
        uint4 a = __ldg(src), b = __ldg(src + 1);
        lo[0] = a.x; lo[1] = a.y; lo[2] = a.z; lo[3] = a.w;
        lo[4] = b.x; lo[5] = b.y; lo[6] = b.z; lo[7] = b.w;
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) lo[q] = 0;
    }
    const bool two = M > 32;
    if (two && lane + 32 < M) {
        const uint4 *src = reinterpret_cast<const uint4 *>(Xr + s_hi * Pp + w0);
        uint4 a = __ldg(src), b = __ldg(src + 1);
        hi[0] = a.x; hi[1] = a.y; hi[2] = a.z; hi[3] = a.w;
        hi[4] = b.x; hi[5] = b.y; hi[6] = b.z; hi[7] = b.w;
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) hi[q] = 0;
    }

    // canonical-key constants of this run
    const int t = c ? 63 - __clzll((long long)c) : 0;
    const uint64_t lowmask = c ? ((1ULL << t) - 1ULL) : 0ULL;
    const uint64_t runbits = (rbits > 0) ? ((uint64_t)r << M) : 0ULL;

#pragma unroll
    for (int q = 0; q < 8; ++q) {
        uint64_t kx = transpose_take(lo[q], lane);
        if (two)
            kx |= (uint64_t)transpose_take(hi[q], lane) << 32;
        const int64_t j = (w0 + q) * 32 + lane;
        if (j < p) {
            uint64_t kc;
            if (c == 0) {
                kc = kx;
            } else {
                uint64_t kxc = kx ^ c;
                uint64_t h = kx < kxc ? kx : kxc;
                uint64_t side = (kx != h) ? 1ULL : 0ULL;
                uint64_t above = (t >= 63) ? 0ULL : ((h >> (t + 1)) << t);
                kc = ((above | (h & lowmask)) << 1) | side;
            }
            const int64_t o = (int64_t)r * p + j;
            keys[o] = (K)(runbits | kc);
            vals[o] = (uint32_t)j;
            if (raw_kx)
                raw_kx[j] = kx;
        }
    }
}

template <typename K>
cudaError_t launch_keybuild(const Packed &pk, int M, uint64_t seed, int64_t l0, int R, int rbits,
                            K *keys, uint32_t *vals, uint8_t *cnz, uint64_t *raw_kx,
                            uint64_t *raw_c, cudaStream_t s, int64_t *launches)
{
    int64_t groups = (pk.P + 7) / 8;
    dim3 grid((unsigned)((groups + KB_WARPS - 1) / KB_WARPS), (unsigned)R);
    keybuild_kernel<K><<<grid, KB_WARPS * 32, 0, s>>>(pk.Xr, pk.Pp, pk.P, pk.yb, pk.n, pk.p, M, seed,
                                                      l0, rbits, keys, vals, cnz, raw_kx, raw_c,
                                                      pk.cdf, pk.wtotal);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_keybuild32(const Packed &pk, int M, uint64_t seed, int64_t l0, int R, int rbits,
                              uint32_t *keys, uint32_t *vals, uint8_t *cnz, uint64_t *raw_kx,
                              uint64_t *raw_c, cudaStream_t s, int64_t *launches)
{
    return launch_keybuild<uint32_t>(pk, M, seed, l0, R, rbits, keys, vals, cnz, raw_kx, raw_c, s,
                                     launches);
}

cudaError_t launch_keybuild64(const Packed &pk, int M, uint64_t seed, int64_t l0, int R, int rbits,
                              uint64_t *keys, uint32_t *vals, uint8_t *cnz, uint64_t *raw_kx,
                              uint64_t *raw_c, cudaStream_t s, int64_t *launches)
{
    return launch_keybuild<uint64_t>(pk, M, seed, l0, R, rbits, keys, vals, cnz, raw_kx, raw_c, s,
                                     launches);
}

}  // namespace xyz
