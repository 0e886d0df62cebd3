// K3 radix sort and exclusive scans.
//
// The equal-pairs search of Section 2.2 sorts the keys of a run and walks
// the distinct values.  Here the keys of a whole launch group of runs are
// sorted at once (the run index occupies the high key bits) with a stable
// LSD radix sort on 8-bit digits: per pass an upsweep writes a 256-bin
// digit histogram per 4096-entry tile (digit-major, so one exclusive scan
// of the histogram table yields every (digit, tile) output offset), and a
// downsweep ranks each tile's entries stably with warp match-any and
// per-warp counters in shared memory, then scatters them.
#include "xyz_internal.cuh"

namespace xyz {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;   // 4096 entries

constexpr int SC_THREADS = 512;
constexpr int SC_ITEMS = 8;
constexpr int SC_BLOCK = SC_THREADS * SC_ITEMS;  // 4096 elements

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename K>
__global__ void __launch_bounds__(RS_THREADS)
    radix_upsweep(const K *__restrict__ keys, int64_t N, int shift, uint32_t *__restrict__ counts,
                  int64_t ntiles)
{
    __shared__ uint32_t hist[256];
    const int lane = threadIdx.x & 31;
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int it = 0; it < RS_ITEMS; ++it) {
        int64_t idx = base + (int64_t)it * RS_THREADS + threadIdx.x;
        bool valid = idx < N;
        uint32_t d = valid ? (uint32_t)((keys[idx] >> shift) & 255u) : 256u;
        uint32_t peers = __match_any_sync(FULL, d);
        if (valid && lane == __ffs(peers) - 1)
            atomicAdd(&hist[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = hist[threadIdx.x];
}

template <typename K>
__global__ void __launch_bounds__(RS_THREADS)
    radix_downsweep(const K *__restrict__ kin, const uint32_t *__restrict__ vin,
                    K *__restrict__ kout, uint32_t *__restrict__ vout, int64_t N, int shift,
                    const uint32_t *__restrict__ offsets, int64_t ntiles)
{
    __shared__ uint32_t wcnt[RS_WARPS][256];
    __shared__ uint32_t tile_off[256];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS)
        wcnt[i / 256][i % 256] = 0;
    tile_off[threadIdx.x] = offsets[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();

    const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * (32 * RS_ITEMS);
    const unsigned lt = lanemask_lt();
    K k[RS_ITEMS];
    uint32_t v[RS_ITEMS];
    uint32_t rank[RS_ITEMS];
    uint32_t dig[RS_ITEMS];
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        int64_t idx = base + it * 32 + lane;
        bool valid = idx < N;
        k[it] = valid ? kin[idx] : (K)0;
        v[it] = valid ? vin[idx] : 0u;
        uint32_t d = valid ? (uint32_t)((k[it] >> shift) & 255u) : 256u;
        uint32_t peers = __match_any_sync(FULL, d);
        uint32_t before = valid ? wcnt[warp][d] : 0u;
        __syncwarp();
        if (valid && (peers & lt) == 0)
            wcnt[warp][d] = before + (uint32_t)__popc(peers);
        __syncwarp();
        rank[it] = before + (uint32_t)__popc(peers & lt);
        dig[it] = d;
    }
    __syncthreads();
    {
        // exclusive prefix of each digit's count over the warps of the tile
        uint32_t d = threadIdx.x, run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            uint32_t cnt = wcnt[w][d];
            wcnt[w][d] = run;
            run += cnt;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        uint32_t d = dig[it];
        if (d < 256u) {
            int64_t pos = (int64_t)tile_off[d] + wcnt[warp][d] + rank[it];
            kout[pos] = k[it];
            vout[pos] = v[it];
        }
    }
}

// ----------------------------------------------------------------- scans

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(FULL, x, o);
        if (lane >= o)
            x += y;
    }
    return x;
}

// Exclusive scan of one value per thread across the block; returns the
// block total through *total.
template <typename T, int THREADS>
__device__ __forceinline__ T block_excl_scan(T x, T *total)
{
    __shared__ T wsum[THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = warp_incl_scan(x, lane);
    if (lane == 31)
        wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = lane < THREADS / 32 ? wsum[lane] : (T)0;
        w = warp_incl_scan(w, lane);
        if (lane < THREADS / 32)
            wsum[lane] = w;
    }
    __syncthreads();
    T excl = incl - x + (warp > 0 ? wsum[warp - 1] : (T)0);
    *total = wsum[THREADS / 32 - 1];
    __syncthreads();
    return excl;
}

__device__ __forceinline__ int64_t scan_count(const uint32_t *count_dev, int64_t count_host)
{
    if (!count_dev)
        return count_host;
    int64_t c = (int64_t)*count_dev;
    return c < count_host ? c : count_host;
}

template <typename T>
__global__ void __launch_bounds__(SC_THREADS)
    scan_reduce(const T *__restrict__ in, const uint32_t *count_dev, int64_t cap,
                T *__restrict__ partials)
{
    const int64_t N = scan_count(count_dev, cap);
    const int64_t base = (int64_t)blockIdx.x * SC_BLOCK;
    if (base >= N)
        return;
    T s = 0;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        int64_t idx = base + (int64_t)i * SC_THREADS + threadIdx.x;
        if (idx < N)
            s += in[idx];
    }
    T total;
    block_excl_scan<T, SC_THREADS>(s, &total);
    if (threadIdx.x == 0)
        partials[blockIdx.x] = total;
}

template <typename T>
__global__ void __launch_bounds__(1024)
    scan_partials(T *__restrict__ partials, const uint32_t *count_dev, int64_t cap,
                  T *__restrict__ total_out, T *__restrict__ total_accum)
{
    const int64_t N = scan_count(count_dev, cap);
    const int64_t nb = (N + SC_BLOCK - 1) / SC_BLOCK;
    T carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
        int64_t i = b0 + threadIdx.x;
        T x = i < nb ? partials[i] : (T)0;
        T total;
        T ex = block_excl_scan<T, 1024>(x, &total);
        if (i < nb)
            partials[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) {
        if (total_out)
            *total_out = carry;
        if (total_accum)
            *total_accum += carry;
    }
}

template <typename T>
__global__ void __launch_bounds__(SC_THREADS)
    scan_down(const T *__restrict__ in, T *__restrict__ out, const uint32_t *count_dev,
              int64_t cap, const T *__restrict__ partials)
{
    const int64_t N = scan_count(count_dev, cap);
    const int64_t base = (int64_t)blockIdx.x * SC_BLOCK;
    if (base >= N)
        return;
    const int64_t first = base + (int64_t)threadIdx.x * SC_ITEMS;
    T x[SC_ITEMS];
    T s = 0;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        int64_t idx = first + i;
        x[i] = idx < N ? in[idx] : (T)0;
        s += x[i];
    }
    T total;
    T ex = block_excl_scan<T, SC_THREADS>(s, &total) + partials[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        int64_t idx = first + i;
        if (idx < N)
            out[idx] = ex;
        ex += x[i];
    }
}

template <typename T>
cudaError_t scan_impl(const T *in, T *out, const uint32_t *count_dev, int64_t cap, T *total_out,
                      T *total_accum, void *temp, cudaStream_t s, int64_t *launches)
{
    if (cap <= 0)
        return cudaSuccess;
    T *partials = reinterpret_cast<T *>(temp);
    int64_t nb = (cap + SC_BLOCK - 1) / SC_BLOCK;
    scan_reduce<T><<<(unsigned)nb, SC_THREADS, 0, s>>>(in, count_dev, cap, partials);
    scan_partials<T><<<1, 1024, 0, s>>>(partials, count_dev, cap, total_out, total_accum);
    scan_down<T><<<(unsigned)nb, SC_THREADS, 0, s>>>(in, out, count_dev, cap, partials);
    *launches += 3;
    return cudaGetLastError();
}

int64_t tiles_for(int64_t N) { return (N + RS_TILE - 1) / RS_TILE; }

template <typename K>
cudaError_t radix_impl(K *k0, uint32_t *v0, K *k1, uint32_t *v1, int64_t N, int bits, void *temp,
                       bool *in_alt, cudaStream_t s, int64_t *launches)
{
    *in_alt = false;
    if (N <= 1 || bits <= 0)
        return cudaSuccess;
    const int64_t nt = tiles_for(N);
    uint32_t *counts = reinterpret_cast<uint32_t *>(temp);
    uint32_t *scan_tmp = counts + 256 * nt;
    K *ks = k0, *kd = k1;
    uint32_t *vs = v0, *vd = v1;
    for (int shift = 0; shift < bits; shift += 8) {
        radix_upsweep<K><<<(unsigned)nt, RS_THREADS, 0, s>>>(ks, N, shift, counts, nt);
        *launches += 1;
        cudaError_t e = scan_impl<uint32_t>(counts, counts, nullptr, 256 * nt, nullptr, nullptr,
                                            scan_tmp, s, launches);
        if (e != cudaSuccess)
            return e;
        radix_downsweep<K><<<(unsigned)nt, RS_THREADS, 0, s>>>(ks, vs, kd, vd, N, shift, counts, nt);
        *launches += 1;
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
        K *tk = ks; ks = kd; kd = tk;
        uint32_t *tv = vs; vs = vd; vd = tv;
        *in_alt = !*in_alt;
    }
    return cudaSuccess;
}

}  // namespace

int radix_passes(int bits) { return bits <= 0 ? 0 : (bits + 7) / 8; }

size_t scan_temp_bytes(int64_t cap)
{
    int64_t nb = (cap + SC_BLOCK - 1) / SC_BLOCK + 1;
    return (size_t)nb * sizeof(uint64_t) + 256;
}

size_t radix_temp_bytes(int64_t N)
{
    int64_t nt = tiles_for(N < 1 ? 1 : N);
    return (size_t)256 * nt * sizeof(uint32_t) + scan_temp_bytes(256 * nt) + 256;
}

cudaError_t radix_sort32(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, int64_t N, int bits,
                         void *temp, bool *in_alt, cudaStream_t s, int64_t *launches)
{
    return radix_impl<uint32_t>(k0, v0, k1, v1, N, bits, temp, in_alt, s, launches);
}

cudaError_t radix_sort64(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int64_t N, int bits,
                         void *temp, bool *in_alt, cudaStream_t s, int64_t *launches)
{
    return radix_impl<uint64_t>(k0, v0, k1, v1, N, bits, temp, in_alt, s, launches);
}

cudaError_t scan_u64_dev(const uint64_t *in, uint64_t *out, const uint32_t *count_dev, int64_t cap,
                         uint64_t *total_out, uint64_t *total_accum, void *temp, cudaStream_t s,
                         int64_t *launches)
{
    return scan_impl<uint64_t>(in, out, count_dev, cap, total_out, total_accum, temp, s, launches);
}

cudaError_t scan_u32_dev(const uint32_t *in, uint32_t *out, const uint32_t *count_dev, int64_t cap,
                         uint32_t *total_out, void *temp, cudaStream_t s, int64_t *launches)
{
    return scan_impl<uint32_t>(in, out, count_dev, cap, total_out, nullptr, temp, s, launches);
}

}  // namespace xyz
