// Per-run survivor filter for the equal-pairs search (Algorithm 2 steps
// 3-4), used for M <= 31 when p is small enough for a shared-memory filter.
//
// In a run whose response key c is non-zero, a column can only be part of a
// candidate pair if some column on the other side of its canonical group
// exists (keys.cu: the group of column j is h = min(kx_j, kx_j ^ c), its side
// is whether kx_j != h).  Almost every column fails that test, so the sort
// that groups equal keys (radix.cu) only needs the few that pass.  One CTA
// (1024 threads) handles one run at a time:
//
//   pass 1  build the keys of all p columns (each thread: the words of the M
//           sampled rows, transposed in registers), store kx to the CTA's
//           L2-resident scratch in bit-major order (coalesced without
//           staging), and set two bits
//           of one word, chosen by hashes of h, in the shared-memory
//           blocked Bloom filter of the column's side;
//   pass 2  keep the columns whose h may be present on the other side (both
//           bits set in the other side's filter word) and append them, as
//           (run << M | Kc, j) with the canonical key Kc of keys.cu, to the
//           CTA's own output segment (warp-aggregated shared-memory cursor,
//           no global atomics).
//
// The survivors of a run (a few percent of its columns) are then grouped on
// chip into buckets and members, ready for verification; a run with too
// many survivors for the chip goes to the CTA's global segment instead, and
// a small second kernel concatenates the segments for the LSD sort and join
// of the general path.  A Bloom filter has no false negatives, so every true
// candidate survives; false positives are single-sided groups that never
// become buckets.  In a run with c == 0 every column survives.
#include <type_traits>

#include "bits.cuh"
#include "xyz_internal.cuh"

namespace xyz {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int FL_THREADS = 1024;
constexpr int FL_LOGB = 19;                       // filter bits per side
constexpr int FL_WORDS = 1 << (FL_LOGB - 5);      // 16384 words per side

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int64_t draw_row(uint64_t seed, uint64_t t, int64_t n)
{
    uint64_t u = mix64(seed + (t + 1ULL) * 0x9E3779B97F4A7C15ULL);
    return (int64_t)__umul64hi(u, (uint64_t)n);
}

// Blocked Bloom filter: a group value h selects one 32-bit word of its
// side's filter and two bits inside it, all from multiplicative hashes
// (Knuth's method with two odd constants, top bits).  Setting is one shared
// atomic OR, testing one shared load.
__device__ __forceinline__ void bloom_pos(uint32_t h, uint32_t &word, uint32_t &mask)
{
    word = (h * 0x9E3779B1u) >> (32 - (FL_LOGB - 5));
    const uint32_t y = h * 0x7FEB352Du + 0x165667B1u;
    mask = (1u << (y >> 27)) | (1u << ((y >> 22) & 31u));
}

constexpr int FL_SMAX = 6144;                    // survivors of one run grouped on chip
constexpr int FL_LOGT = 13;
constexpr int FL_T = 1 << FL_LOGT;                // table slots, in the filter's memory
constexpr uint32_t FL_EMPTY = 0xFFFFFFFFu;

// One CTA per run at a time.  Passes 1-2 as described at the top of the
// file; then, when the run has at most FL_SMAX survivors, they are grouped
// on chip: the 128 KB that held the two filters becomes a hash table of
// FL_T group keys with side counts, each group with candidates becomes a
// bucket (bucket and member space reserved with one global atomic pair per
// run) and its members are written side A first.  A run with more survivors
// (for example every column of a run whose c is 0) re-runs pass 2 into the
// CTA's global segment instead, as (run << M | Kc, j), for the general sort
// and join.  Spilled survivors carry ((b << rbits | run) << M) | Kc in 64-bit
// keys, run counted from the start of the search, and the per-CTA segments
// fill across launch groups: the search sorts all of them once at its end.
// kc_scratch holds, per CTA, the keys of its current run in bit-major
// order: kx of column 32w + cc at cc * P + w.
//
// BATCH: B responses share X and the row stream.  The keys of a run are
// built once; the filter, survivors and grouping then run once per response
// b (its response key c_b, its filters) and buckets carry b in their `pad`
// field.  cnz is indexed (b << rbits) | run.
template <int MB, bool BATCH>
__global__ void __launch_bounds__(FL_THREADS, 1)
    filter_kernel(const uint32_t *__restrict__ Xr, int64_t Pp, int64_t P,
                  const uint32_t *__restrict__ ybs, int64_t Wp, int B, int64_t n, int64_t p, int M,
                  uint64_t seed, int64_t l0, int R, int NB, int BB, int rbits, int64_t rbase,
                  uint32_t mcap, uint32_t bcap, uint32_t *__restrict__ kc_scratch,
                  void *__restrict__ seg_keys_v, uint32_t *__restrict__ seg_vals,
                  uint32_t *__restrict__ seg_count, uint32_t seg_cap, int *__restrict__ overflow,
                  uint8_t *__restrict__ cnz, uint32_t *__restrict__ members,
                  uint32_t *__restrict__ members_count, Bucket *__restrict__ buckets,
                  uint64_t *__restrict__ pair_counts, uint32_t *__restrict__ nbuckets)
{
    using SegKey = uint64_t;
    extern __shared__ __align__(16) uint32_t fl_smem[];
    uint32_t *bmA = fl_smem;                       // [FL_WORDS]   (passes 1-2)
    uint32_t *bmB = fl_smem + FL_WORDS;            // [FL_WORDS]
    uint32_t *tkey = fl_smem;                      // [FL_T]       (grouping)
    uint32_t *cA = fl_smem + FL_T;                 // [FL_T]
    uint32_t *cB = fl_smem + 2 * FL_T;             // [FL_T]
    uint32_t *tok = fl_smem + 3 * FL_T;            // [FL_T] 1 = group has a bucket
    uint64_t *sv = reinterpret_cast<uint64_t *>(fl_smem + 2 * FL_WORDS);   // [FL_SMAX]
    const int t = threadIdx.x;
    const int lane = t & 31, wp = t >> 5;
    __shared__ int64_t rowoff[32];      // row s_m times the row pitch
    __shared__ int64_t rowidx[32];      // row s_m
    __shared__ uint32_t c_sh;
    __shared__ uint32_t cursor;         // global segment fill
    __shared__ uint32_t ns;             // survivors of the current (run, response)
    __shared__ uint32_t wsum[FL_THREADS / 32];
    __shared__ uint32_t mbase_sh, bbase_sh;
    uint32_t *kcs = kc_scratch + (int64_t)blockIdx.x * 32 * P;
    SegKey *okeys = reinterpret_cast<SegKey *>(seg_keys_v) + (int64_t)blockIdx.x * seg_cap;
    uint32_t *ovals = seg_vals + (int64_t)blockIdx.x * seg_cap;
    const uint32_t P32 = (uint32_t)P, p32 = (uint32_t)p;
    const uint32_t steps = (P32 + FL_THREADS - 1) / FL_THREADS;
    if (t == 0)
        cursor = seg_count[blockIdx.x];     // segments fill across launch groups

    // work item = (run r, block of responses [b0, b1)); the keys of the run
    // are built once per item
    for (int item = blockIdx.x; item < R * NB; item += gridDim.x) {
        const int r = item / NB;
        const int b0 = (item - r * NB) * BB;
        const int b1 = (b0 + BB < B) ? b0 + BB : B;
        const uint64_t rl = (uint64_t)(rbase + r);   // run index within the search
        if (!BATCH)
            for (int i = t; i < 2 * FL_WORDS; i += FL_THREADS)
                fl_smem[i] = 0;
        if (wp == 0) {
            int64_t s = 0;
            if (lane < M)
                s = draw_row(seed, (uint64_t)(l0 + r) * (uint64_t)M + (uint64_t)lane, n);
            rowoff[lane] = s * Pp;
            rowidx[lane] = s;
            if (!BATCH) {
                const uint32_t ybit = lane < M ? (ybs[s >> 5] >> (s & 31)) & 1u : 0u;
                const uint32_t c = __ballot_sync(FULL, ybit);
                if (lane == 0) {
                    c_sh = c;
                    ns = 0;
                    cnz[rl] = (c != 0);
                }
            }
        }
        __syncthreads();

        // pass 1: keys to the scratch rows (and, for one response, the filter
        // bits of each side).  Rows at or past MB are zero at compile time.
        {
            const uint32_t c = BATCH ? 0u : c_sh;
            const bool nz = c != 0;
            for (uint32_t w = t; w < P32; w += FL_THREADS) {
                uint32_t A[32];
#pragma unroll
                for (int m = 0; m < 32; ++m)
                    A[m] = (m < MB && m < M) ? __ldg(Xr + rowoff[m] + w) : 0u;
                transpose32(A);
#pragma unroll
                for (int cc = 0; cc < 32; ++cc)
                    kcs[cc * P32 + w] = A[cc];         // bit-major: coalesced across the warp
                if (!BATCH && nz) {
                    const uint32_t ncol = (32 * w + 32 <= p32) ? 32u : p32 - 32 * w;
#pragma unroll
                    for (int cc = 0; cc < 32; ++cc) {
                        if ((uint32_t)cc < ncol) {
                            const uint32_t kx = A[cc];
                            const uint32_t kxc = kx ^ c;
                            const uint32_t h = kx < kxc ? kx : kxc;
                            uint32_t word, mask;
                            bloom_pos(h, word, mask);
                            atomicOr(((kx != h) ? bmB : bmA) + word, mask);
                        }
                    }
                }
            }
        }
        __syncthreads();

        for (int b = b0; b < b1; ++b) {
            if (BATCH) {
                // this response's key c_b and filters
                for (int i = t; i < 2 * FL_WORDS; i += FL_THREADS)
                    fl_smem[i] = 0;
                if (wp == 0) {
                    const int64_t s = rowidx[lane];
                    const uint32_t *ybb = ybs + (int64_t)b * Wp;
                    const uint32_t ybit = lane < M ? (ybb[s >> 5] >> (s & 31)) & 1u : 0u;
                    const uint32_t c = __ballot_sync(FULL, ybit);
                    if (lane == 0) {
                        c_sh = c;
                        ns = 0;
                        cnz[((uint64_t)b << rbits) | rl] = (c != 0);
                    }
                }
                __syncthreads();
                const uint32_t c = c_sh;
                if (c != 0) {
                    for (uint32_t cc = 0; cc < 32; ++cc)
                    for (uint32_t w = t; w < P32; w += FL_THREADS) {
                        if (32 * w + cc >= p32)
                            continue;
                        const uint32_t kx = kcs[cc * P32 + w];
                        const uint32_t kxc = kx ^ c;
                        const uint32_t h = kx < kxc ? kx : kxc;
                        uint32_t word, mask;
                        bloom_pos(h, word, mask);
                        atomicOr(((kx != h) ? bmB : bmA) + word, mask);
                    }
                }
                __syncthreads();
            }
            const uint32_t c = c_sh;
            const bool nz = c != 0;
            const int tb = nz ? 31 - __clz(c) : 0;
            const uint32_t lowmask = nz ? ((1u << tb) - 1u) : 0u;

            // pass 2: the survivors.  to_global = false: into the shared
            // survivor array (only counted past FL_SMAX); true: into the
            // CTA's global segment with the composite key.
            auto pass2 = [&](bool to_global) {
                const SegKey runbits = (SegKey)((((uint64_t)b << rbits) | rl) << M);
                for (uint32_t st = 0; st < steps; ++st) {
                    const uint32_t w = st * FL_THREADS + t;
                    uint32_t kv[32];
#pragma unroll
                    for (int cc = 0; cc < 32; ++cc)
                        kv[cc] = (w < P32) ? kcs[cc * P32 + w] : 0u;
                    uint32_t keep = 0;     // bit cc: column 32w + cc survives
                    if (w < P32) {
                        const uint32_t valid = (32 * w + 32 <= p32) ? 0xFFFFFFFFu
                                                                    : ((1u << (p32 - 32 * w)) - 1u);
                        if (!nz) {
                            keep = valid;
                        } else {
#pragma unroll
                            for (int cc = 0; cc < 32; ++cc) {
                                const uint32_t kx = kv[cc];
                                const uint32_t kxc = kx ^ c;
                                const uint32_t h = kx < kxc ? kx : kxc;
                                uint32_t word, mask;
                                bloom_pos(h, word, mask);
                                const uint32_t have = ((kx != h) ? bmA : bmB)[word];
                                keep |= ((have & mask) == mask ? 1u : 0u) << cc;
                            }
                            keep &= valid;
                        }
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
                    uint32_t wbase = 0;
                    if (lane == 31)
                        wbase = atomicAdd(to_global ? &cursor : &ns, wtot);
                    wbase = __shfl_sync(FULL, wbase, 31);
                    uint32_t o = wbase + incl - cnt;
                    while (keep) {
                        const int cc = __ffs(keep) - 1;
                        keep &= keep - 1;
                        const uint32_t kx = kcs[cc * P32 + w];   // survivors only: re-read, cache-hot
                        uint32_t key = kx;
                        if (nz) {
                            const uint32_t kxc = kx ^ c;
                            const uint32_t h = kx < kxc ? kx : kxc;
                            const uint32_t above = (h >> (tb + 1)) << tb;
                            key = ((above | (h & lowmask)) << 1) | ((kx != h) ? 1u : 0u);
                        }
                        if (to_global) {
                            if (o < seg_cap) {
                                okeys[o] = runbits | (SegKey)key;
                                ovals[o] = 32 * w + cc;
                            }
                        } else if (o < FL_SMAX) {
                            sv[o] = ((uint64_t)key << 32) | (32 * w + cc);
                        }
                        ++o;
                    }
                }
            };
            pass2(false);
            __syncthreads();
            const uint32_t s = ns;
            if (s > FL_SMAX) {
                pass2(true);            // too many for the chip: the general path groups them
                __syncthreads();
                continue;
            }

            // grouping on chip; the filters are dead, their memory is the table
            for (int i = t; i < FL_T; i += FL_THREADS) {
                tkey[i] = FL_EMPTY;
                cA[i] = 0;
                cB[i] = 0;
            }
            __syncthreads();
            // phase I: insert group keys, count sides; keep (side, slot, j)
            for (uint32_t i = t; i < s; i += FL_THREADS) {
                const uint64_t e = sv[i];
                const uint32_t Kc = (uint32_t)(e >> 32);
                const uint32_t g = nz ? (Kc >> 1) : Kc;
                const uint32_t side = nz ? (Kc & 1u) : 0u;
                uint32_t slot = (g * 0x9E3779B1u) >> (32 - FL_LOGT);
                for (int probe = 0; probe < FL_T; ++probe) {     // s < FL_T: always ends
                    const uint32_t old = atomicCAS(&tkey[slot], FL_EMPTY, g);
                    if (old == FL_EMPTY || old == g)
                        break;
                    slot = (slot + 1) & (FL_T - 1);
                }
                atomicAdd(side ? &cB[slot] : &cA[slot], 1u);
                sv[i] = ((uint64_t)((side << 31) | slot) << 32) | (uint32_t)e;
            }
            __syncthreads();
            // phase II: groups with candidates -> buckets; one global atomic
            // pair per (run, response) reserves their space
            {
                constexpr int PER = FL_T / FL_THREADS;
                uint32_t packed[PER];          // members << 16 | buckets of each slot
                uint32_t mysum = 0;
#pragma unroll
                for (int q = 0; q < PER; ++q) {
                    const int slot = t * PER + q;
                    uint32_t v = 0;
                    if (tkey[slot] != FL_EMPTY) {
                        const uint32_t nA = cA[slot], nB = cB[slot];
                        const bool ok = nz ? (nA > 0 && nB > 0) : (nA > 1);
                        if (ok)
                            v = ((nA + nB) << 16) | 1u;
                    }
                    packed[q] = v;
                    mysum += v;
                }
                uint32_t incl = mysum;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o)
                        incl += y;
                }
                if (lane == 31)
                    wsum[wp] = incl;
                __syncthreads();
                uint32_t before = 0, total = 0;
                for (int i = 0; i < FL_THREADS / 32; ++i) {
                    before += (i < wp) ? wsum[i] : 0u;
                    total += wsum[i];
                }
                if (t == 0) {
                    const uint32_t mt = total >> 16, bt = total & 0xFFFFu;
                    mbase_sh = bt ? atomicAdd(members_count, mt) : 0u;
                    bbase_sh = bt ? atomicAdd(nbuckets, bt) : 0u;
                    if (bt && ((uint64_t)mbase_sh + mt > mcap || (uint64_t)bbase_sh + bt > bcap)) {
                        atomicOr(overflow, 2);      // host grows the space and redoes the search
                        mbase_sh = 0xFFFFFFFFu;
                    }
                }
                __syncthreads();
                if (mbase_sh == 0xFFFFFFFFu)
                    continue;
                uint32_t run_off = before + incl - mysum;
#pragma unroll
                for (int q = 0; q < PER; ++q) {
                    const int slot = t * PER + q;
                    const uint32_t v = packed[q];
                    tok[slot] = v ? 1u : 0u;
                    if (v) {
                        const uint32_t nA = cA[slot], nB = cB[slot];
                        const uint32_t base = mbase_sh + (run_off >> 16);
                        const uint32_t bi = bbase_sh + (run_off & 0xFFFFu);
                        buckets[bi] = Bucket{base, nA, nz ? nB : 0u, (uint32_t)b};
                        pair_counts[bi] = nz ? (uint64_t)nA * nB : (uint64_t)nA * (nA - 1) / 2;
                        cA[slot] = base + nA;          // end of side A: cursor counts down
                        cB[slot] = base + nA + nB;     // end of side B
                    }
                    run_off += v;
                }
            }
            __syncthreads();
            // phase III: members, side A first
            for (uint32_t i = t; i < s; i += FL_THREADS) {
                const uint64_t e = sv[i];
                const uint32_t hi = (uint32_t)(e >> 32);
                const uint32_t slot = hi & 0x7FFFFFFFu;
                if (!tok[slot])
                    continue;
                const uint32_t pos = atomicSub((hi >> 31) ? &cB[slot] : &cA[slot], 1u) - 1u;
                members[pos] = (uint32_t)e;
            }
            __syncthreads();
        }
    }
    if (t == 0) {
        seg_count[blockIdx.x] = cursor < seg_cap ? cursor : seg_cap;
        if (cursor > seg_cap)
            atomicOr(overflow, 1);
    }
}

// Zero the per-CTA segment fills before a search.
__global__ void seg_reset_kernel(uint32_t *seg_count, int n)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        seg_count[i] = 0;
}

// Concatenate the CTA segments: block b copies segment b to the sum of the
// counts before it; the last block stores the total.
template <typename K>
__global__ void __launch_bounds__(256)
    compact_kernel(const K *__restrict__ seg_keys, const uint32_t *__restrict__ seg_vals,
                   const uint32_t *__restrict__ seg_count, uint32_t seg_cap, int nseg,
                   K *__restrict__ out_keys, uint32_t *__restrict__ out_vals,
                   uint32_t *__restrict__ total)
{
    __shared__ uint32_t base_sh;
    const int b = blockIdx.x;
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int i = 0; i < b; ++i)
            s += seg_count[i];
        base_sh = s;
        if (b == nseg - 1)
            *total = s + seg_count[b];
    }
    __syncthreads();
    const uint32_t base = base_sh, cnt = seg_count[b];
    const K *sk = seg_keys + (int64_t)b * seg_cap;
    const uint32_t *sv = seg_vals + (int64_t)b * seg_cap;
    for (uint32_t i = threadIdx.x; i < cnt; i += 256) {
        out_keys[base + i] = sk[i];
        out_vals[base + i] = sv[i];
    }
}

}  // namespace

bool filter_supported(int64_t p, int M) { return M <= 31 && p <= 262144; }

size_t filter_smem_bytes() { return (size_t)(2 * FL_WORDS) * 4 + (size_t)FL_SMAX * 8; }

int64_t filter_run_cap() { return FL_SMAX; }

int filter_grid()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 152;
}

size_t filter_scratch_words(int64_t p) { return (size_t)filter_grid() * 32 * (size_t)((p + 31) / 32); }

cudaError_t launch_seg_reset(uint32_t *seg_count, cudaStream_t s, int64_t *launches)
{
    seg_reset_kernel<<<1, 256, 0, s>>>(seg_count, filter_grid());
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_compact(const uint64_t *seg_keys, const uint32_t *seg_vals,
                           const uint32_t *seg_count, uint32_t seg_cap, int nseg, uint64_t *out_keys,
                           uint32_t *out_vals, uint32_t *total, cudaStream_t s, int64_t *launches)
{
    compact_kernel<uint64_t><<<nseg, 256, 0, s>>>(seg_keys, seg_vals, seg_count, seg_cap, nseg,
                                                  out_keys, out_vals, total);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_filter(const Packed &pk, const uint32_t *ybs, int B, int M, uint64_t seed,
                          int64_t l0, int R, int NB, int BB, int rbits, int64_t rbase, int grid,
                          uint32_t mcap, uint32_t bcap, uint32_t *kc_scratch, uint64_t *seg_keys,
                          uint32_t *seg_vals, uint32_t *seg_count, uint32_t seg_cap, int *overflow,
                          uint8_t *cnz, uint32_t *members, uint32_t *members_count, Bucket *buckets,
                          uint64_t *pair_counts, uint32_t *nbuckets, cudaStream_t s,
                          int64_t *launches)
{
    const size_t smem = filter_smem_bytes();
    const bool batch = B > 1;
    using KernT = void (*)(const uint32_t *, int64_t, int64_t, const uint32_t *, int64_t, int, int64_t,
                           int64_t, int, uint64_t, int64_t, int, int, int, int, int64_t, uint32_t, uint32_t,
                           uint32_t *, void *, uint32_t *, uint32_t *, uint32_t, int *, uint8_t *,
                           uint32_t *, uint32_t *, Bucket *, uint64_t *, uint32_t *);
    KernT kern;
    if (batch)
        kern = M <= 8 ? filter_kernel<8, true> : M <= 16 ? filter_kernel<16, true>
               : M <= 24 ? filter_kernel<24, true> : filter_kernel<32, true>;
    else
        kern = M <= 8 ? filter_kernel<8, false> : M <= 16 ? filter_kernel<16, false>
               : M <= 24 ? filter_kernel<24, false> : filter_kernel<32, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    kern<<<grid, FL_THREADS, smem, s>>>(pk.Xr, pk.Pp, pk.P, ybs, pk.Wp, B, pk.n, pk.p, M, seed, l0, R,
                                        NB, BB, rbits, rbase, mcap, bcap, kc_scratch, seg_keys, seg_vals,
                                        seg_count, seg_cap, overflow, cnz, members, members_count,
                                        buckets, pair_counts, nbuckets);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace xyz
