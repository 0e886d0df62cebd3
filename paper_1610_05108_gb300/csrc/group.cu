// Partitioned equal-pairs search (the projection and equal-pairs steps of
// Algorithm 2, Section 2.2) for M <= 31, in two kernels per launch group of
// R runs.
//
// keybuild_part: one thread per (run, 32-column word).  The thread loads
// the word of each of the M sampled rows (neighbouring threads read
// neighbouring words, so every row read is coalesced), transposes the
// M x 32 bit tile in registers (transpose32: plain ALU, no warp votes) to
// get the M-bit keys kx of its 32 columns, and forms the canonical key Kc
// (see keys.cu: groups of Kc >> 1 are the candidate groups when c != 0, with
// the side in bit 0; Kc = kx when c == 0).  A block owns 4096 consecutive
// columns of one run and counting-sorts its entries (Kc << 32 | j) by
// partition q = top d bits of mix32(group key) into its own region of the
// entry array, writing one (offset, count) word per (run, partition, block)
// to the segment table.  Keys are computed once and written once.
//
// group: one CTA per (run, partition).  It gathers the partition's segments
// (L2-resident), inserts every group key into a shared-memory hash table
// (open addressing, probe length bounded by the table size) counting side-A
// and side-B members, turns each group with candidates into a bucket whose
// members it writes contiguously (A then B) to the member array, and
// appends the bucket's pair count.  If a partition holds more distinct
// groups than the table takes, the CTA splits it by further bits of the
// same hash and handles the halves one after the other; equal keys never
// split, so a heavy group costs one table slot however large it is.
#include "bits.cuh"
#include "rows.cuh"
#include "xyz_internal.cuh"

namespace xyz {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int KP_THREADS = 128;
constexpr int KP_COLS = KP_THREADS * 32;      // columns per block
constexpr int GR_THREADS = 256;
constexpr int GR_LOGT = 11;
constexpr int GR_T = 1 << GR_LOGT;            // hash table slots
constexpr uint32_t GR_MAXDIST = GR_T * 3 / 4; // distinct groups per pass
constexpr uint32_t EMPTY = 0xFFFFFFFFu;
constexpr int GR_STACK = 64;
constexpr int GR_CACHE = 8;                  // entries per thread kept in registers

__device__ __forceinline__ uint32_t group_key(uint32_t Kc, bool nz) { return nz ? (Kc >> 1) : Kc; }

__device__ __forceinline__ uint32_t part_of(uint32_t g, int d)
{
    return d ? (mix32(g) >> (32 - d)) : 0u;
}

__global__ void __launch_bounds__(KP_THREADS)
    keybuild_part_kernel(const uint32_t *__restrict__ Xr, int64_t Pp, int64_t P,
                         const uint32_t *__restrict__ yb, int64_t n, int64_t p, int M,
                         uint64_t seed, int64_t l0, int d, int nblk, uint64_t *__restrict__ ents,
                         uint32_t *__restrict__ seg, uint8_t *__restrict__ cnz,
                         const uint64_t *__restrict__ cdf, uint64_t wtot)
{
    extern __shared__ __align__(16) unsigned char kp_smem[];
    uint64_t *ent = reinterpret_cast<uint64_t *>(kp_smem);                 // [KP_COLS]
    uint16_t *rk = reinterpret_cast<uint16_t *>(ent + KP_COLS);            // [KP_COLS]
    uint32_t *hist = reinterpret_cast<uint32_t *>(rk + KP_COLS);           // [Q]
    uint32_t *excl = hist + (1 << d);                                      // [Q]
    __shared__ int64_t rows[32];
    __shared__ uint32_t c_sh;
    __shared__ uint32_t wsum[KP_THREADS / 32];

    const int t = threadIdx.x;
    const int r = blockIdx.y;
    const int b = blockIdx.x;
    const int Q = 1 << d;
    const int64_t run = l0 + r;
    for (int q = t; q < Q; q += KP_THREADS)
        hist[q] = 0;
    if (t < 32) {
        int64_t s = 0;
        uint32_t ybit = 0;
        if (t < M) {
            s = draw_row(seed, (uint64_t)run * (uint64_t)M + (uint64_t)t, n, cdf, wtot);
            ybit = (yb[s >> 5] >> (s & 31)) & 1u;
        }
        rows[t] = s;
        uint32_t c = __ballot_sync(FULL, ybit);
        if (t == 0) {
            c_sh = c;
            if (b == 0)
                cnz[r] = (c != 0);
        }
    }
    __syncthreads();
    const uint32_t c = c_sh;
    const bool nz = c != 0;
    const int tb = nz ? 31 - __clz(c) : 0;
    const uint32_t lowmask = nz ? ((1u << tb) - 1u) : 0u;

    const int64_t w = (int64_t)b * KP_THREADS + t;
    uint32_t A[32];
#pragma unroll
    for (int m = 0; m < 32; ++m)
        A[m] = (m < M && w < P) ? __ldg(Xr + rows[m] * Pp + w) : 0u;
    transpose32(A);

#pragma unroll
    for (int cc = 0; cc < 32; ++cc) {
        const int64_t j = 32 * w + cc;
        uint64_t e = ~0ULL;
        uint16_t rank = 0;
        if (w < P && j < p) {
            const uint32_t kx = A[cc];
            uint32_t Kc;
            if (!nz) {
                Kc = kx;
            } else {
                const uint32_t kxc = kx ^ c;
                const uint32_t h = kx < kxc ? kx : kxc;
                const uint32_t side = (kx != h) ? 1u : 0u;
                const uint32_t above = (h >> (tb + 1)) << tb;
                Kc = ((above | (h & lowmask)) << 1) | side;
            }
            const uint32_t q = part_of(group_key(Kc, nz), d);
            rank = (uint16_t)atomicAdd(&hist[q], 1u);
            e = ((uint64_t)Kc << 32) | (uint32_t)j;
        }
        ent[cc * KP_THREADS + t] = e;
        rk[cc * KP_THREADS + t] = rank;
    }
    __syncthreads();

    // exclusive scan of the block histogram (Q <= 4096 bins, 128 threads)
    {
        const int per = (Q + KP_THREADS - 1) / KP_THREADS;
        const int q0 = t * per;
        uint32_t s = 0;
        for (int i = 0; i < per; ++i)
            if (q0 + i < Q)
                s += hist[q0 + i];
        const int lane = t & 31, wp = t >> 5;
        uint32_t incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o)
                incl += y;
        }
        if (lane == 31)
            wsum[wp] = incl;
        __syncthreads();
        uint32_t base = 0;
        for (int i = 0; i < wp; ++i)
            base += wsum[i];
        uint32_t run_s = base + incl - s;
        for (int i = 0; i < per; ++i)
            if (q0 + i < Q) {
                excl[q0 + i] = run_s;
                run_s += hist[q0 + i];
            }
    }
    __syncthreads();

    uint64_t *region = ents + (int64_t)r * p + (int64_t)b * KP_COLS;
#pragma unroll 4
    for (int cc = 0; cc < 32; ++cc) {
        const uint64_t e = ent[cc * KP_THREADS + t];
        if (e != ~0ULL) {
            const uint32_t q = part_of(group_key((uint32_t)(e >> 32), nz), d);
            region[excl[q] + rk[cc * KP_THREADS + t]] = e;
        }
    }
    for (int q = t; q < Q; q += KP_THREADS)
        seg[((int64_t)r * Q + q) * nblk + b] = (excl[q] << 16) | hist[q];
}

// Shared-memory state of one group CTA.
struct GroupSmem {
    uint32_t tkey[GR_T];     // group key, EMPTY when free
    uint32_t cntA[GR_T];     // side-A members (count, then cursor)
    uint32_t cntB[GR_T];     // side-B members
    uint32_t baseA[GR_T];    // first member slot of side A, EMPTY if no bucket
    uint32_t baseB[GR_T];    // first member slot of side B
    uint16_t used[GR_T];     // slots claimed in the current pass
    uint32_t stk_v[GR_STACK];
    int stk_e[GR_STACK];
    uint32_t wsum[GR_THREADS / 32];
    uint32_t nused;
    uint32_t ndist;
    int sp;
    int ovf;
};

__device__ __forceinline__ uint32_t slot_of(uint32_t h) { return (h * 0x9E3779B1u) >> (32 - GR_LOGT); }

__global__ void __launch_bounds__(GR_THREADS)
    group_kernel(const uint64_t *__restrict__ ents, const uint32_t *__restrict__ seg, int64_t p,
                 int d, int nblk, int64_t nparts, const uint8_t *__restrict__ cnz,
                 uint32_t *__restrict__ members, uint32_t *__restrict__ members_count,
                 Bucket *__restrict__ buckets, uint64_t *__restrict__ pair_counts,
                 uint32_t *__restrict__ nbuckets, int *__restrict__ err)
{
    __shared__ GroupSmem S;
    extern __shared__ uint32_t gr_dyn[];
    uint32_t *pre = gr_dyn;               // [nblk + 1] exclusive prefix of segment counts
    uint32_t *off = gr_dyn + nblk + 1;    // [nblk] segment offsets in their block regions
    const int t = threadIdx.x;
    const int lane = t & 31, wp = t >> 5;

    for (int i = t; i < GR_T; i += GR_THREADS) {
        S.tkey[i] = EMPTY;
        S.cntA[i] = 0;
        S.cntB[i] = 0;
    }
    if (t == 0)
        S.nused = 0;

    for (int64_t part = blockIdx.x; part < nparts; part += gridDim.x) {
        const int64_t r = part >> d;
        const bool nz = cnz[r] != 0;
        const uint64_t *run_ents = ents + r * p;
        __syncthreads();

        // segment table of this partition -> exclusive prefix of counts
        uint32_t carry = 0;
        for (int b0 = 0; b0 < nblk; b0 += GR_THREADS) {
            const int bb = b0 + t;
            uint32_t cntv = 0;
            if (bb < nblk) {
                const uint32_t v = seg[part * nblk + bb];
                cntv = v & 0xFFFFu;
                off[bb] = v >> 16;
            }
            uint32_t incl = cntv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o)
                    incl += y;
            }
            if (lane == 31)
                S.wsum[wp] = incl;
            __syncthreads();
            uint32_t base = carry, tot = 0;
#pragma unroll
            for (int i = 0; i < GR_THREADS / 32; ++i) {
                base += (i < wp) ? S.wsum[i] : 0u;
                tot += S.wsum[i];
            }
            if (bb < nblk)
                pre[bb] = base + incl - cntv;
            carry += tot;
            __syncthreads();
        }
        if (t == 0) {
            pre[nblk] = carry;
            S.sp = 1;
            S.stk_v[0] = 0;
            S.stk_e[0] = 0;
        }
        __syncthreads();
        const uint32_t s = carry;

        auto load = [&](uint32_t i) -> uint64_t {
            int lo = 0, hi = nblk;     // pre[lo] <= i < pre[hi]
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (pre[mid] <= i)
                    lo = mid;
                else
                    hi = mid;
            }
            return run_ents[(int64_t)lo * KP_COLS + off[lo] + (i - pre[lo])];
        };

        // the first GR_CACHE * GR_THREADS entries stay in registers
        uint64_t ec[GR_CACHE];
#pragma unroll
        for (int k = 0; k < GR_CACHE; ++k) {
            const uint32_t i = t + k * GR_THREADS;
            ec[k] = i < s ? load(i) : 0ULL;
        }

        while (true) {
            const int cur_sp = S.sp;
            if (cur_sp == 0)
                break;
            const uint32_t v = S.stk_v[cur_sp - 1];
            const int eb = S.stk_e[cur_sp - 1];
            const uint32_t emask = eb ? ((1u << eb) - 1u) : 0u;
            __syncthreads();
            if (t == 0) {
                S.sp = cur_sp - 1;
                S.ovf = 0;
                S.ndist = 0;
            }
            __syncthreads();

            // phase 1: insert group keys, count the two sides
            uint32_t sl[GR_CACHE];
            auto insert = [&](uint64_t e) -> uint32_t {
                const uint32_t Kc = (uint32_t)(e >> 32);
                const uint32_t g = group_key(Kc, nz);
                const uint32_t h = mix32(g);
                if ((h & emask) != v)
                    return EMPTY;
                uint32_t slot = slot_of(h);
                for (int probe = 0; probe < GR_T; ++probe) {
                    const uint32_t old = atomicCAS(&S.tkey[slot], EMPTY, g);
                    if (old == EMPTY) {
                        S.used[atomicAdd(&S.nused, 1u)] = (uint16_t)slot;
                        if (atomicAdd(&S.ndist, 1u) >= GR_MAXDIST)
                            S.ovf = 1;
                        break;
                    }
                    if (old == g)
                        break;
                    slot = (slot + 1) & (GR_T - 1);
                    if (probe + 1 == GR_T) {
                        S.ovf = 1;
                        return EMPTY;
                    }
                }
                atomicAdd((nz && (Kc & 1u)) ? &S.cntB[slot] : &S.cntA[slot], 1u);
                return slot;
            };
#pragma unroll
            for (int k = 0; k < GR_CACHE; ++k) {
                const uint32_t i = t + k * GR_THREADS;
                sl[k] = (i < s && !*(volatile int *)&S.ovf) ? insert(ec[k]) : EMPTY;
            }
            for (uint32_t i = t + GR_CACHE * GR_THREADS; i < s; i += GR_THREADS) {
                if (*(volatile int *)&S.ovf)
                    break;
                insert(load(i));
            }
            __syncthreads();
            const bool overflow = S.ovf != 0;
            if (!overflow) {
                // phase 2: groups with candidates become buckets
                const uint32_t nu = S.nused;
                for (uint32_t u = t; u < nu; u += GR_THREADS) {
                    const uint32_t slot = S.used[u];
                    const uint32_t nA = S.cntA[slot], nB = S.cntB[slot];
                    const bool valid = nz ? (nA > 0 && nB > 0) : (nA > 1);
                    uint32_t base = EMPTY;
                    if (valid) {
                        base = atomicAdd(members_count, nA + nB);
                        const uint32_t bi = atomicAdd(nbuckets, 1u);
                        buckets[bi] = Bucket{base, nA, nz ? nB : 0u, 0u};
                        pair_counts[bi] = nz ? (uint64_t)nA * nB : (uint64_t)nA * (nA - 1) / 2;
                        S.baseB[slot] = base + nA;
                    }
                    S.baseA[slot] = base;
                }
                __syncthreads();
                // phase 3: members, counting the side counters back down to 0
                auto place = [&](uint64_t e, uint32_t slot) {
                    const uint32_t bA = S.baseA[slot];
                    if (bA == EMPTY)
                        return;
                    const bool sideB = nz && ((uint32_t)(e >> 32) & 1u);
                    const uint32_t pos = sideB ? S.baseB[slot] + atomicSub(&S.cntB[slot], 1u) - 1u
                                               : bA + atomicSub(&S.cntA[slot], 1u) - 1u;
                    members[pos] = (uint32_t)e;
                };
#pragma unroll
                for (int k = 0; k < GR_CACHE; ++k)
                    if (sl[k] != EMPTY)
                        place(ec[k], sl[k]);
                for (uint32_t i = t + GR_CACHE * GR_THREADS; i < s; i += GR_THREADS) {
                    const uint64_t e = load(i);
                    const uint32_t g = group_key((uint32_t)(e >> 32), nz);
                    const uint32_t h = mix32(g);
                    if ((h & emask) != v)
                        continue;
                    uint32_t slot = slot_of(h);
                    for (int probe = 0; probe < GR_T && S.tkey[slot] != g; ++probe)
                        slot = (slot + 1) & (GR_T - 1);
                    if (S.tkey[slot] == g)
                        place(e, slot);
                }
            } else if (t == 0) {
                // too many distinct groups in this pass: split by one more hash bit
                if (eb >= 30 || S.sp + 2 > GR_STACK) {
                    atomicOr(err, 1);
                } else {
                    S.stk_v[S.sp] = v;
                    S.stk_e[S.sp] = eb + 1;
                    S.stk_v[S.sp + 1] = v | (1u << eb);
                    S.stk_e[S.sp + 1] = eb + 1;
                    S.sp += 2;
                }
            }
            __syncthreads();
            // clean the slots this pass used
            const uint32_t nu = S.nused;
            for (uint32_t u = t; u < nu; u += GR_THREADS) {
                const uint32_t slot = S.used[u];
                S.tkey[slot] = EMPTY;
                S.cntA[slot] = 0;
                S.cntB[slot] = 0;
            }
            __syncthreads();
            if (t == 0)
                S.nused = 0;
            __syncthreads();
        }
    }
}

// ------------------------------------------------- warp-per-partition path
//
// The same grouping with one warp per partition: a warp-private hash table
// (GW_T slots of key, side-A count, side-B count), no block barriers, and
// the partition's bucket/member space reserved with one pair of global
// atomics per partition.  Lanes holding the same group key are merged with
// __match_any_sync first, so a heavy group costs one table update per warp
// step instead of 32 serialised atomics.  After counting, a valid group's
// two counters are replaced by the end positions of its A and B member
// ranges and serve as decrementing cursors while members are placed.
constexpr int GW_WARPS = 7;
constexpr int GW_LOGT = 10;
constexpr int GW_T = 1 << GW_LOGT;
constexpr uint32_t GW_MAXDIST = GW_T * 3 / 4;
constexpr int GW_MAXBLK = 256;
constexpr int GW_CACHE = 12;
constexpr int GW_STACK = 32;
constexpr uint32_t NOKEY = 0xFFFFFFFFu;   // never a group key (keys have <= 31 bits)

// Per-warp shared memory: fixed part, then pre[nblk+1] and off[nblk].
struct WarpFixed {
    uint32_t key[GW_T];
    uint32_t ca[GW_T];
    uint32_t cb[GW_T];
    uint16_t used[GW_T];
    uint32_t stk_v[GW_STACK];
    int stk_e[GW_STACK];
    uint32_t nused;
    int ovf;
};

__host__ __device__ constexpr size_t warp_words(int nblk)
{
    return (sizeof(WarpFixed) + 3) / 4 + (size_t)(2 * nblk + 1);
}

__device__ __forceinline__ uint32_t wslot_of(uint32_t h) { return (h * 0x9E3779B1u) >> (32 - GW_LOGT); }

__global__ void __launch_bounds__(GW_WARPS * 32)
    group_warp_kernel(const uint64_t *__restrict__ ents, const uint32_t *__restrict__ seg, int64_t p,
                      int d, int nblk, int64_t nparts, const uint8_t *__restrict__ cnz,
                      uint32_t *__restrict__ members, uint32_t *__restrict__ members_count,
                      Bucket *__restrict__ buckets, uint64_t *__restrict__ pair_counts,
                      uint32_t *__restrict__ nbuckets, int *__restrict__ err)
{
    extern __shared__ __align__(16) uint32_t gw_smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint32_t *wbase = gw_smem + (size_t)wib * warp_words(nblk);
    WarpFixed &W = *reinterpret_cast<WarpFixed *>(wbase);
    uint32_t *pre = wbase + (sizeof(WarpFixed) + 3) / 4;   // [nblk + 1]
    uint32_t *off = pre + nblk + 1;                        // [nblk]
    const unsigned lt = (1u << lane) - 1u;

    for (int i = lane; i < GW_T; i += 32) {
        W.key[i] = EMPTY;
        W.ca[i] = 0;
        W.cb[i] = 0;
    }
    if (lane == 0)
        W.nused = 0;
    __syncwarp();

    const int64_t warps_total = (int64_t)gridDim.x * GW_WARPS;
    for (int64_t part = (int64_t)blockIdx.x * GW_WARPS + wib; part < nparts; part += warps_total) {
        const int64_t r = part >> d;
        const bool nz = cnz[r] != 0;
        const uint64_t *run_ents = ents + r * p;

        // segments -> exclusive prefix of counts
        uint32_t carry = 0;
        for (int b0 = 0; b0 < nblk; b0 += 32) {
            const int bb = b0 + lane;
            uint32_t cntv = 0;
            if (bb < nblk) {
                const uint32_t v = seg[part * nblk + bb];
                cntv = v & 0xFFFFu;
                off[bb] = v >> 16;
            }
            uint32_t incl = cntv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o)
                    incl += y;
            }
            if (bb < nblk)
                pre[bb] = carry + incl - cntv;
            carry += __shfl_sync(FULL, incl, 31);
        }
        if (lane == 0) {
            pre[nblk] = carry;
            W.stk_v[0] = 0;
            W.stk_e[0] = 0;
        }
        __syncwarp();
        const uint32_t s = carry;
        if (s == 0)
            continue;

        auto load = [&](uint32_t i) -> uint64_t {
            int lo = 0, hi = nblk;     // pre[lo] <= i < pre[hi]
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (pre[mid] <= i)
                    lo = mid;
                else
                    hi = mid;
            }
            return run_ents[(int64_t)lo * KP_COLS + off[lo] + (i - pre[lo])];
        };

        uint64_t ec[GW_CACHE];
#pragma unroll
        for (int k = 0; k < GW_CACHE; ++k) {
            const uint32_t i = lane + 32 * k;
            ec[k] = i < s ? load(i) : 0ULL;
        }
        // warp-uniform number of steps over the entries past the cache
        const uint32_t tail_steps = s > 32u * GW_CACHE ? (s - 32u * GW_CACHE + 31u) / 32u : 0u;

        int sp = 1;                    // warp-uniform stack depth
        while (sp > 0) {
            --sp;
            const uint32_t v = W.stk_v[sp];
            const int eb = W.stk_e[sp];
            const uint32_t emask = eb ? ((1u << eb) - 1u) : 0u;
            if (lane == 0)
                W.ovf = 0;
            __syncwarp();

            // phase 1: insert and count; all lanes call this together
            auto insert = [&](bool have, uint64_t e) -> uint32_t {
                const uint32_t Kc = (uint32_t)(e >> 32);
                const uint32_t g = group_key(Kc, nz);
                const uint32_t h = mix32(g);
                const bool mine = have && ((h & emask) == v);
                const uint32_t gk = mine ? g : NOKEY;
                const unsigned peers = __match_any_sync(FULL, gk);
                const int leader = __ffs(peers) - 1;
                const bool sideB = nz && (Kc & 1u);
                const unsigned bmask = __ballot_sync(FULL, mine && sideB);
                uint32_t slot = EMPTY;
                if (mine && lane == leader) {
                    slot = wslot_of(h);
                    for (int probe = 0;; ++probe) {
                        if (probe == GW_T) {
                            W.ovf = 1;
                            slot = EMPTY;
                            break;
                        }
                        const uint32_t old = atomicCAS(&W.key[slot], EMPTY, g);
                        if (old == EMPTY) {
                            const uint32_t u = atomicAdd(&W.nused, 1u);
                            W.used[u] = (uint16_t)slot;
                            if (u + 1 > GW_MAXDIST)
                                W.ovf = 1;
                            break;
                        }
                        if (old == g)
                            break;
                        slot = (slot + 1) & (GW_T - 1);
                    }
                    if (slot != EMPTY) {
                        const uint32_t nb = __popc(peers & bmask);
                        const uint32_t na = __popc(peers) - nb;
                        if (na)
                            atomicAdd(&W.ca[slot], na);
                        if (nb)
                            atomicAdd(&W.cb[slot], nb);
                    }
                }
                slot = __shfl_sync(FULL, slot, leader);
                return mine ? slot : EMPTY;
            };
            uint32_t sl[GW_CACHE];
#pragma unroll
            for (int k = 0; k < GW_CACHE; ++k) {
                const uint32_t i = lane + 32 * k;
                sl[k] = (32u * k < s) ? insert(i < s, ec[k]) : EMPTY;
            }
            for (uint32_t st = 0; st < tail_steps; ++st) {
                __syncwarp();
                if (*(volatile int *)&W.ovf)       // same value in every lane
                    break;
                const uint32_t i = 32u * GW_CACHE + 32u * st + lane;
                insert(i < s, i < s ? load(i) : 0ULL);
            }
            __syncwarp();
            const bool overflow = *(volatile int *)&W.ovf != 0;
            const uint32_t nu = W.nused;

            if (!overflow) {
                // phase 2: reserve the warp's buckets and members with one
                // atomic pair, then give each group its ranges
                uint32_t my_b = 0, my_m = 0;
                for (uint32_t u = lane; u < nu; u += 32) {
                    const uint32_t i = W.used[u];
                    const uint32_t nA = W.ca[i], nB = W.cb[i];
                    if (nz ? (nA > 0 && nB > 0) : (nA > 1)) {
                        my_b += 1;
                        my_m += nA + nB;
                    }
                }
                uint32_t inc_b = my_b, inc_m = my_m;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t yb = __shfl_up_sync(FULL, inc_b, o);
                    uint32_t ym = __shfl_up_sync(FULL, inc_m, o);
                    if (lane >= o) {
                        inc_b += yb;
                        inc_m += ym;
                    }
                }
                const uint32_t tot_b = __shfl_sync(FULL, inc_b, 31);
                const uint32_t tot_m = __shfl_sync(FULL, inc_m, 31);
                uint32_t bb0 = 0, mb0 = 0;
                if (lane == 0 && tot_b) {
                    bb0 = atomicAdd(nbuckets, tot_b);
                    mb0 = atomicAdd(members_count, tot_m);
                }
                bb0 = __shfl_sync(FULL, bb0, 0) + inc_b - my_b;
                mb0 = __shfl_sync(FULL, mb0, 0) + inc_m - my_m;
                for (uint32_t u = lane; u < nu; u += 32) {
                    const uint32_t i = W.used[u];
                    const uint32_t nA = W.ca[i], nB = W.cb[i];
                    if (nz ? (nA > 0 && nB > 0) : (nA > 1)) {
                        buckets[bb0] = Bucket{mb0, nA, nz ? nB : 0u, 0u};
                        pair_counts[bb0] = nz ? (uint64_t)nA * nB : (uint64_t)nA * (nA - 1) / 2;
                        W.ca[i] = mb0 + nA;            // end of side A
                        W.cb[i] = mb0 + nA + nB;       // end of side B
                        ++bb0;
                        mb0 += nA + nB;
                    } else {
                        W.ca[i] = EMPTY;
                    }
                }
                __syncwarp();
                // phase 3: place members; lanes of one (group, side) take one
                // cursor step together
                auto place = [&](uint32_t slot, uint64_t e) {
                    const bool have = slot != EMPTY && W.ca[slot] != EMPTY;
                    const bool sideB = nz && ((uint32_t)(e >> 32) & 1u);
                    const uint32_t tag = have ? (slot << 1) | (sideB ? 1u : 0u) : NOKEY;
                    const unsigned peers = __match_any_sync(FULL, tag);
                    const int leader = __ffs(peers) - 1;
                    uint32_t top = 0;
                    if (have && lane == leader)
                        top = atomicSub(sideB ? &W.cb[slot] : &W.ca[slot], (uint32_t)__popc(peers));
                    top = __shfl_sync(FULL, top, leader);
                    if (have)
                        members[top - 1u - __popc(peers & lt)] = (uint32_t)e;
                };
#pragma unroll
                for (int k = 0; k < GW_CACHE; ++k)
                    if (32u * k < s)
                        place(sl[k], ec[k]);
                for (uint32_t st = 0; st < tail_steps; ++st) {
                    const uint32_t i = 32u * GW_CACHE + 32u * st + lane;
                    uint32_t slot = EMPTY;
                    uint64_t e = 0;
                    if (i < s) {
                        e = load(i);
                        const uint32_t g = group_key((uint32_t)(e >> 32), nz);
                        const uint32_t h = mix32(g);
                        if ((h & emask) == v) {
                            slot = wslot_of(h);
                            for (int probe = 0; probe < GW_T && W.key[slot] != g; ++probe)
                                slot = (slot + 1) & (GW_T - 1);
                            if (W.key[slot] != g)
                                slot = EMPTY;
                        }
                    }
                    place(slot, e);
                }
            } else if (lane == 0) {
                if (eb >= 30 || sp + 2 > GW_STACK) {
                    atomicOr(err, 1);
                } else {
                    W.stk_v[sp] = v;
                    W.stk_e[sp] = eb + 1;
                    W.stk_v[sp + 1] = v | (1u << eb);
                    W.stk_e[sp + 1] = eb + 1;
                }
            }
            if (overflow && eb < 30 && sp + 2 <= GW_STACK)
                sp += 2;
            __syncwarp();
            // clean the slots this pass used
            for (uint32_t u = lane; u < nu; u += 32) {
                const uint32_t i = W.used[u];
                W.key[i] = EMPTY;
                W.ca[i] = 0;
                W.cb[i] = 0;
            }
            __syncwarp();
            if (lane == 0)
                W.nused = 0;
            __syncwarp();
        }
    }
}

}  // namespace

int part_bits(int64_t p)
{
    // about 512 entries per partition on average
    int d = 0;
    while (d < 12 && (p >> (d + 9)) > 0)
        ++d;
    return d;
}

int part_blocks(int64_t p) { return (int)((p + KP_COLS - 1) / KP_COLS); }

bool part_supported(int64_t p, int M) { return M <= 31 && part_blocks(p) <= 4096; }

size_t part_seg_words(int64_t p, int R) { return (size_t)R * ((size_t)1 << part_bits(p)) * part_blocks(p); }

cudaError_t launch_keybuild_part(const Packed &pk, int M, uint64_t seed, int64_t l0, int R,
                                 uint64_t *ents, uint32_t *seg, uint8_t *cnz, cudaStream_t s,
                                 int64_t *launches)
{
    const int d = part_bits(pk.p);
    const int nblk = part_blocks(pk.p);
    const size_t smem = (size_t)KP_COLS * (8 + 2) + 2 * ((size_t)1 << d) * 4;
    cudaError_t ae = cudaFuncSetAttribute(keybuild_part_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    if (ae != cudaSuccess)
        return ae;
    dim3 grid((unsigned)nblk, (unsigned)R);
    keybuild_part_kernel<<<grid, KP_THREADS, smem, s>>>(pk.Xr, pk.Pp, pk.P, pk.yb, pk.n, pk.p, M,
                                                        seed, l0, d, nblk, ents, seg, cnz, pk.cdf,
                                                        pk.wtotal);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_group(const Packed &pk, int R, const uint64_t *ents, const uint32_t *seg,
                         const uint8_t *cnz, uint32_t *members, uint32_t *members_count,
                         Bucket *buckets, uint64_t *pair_counts, uint32_t *nbuckets, int *err,
                         cudaStream_t s, int64_t *launches)
{
    const int d = part_bits(pk.p);
    const int nblk = part_blocks(pk.p);
    const size_t dyn = (size_t)(2 * nblk + 1) * 4;
    cudaError_t ae =
        cudaFuncSetAttribute(group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024);
    if (ae != cudaSuccess)
        return ae;
    const int64_t parts = (int64_t)R << d;
    int dev = 0, sms = 0, per_sm = 0;
    if (nblk <= GW_MAXBLK) {
        const size_t wsm = warp_words(nblk) * 4 * GW_WARPS;
        cudaError_t we = cudaFuncSetAttribute(group_warp_kernel,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm);
        if (we != cudaSuccess)
            return we;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, group_warp_kernel, GW_WARPS * 32, wsm);
        int64_t grid = (int64_t)(sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 1);
        const int64_t need = (parts + GW_WARPS - 1) / GW_WARPS;
        if (grid > need)
            grid = need;
        group_warp_kernel<<<(unsigned)grid, GW_WARPS * 32, wsm, s>>>(
            ents, seg, pk.p, d, nblk, parts, cnz, members, members_count, buckets, pair_counts,
            nbuckets, err);
        *launches += 1;
        return cudaGetLastError();
    }
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, group_kernel, GR_THREADS, dyn);
    int64_t grid = (int64_t)(sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 1);
    if (grid > parts)
        grid = parts;
    group_kernel<<<(unsigned)grid, GR_THREADS, dyn, s>>>(ents, seg, pk.p, d, nblk, parts, cnz,
                                                         members, members_count, buckets,
                                                         pair_counts, nbuckets, err);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace xyz
