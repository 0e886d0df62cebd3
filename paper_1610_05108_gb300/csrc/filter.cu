// Per-run survivor filter for the equal-pairs search (the projection and
// equal-pairs steps of Algorithm 2): filter_kernel for M <= 31 when p is
// small enough for one shared-memory filter of a run's keys,
// filter_big_kernel (further down) for larger p with the keys split into 16
// linear classes.
//
// In run l with response key c, columns j and k form a candidate exactly
// when kx_j ^ kx_k = c (keys.cu: X_j and Z_k agree on the sampled rows).  A
// column can therefore only be part of a candidate pair if the key kx_j ^ c
// is present among the run's column keys.  Almost every column fails that
// test, so the grouping of equal canonical keys only needs the few that
// pass.  One CTA (640-1024 threads) handles one run at a time:
//
//   pass 1  build the keys of all p columns (each thread: the words of the M
//           sampled rows, transposed in registers), store kx to the CTA's
//           L2-resident scratch in bit-major order (coalesced without
//           staging), and set two bits of one word, chosen by hashes of kx,
//           in the shared-memory blocked Bloom filter F of the run;
//   pass 2  keep the columns whose kx ^ c may be in F (both bits set) and
//           append them, as (Kc, j) with the canonical key Kc of keys.cu, to
//           the shared survivor array (warp-aggregated cursor).
//
// A Bloom filter has no false negatives, and when kx_j ^ c = kx_k both j and
// k pass (kx_k ^ c = kx_j), so every column of every candidate pair
// survives; false positives are groups with one side only, which yield no
// bucket.  When a run keeps more columns than the chip can group, the
// survivors are filtered again with a fresh filter built from the survivors
// alone (refinement: a candidate pair's columns are both survivors, so
// they still find each other), and what remains after a few rounds goes to
// the CTA's global segment: grouped from there on chip in hash partitions
// of the group keys, or, when one partition is still too large, left for
// the general sort and join.  The survivors of a run are grouped on chip
// into buckets and members, ready for verification.  In a run with c == 0
// every column survives.
#include <cstring>
#include <type_traits>

#include "bits.cuh"
#include "rows.cuh"
#include "xyz_internal.cuh"

namespace xyz {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int FL_THREADS = 1024;
constexpr int FL_LOGF = 20;                       // bits of the run filter F
constexpr int FL_FWORDS = 1 << (FL_LOGF - 5);     // 32768 words (128 KB)
constexpr int FL_LOGR = 13;
constexpr int FL_RWORDS = 1 << FL_LOGR;           // refinement filter, in the survivor array
constexpr int FL_KWORDS = 262144 / 32;            // keep-mask words: p <= 262144
constexpr int FL_LOGT_B = 13;                     // grouping table slots, batched kernel: 2^13
constexpr int FL_ROUNDS = 3;                      // refinement rounds at most
constexpr uint32_t FL_EMPTY = 0xFFFFFFFFu;

// Shared-memory layout, in 32-bit words.  One response per run: the filter
// F is dead once the survivors are known, so the grouping table takes its
// place and the survivor array can hold 8192 entries.  Several responses per
// run: F must outlive every response's grouping, so the table has its own
// region (where the keep mask also lives) and the survivor array holds 4096.
template <bool BATCH>
struct FlLayout {
    static constexpr int SMAX = BATCH ? 4096 : 8192;           // survivors grouped on chip
    static constexpr int LOGT = BATCH ? FL_LOGT_B : 14;        // grouping table slots: 2^LOGT
    static constexpr int T = 1 << LOGT;
    static constexpr int OFF_SV = FL_FWORDS;                   // [SMAX] u64 | refinement filter
    static constexpr int OFF_KM = OFF_SV + 2 * SMAX;           // [FL_KWORDS] keep mask
    static constexpr int OFF_TAB = BATCH ? OFF_KM : 0;         // [T] keys, [T] counts
    static constexpr int WORDS = BATCH ? OFF_TAB + 2 * T : OFF_KM + FL_KWORDS;
    static_assert(2 * SMAX >= FL_RWORDS, "the refinement filter fits the survivor array");
    static_assert(!BATCH || 2 * T >= FL_KWORDS, "the keep mask lies inside the table");
    static_assert(BATCH || 2 * T <= FL_FWORDS, "the table fits the filter's memory");
    static_assert(SMAX < T, "the table has a free slot for every survivor");
};

// Blocked Bloom filter of 2^k words: a key selects one 32-bit word and
// two bits inside it, all from multiplicative hashes (Knuth's method with
// two odd constants, top bits).  Setting is one shared atomic OR, testing
// one shared load.
__device__ __forceinline__ void bloom_pos(uint32_t h, int shift, uint32_t &word, uint32_t &mask)
{
    word = (h * 0x9E3779B1u) >> shift;          // shift = 32 - log2(filter words)
    const uint32_t y = h * 0x7FEB352Du + 0x165667B1u;
    // bits y >> 27 and (y >> 22) mod 32; the funnel shift takes its amount mod 32
    mask = (1u << (y >> 27)) | __funnelshift_l(1u, 1u, y >> 22);
}

// 1 when both bits of h are set in its word of F (the same positions as
// bloom_pos), else 0: two shifts of the loaded word instead of a mask.
__device__ __forceinline__ uint32_t bloom_has(const uint32_t *F, uint32_t h, int shift)
{
    const uint32_t f = F[(h * 0x9E3779B1u) >> shift];
    const uint32_t y = h * 0x7FEB352Du + 0x165667B1u;
    return (f >> (y >> 27)) & __funnelshift_r(f, f, y >> 22) & 1u;
}

// The same with three bits per key in the word (bits y >> 27, (y >> 22) mod
// 32 and (y >> 17) mod 32): fewer false positives for a filter whose words
// hold few keys each (the class-split filter's).
__device__ __forceinline__ void bloom_pos3(uint32_t h, int shift, uint32_t &word, uint32_t &mask)
{
    word = (h * 0x9E3779B1u) >> shift;
    const uint32_t y = h * 0x7FEB352Du + 0x165667B1u;
    mask = (1u << (y >> 27)) | __funnelshift_l(1u, 1u, y >> 22) | __funnelshift_l(1u, 1u, y >> 17);
}

__device__ __forceinline__ uint32_t bloom_has3(const uint32_t *F, uint32_t h, int shift)
{
    const uint32_t f = F[(h * 0x9E3779B1u) >> shift];
    const uint32_t y = h * 0x7FEB352Du + 0x165667B1u;
    return (f >> (y >> 27)) & __funnelshift_r(f, f, y >> 22) & __funnelshift_r(f, f, y >> 17) & 1u;
}

// Canonical key of a surviving column (keys.cu): group h = min(kx, kx ^ c)
// with bit tb = msb(c) removed, shifted left, side bit kx != h at the bottom.
__device__ __forceinline__ uint32_t canon(uint32_t kx, uint32_t c, int tb, uint32_t lowmask)
{
    if (c == 0)
        return kx;
    const uint32_t kxc = kx ^ c;
    const uint32_t h = kx < kxc ? kx : kxc;
    const uint32_t above = (h >> (tb + 1)) << tb;
    return ((above | (h & lowmask)) << 1) | ((kx != h) ? 1u : 0u);
}

// Where the on-chip grouping writes its buckets and members, and the
// space it may use (reserved with one global atomic pair per grouping).
struct GroupOut {
    uint32_t *members;
    uint32_t *members_count;
    Bucket *buckets;
    uint64_t *pair_counts;
    uint32_t *nbuckets;
    uint32_t mcap, bcap;
    int *overflow;
    unsigned long long *members_total;   // bucket members written, over the search
};

// Phase II of the on-chip grouping: every slot of the table (tkey / tcnt,
// side counts packed A << 16 | B) whose group has candidates becomes a
// bucket (response b in its pad); one global atomic pair per call reserves
// the bucket and member space.  With occ, only the nocc slots listed there
// (every occupied slot, in any order) are visited; otherwise all tsize.  Afterwards curA / tcnt of a bucket's slot are
// the end cursors of its sides A / B (curA may be tkey itself when phase III
// no longer needs the keys), and tcnt is FL_EMPTY for a slot without a
// bucket.  Returns false when the space ran out (overflow bit 2 set: the host
// grows it and redoes the search).  Called by every thread of the CTA.
__device__ __forceinline__ bool assign_buckets(uint32_t *tkey, uint32_t *tcnt, uint32_t *curA, int tsize, bool nz,
                                               int b, const GroupOut &g, const uint32_t *occ = nullptr,
                                               int nocc = 0)
{
    __shared__ uint32_t mbase_sh, bbase_sh;
    __shared__ uint32_t wsum[FL_THREADS / 32];
    const int t = threadIdx.x, T = (int)blockDim.x;
    const int lane = t & 31, wp = t >> 5, nwarps = T >> 5;
    // each thread owns a contiguous range of slots (of the list's entries
    // with occ); the value of a slot is members << 16 | 1 when its group
    // yields a bucket
    const int items = occ ? nocc : tsize;
    const int per = (items + T - 1) / T;
    const int s0 = t * per < items ? t * per : items;
    const int s1 = s0 + per < items ? s0 + per : items;
    auto slot_of = [&](int i) -> int { return occ ? (int)occ[i] : i; };
    auto slot_value = [&](int slot) -> uint32_t {
        if (tkey[slot] == FL_EMPTY)
            return 0u;
        const uint32_t nA = tcnt[slot] >> 16, nB = tcnt[slot] & 0xFFFFu;
        const bool ok = nz ? (nA > 0 && nB > 0) : (nA > 1);
        return ok ? ((nA + nB) << 16) | 1u : 0u;
    };
    uint32_t mysum = 0;
    for (int i = s0; i < s1; ++i)
        mysum += slot_value(slot_of(i));
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
    for (int i = 0; i < nwarps; ++i) {
        before += (i < wp) ? wsum[i] : 0u;
        total += wsum[i];
    }
    if (t == 0) {
        const uint32_t mt = total >> 16, bt = total & 0xFFFFu;
        mbase_sh = bt ? atomicAdd(g.members_count, mt) : 0u;
        bbase_sh = bt ? atomicAdd(g.nbuckets, bt) : 0u;
        if (bt && ((uint64_t)mbase_sh + mt > g.mcap || (uint64_t)bbase_sh + bt > g.bcap)) {
            atomicOr(g.overflow, 2);      // host grows the space and redoes the search
            mbase_sh = 0xFFFFFFFFu;
        } else if (bt) {
            atomicAdd(g.members_total, (unsigned long long)mt);
        }
    }
    __syncthreads();
    if (mbase_sh == 0xFFFFFFFFu)
        return false;
    uint32_t run_off = before + incl - mysum;
    for (int i = s0; i < s1; ++i) {
        const int slot = slot_of(i);
        const uint32_t v = slot_value(slot);
        if (v) {
            const uint32_t nA = tcnt[slot] >> 16, nB = tcnt[slot] & 0xFFFFu;
            const uint32_t base = mbase_sh + (run_off >> 16);
            const uint32_t bi = bbase_sh + (run_off & 0xFFFFu);
            g.buckets[bi] = Bucket{base, nA, nz ? nB : 0u, (uint32_t)b};
            g.pair_counts[bi] = nz ? (uint64_t)nA * nB : (uint64_t)nA * (nA - 1) / 2;
            curA[slot] = base + nA;          // end of side A: cursor counts down
            tcnt[slot] = base + nA + nB;     // end of side B
        } else {
            tcnt[slot] = FL_EMPTY;
        }
        run_off += v;
    }
    __syncthreads();
    return true;
}

// Groups the s <= SMAX survivors (Kc << 32 | j) in sv on chip: a hash table
// of group keys with packed side counts (tkey / tcnt); each group with
// candidates becomes a bucket (response b in its pad) and its members are
// written side A first.  occ (optional, room for s entries of shared memory
// outside the table and sv): the inserts list the slots they occupy there,
// and phase II visits only those.  Called by every thread of the CTA.
template <class Lay>
__device__ __forceinline__ void group_on_chip(uint64_t *sv, uint32_t s, uint32_t *tkey, uint32_t *tcnt, bool nz,
                                              int b, const GroupOut &g, uint32_t *occ = nullptr)
{
    __shared__ uint32_t nocc_sh;
    const int t = threadIdx.x, T = (int)blockDim.x;
    // grouping on chip in the table (the keep mask and, for one
    // response, the filter are dead)
    // table of 2^tlog slots, at least 4/3 of the survivors (load <= 3/4)
    int tlog = 8;
    while (tlog < Lay::LOGT && 3u * (1u << tlog) < 4 * s)
        ++tlog;
    const int tsize = 1 << tlog;
    for (int i = t; i < tsize; i += T) {
        tkey[i] = FL_EMPTY;
        tcnt[i] = 0;
    }
    if (t == 0)
        nocc_sh = 0;
    __syncthreads();
    // phase I: insert group keys, count sides (A high half, B low
    // half); keep (side, slot, j)
    for (uint32_t i = t; i < s; i += T) {
        const uint64_t e = sv[i];
        const uint32_t Kc = (uint32_t)(e >> 32);
        const uint32_t gk = nz ? (Kc >> 1) : Kc;
        const uint32_t side = nz ? (Kc & 1u) : 0u;
        uint32_t slot = (gk * 0x9E3779B1u) >> (32 - tlog);
        for (int probe = 0; probe < tsize; ++probe) {    // s < tsize: always ends
            const uint32_t old = atomicCAS(&tkey[slot], FL_EMPTY, gk);
            if (old == FL_EMPTY) {
                if (occ)
                    occ[atomicAdd(&nocc_sh, 1u)] = slot;   // at most s slots become occupied
                break;
            }
            if (old == gk)
                break;
            slot = (slot + 1) & (tsize - 1);
        }
        atomicAdd(&tcnt[slot], side ? 1u : 0x10000u);
        sv[i] = ((uint64_t)((side << 31) | slot) << 32) | (uint32_t)e;
    }
    __syncthreads();
    // phase II (the keys are not needed afterwards: tkey holds the side-A cursors)
    if (!assign_buckets(tkey, tcnt, tkey, tsize, nz, b, g, occ, (int)nocc_sh))
        return;              // the host grows the space and redoes the search
    // phase III: members, side A first
    for (uint32_t i = t; i < s; i += T) {
        const uint64_t e = sv[i];
        const uint32_t hi = (uint32_t)(e >> 32);
        const uint32_t slot = hi & 0x7FFFFFFFu;
        if (tcnt[slot] == FL_EMPTY)
            continue;
        const uint32_t pos = atomicSub((hi >> 31) ? &tcnt[slot] : &tkey[slot], 1u) - 1u;
        g.members[pos] = (uint32_t)e;
    }
    __syncthreads();
}

// The same grouping for a bin too large for sv, its n < 2^16 entries
// (Kc << 32 | j) read from global memory E: the table (all 2^LOGT slots)
// holds its distinct group keys, so it works whenever those number at most
// 3/4 of the table, however many entries share them (one group of tens of
// thousands of low-minor-frequency columns, say).  Phase III finds each
// entry's slot by probing again, so the side-A cursors go to curA (shared
// memory of 2^LOGT words outside the table).  Returns false, with nothing
// written, when the distinct keys did not fit.  Called by every thread.
template <class Lay>
__device__ __forceinline__ bool group_stream(const uint64_t *E, uint32_t n, uint32_t *tkey, uint32_t *tcnt,
                                             uint32_t *curA, bool nz, int b, const GroupOut &g)
{
    __shared__ uint32_t ndist, fail;
    constexpr int GS = 4;                 // entries per thread and step (loads in flight)
    const int t = threadIdx.x, T = (int)blockDim.x;
    const int tsize = Lay::T;
    const uint32_t limit = (uint32_t)(3 * tsize / 4);
    for (int i = t; i < tsize; i += T) {
        tkey[i] = FL_EMPTY;
        tcnt[i] = 0;
    }
    if (t == 0) {
        ndist = 0;
        fail = 0;
    }
    __syncthreads();
    // phase I: distinct keys into the table; a thread stops inserting once it
    // sees the limit passed, so at most limit + T slots are ever taken
    for (uint32_t i0 = t; i0 - t < n; i0 += GS * (uint32_t)T) {
        uint64_t e[GS];
#pragma unroll
        for (int u = 0; u < GS; ++u) {
            const uint32_t i = i0 + u * (uint32_t)T;
            e[u] = i < n ? E[i] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < GS; ++u) {
            if (i0 + u * (uint32_t)T >= n || *(volatile uint32_t *)&fail)
                continue;
            const uint32_t Kc = (uint32_t)(e[u] >> 32);
            const uint32_t gk = nz ? (Kc >> 1) : Kc;
            const uint32_t side = nz ? (Kc & 1u) : 0u;
            uint32_t slot = (gk * 0x9E3779B1u) >> (32 - Lay::LOGT);
            for (int probe = 0; probe < tsize; ++probe) {
                const uint32_t old = atomicCAS(&tkey[slot], FL_EMPTY, gk);
                if (old == FL_EMPTY) {
                    if (atomicAdd(&ndist, 1u) + 1u > limit)
                        fail = 1;
                    break;
                }
                if (old == gk)
                    break;
                slot = (slot + 1) & (tsize - 1);
            }
            atomicAdd(&tcnt[slot], side ? 1u : 0x10000u);
        }
    }
    __syncthreads();
    if (fail)
        return false;
    if (!assign_buckets(tkey, tcnt, curA, tsize, nz, b, g))
        return true;         // the host grows the space and redoes the search
    // phase III: members, side A first; each entry's slot found again
    for (uint32_t i0 = t; i0 - t < n; i0 += GS * (uint32_t)T) {
        uint64_t e[GS];
#pragma unroll
        for (int u = 0; u < GS; ++u) {
            const uint32_t i = i0 + u * (uint32_t)T;
            e[u] = i < n ? E[i] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < GS; ++u) {
            if (i0 + u * (uint32_t)T >= n)
                continue;
            const uint32_t Kc = (uint32_t)(e[u] >> 32);
            const uint32_t gk = nz ? (Kc >> 1) : Kc;
            const uint32_t side = nz ? (Kc & 1u) : 0u;
            uint32_t slot = (gk * 0x9E3779B1u) >> (32 - Lay::LOGT);
            for (int probe = 0; probe < tsize && tkey[slot] != gk; ++probe)
                slot = (slot + 1) & (tsize - 1);
            if (tcnt[slot] == FL_EMPTY)
                continue;
            const uint32_t pos = atomicSub(side ? &tcnt[slot] : &curA[slot], 1u) - 1u;
            g.members[pos] = (uint32_t)e[u];
        }
    }
    __syncthreads();
    return true;
}

// The s entries of one (run, response) at seg[seg0 ..) -- key runbits | Kc
// and column -- grouped on chip: they fall into 32 bins by a hash of their
// group key, and contiguous bin ranges of at most SMAX entries are gathered
// into sv and grouped one after the other (a group lies in one bin).
// Returns false, with nothing grouped, when a bin is above SMAX, more than
// part_max ranges are needed or the entries did not all fit the segment;
// the run then stays in the segment for the general path.  Called by every
// thread of the CTA.
template <class Lay>
__device__ __forceinline__ bool group_from_segment(const uint64_t *okeys, const uint32_t *ovals, uint32_t seg0,
                                                   uint32_t s, uint32_t seg_cap, int part_max, uint32_t kcmask,
                                                   uint64_t *sv, uint32_t *tkey, uint32_t *tcnt, bool nz, int b,
                                                   const GroupOut &g)
{
    __shared__ uint32_t hist[32];       // entries per bin of the group-key hash
    __shared__ uint32_t pstart[33];     // partition q covers bins [pstart[q], pstart[q + 1])
    __shared__ uint32_t nparts_sh, scur;
    constexpr int SMAX = Lay::SMAX;
    const int t = threadIdx.x, T = (int)blockDim.x;
    if (part_max <= 0 || (uint64_t)seg0 + s > seg_cap)
        return false;
    if (t < 32)
        hist[t] = 0;
    __syncthreads();
    constexpr int GB = 4;               // segment entries per thread and step (loads in flight)
    for (uint32_t i0 = t; i0 - t < s; i0 += GB * (uint32_t)T) {
        uint32_t Kc[GB];
#pragma unroll
        for (int u = 0; u < GB; ++u) {
            const uint32_t i = i0 + u * (uint32_t)T;
            Kc[u] = i < s ? (uint32_t)(okeys[seg0 + i] & kcmask) : 0u;
        }
#pragma unroll
        for (int u = 0; u < GB; ++u)
            if (i0 + u * (uint32_t)T < s)
                atomicAdd(&hist[mix32(nz ? (Kc[u] >> 1) : Kc[u]) >> 27], 1u);
    }
    __syncthreads();
    if (t == 0) {
        uint32_t np = 0, acc = 0;
        bool ok = true;
        pstart[0] = 0;
        for (int bn = 0; bn < 32; ++bn) {
            const uint32_t h = hist[bn];
            ok = ok && h <= (uint32_t)SMAX;
            if (acc + h > (uint32_t)SMAX) {
                pstart[++np] = (uint32_t)bn;
                acc = 0;
            }
            acc += h;
        }
        pstart[++np] = 32;
        nparts_sh = (ok && np <= (uint32_t)part_max) ? np : 0u;
    }
    __syncthreads();
    const uint32_t nparts = nparts_sh;
    if (nparts == 0)
        return false;
    for (uint32_t part = 0; part < nparts; ++part) {
        // this partition's entries from the segment to the survivor array
        if (t == 0)
            scur = 0;
        __syncthreads();
        const uint32_t blo = pstart[part], bhi = pstart[part + 1];
        for (uint32_t i0 = t; i0 - t < s; i0 += GB * (uint32_t)T) {
            uint32_t Kc[GB];
#pragma unroll
            for (int u = 0; u < GB; ++u) {
                const uint32_t i = i0 + u * (uint32_t)T;
                Kc[u] = i < s ? (uint32_t)(okeys[seg0 + i] & kcmask) : 0u;
            }
            bool in[GB];
            uint32_t col[GB];
#pragma unroll
            for (int u = 0; u < GB; ++u) {
                const uint32_t bn = mix32(nz ? (Kc[u] >> 1) : Kc[u]) >> 27;
                in[u] = i0 + u * (uint32_t)T < s && bn >= blo && bn < bhi;
                col[u] = in[u] ? ovals[seg0 + i0 + u * (uint32_t)T] : 0u;
            }
#pragma unroll
            for (int u = 0; u < GB; ++u)
                if (in[u])
                    sv[atomicAdd(&scur, 1u)] = ((uint64_t)Kc[u] << 32) | col[u];
        }
        __syncthreads();
        group_on_chip<Lay>(sv, scur, tkey, tcnt, nz, b, g);
    }
    return true;
}

// The s entries of one run at seg[seg0 ..) -- key runbits | Kc and column
// -- grouped on chip with one counting sort by a hash of the group key (32
// bins) into tmp (tmp_cap entries of global memory, Kc << 32 | column): the
// entries of contiguous bin ranges of at most SMAX entries are then copied
// to sv and grouped there, and a bin above SMAX is grouped straight from
// tmp (group_stream).  A bin whose distinct group keys do not fit the table
// is written back to the segment (runbits | Kc, column) for the general sort
// and join.  Returns the number of entries left in the segment at seg0, or
// GS_NONE when nothing was done because the run overflowed the segment or
// s > tmp_cap (the segment then still holds all of them).  occ: SMAX words
// of shared memory for the on-chip grouping's list of occupied slots.
// Called by every thread of the CTA.
constexpr uint32_t GS_NONE = 0xFFFFFFFFu;
template <class Lay>
__device__ __forceinline__ uint32_t group_segment_sorted(uint64_t *okeys, uint32_t *ovals, uint32_t seg0,
                                                         uint32_t s, uint32_t seg_cap, uint32_t kcmask,
                                                         uint64_t runbits, uint64_t *sv, uint32_t *tkey,
                                                         uint32_t *tcnt, bool nz, int b, const GroupOut &g,
                                                         uint64_t *tmp, uint32_t tmp_cap, uint32_t *occ)
{
    __shared__ uint32_t bstart[33];     // bin q of tmp: [bstart[q], bstart[q + 1])
    __shared__ uint32_t wsum2[FL_THREADS / 32];
    __shared__ uint32_t left_sh;
    constexpr int GB = 8;               // entries per thread and step (loads in flight)
    constexpr uint32_t SMAX = (uint32_t)Lay::SMAX;
    const int t = threadIdx.x, T = (int)blockDim.x;
    const int lane = t & 31, wp = t >> 5, nwarps = T >> 5;
    if ((uint64_t)seg0 + s > seg_cap || s > tmp_cap)
        return GS_NONE;
    // per-warp bin counts, then cursors, in the survivor array's memory:
    // entry i is taken by thread i mod T in both passes, so by one warp
    uint32_t *hw = reinterpret_cast<uint32_t *>(sv);          // [nwarps][32]
    if (t < 32 * nwarps)
        hw[t] = 0;
    if (t == 0)
        left_sh = 0;
    __syncthreads();
    auto bin_of = [&](uint32_t Kc) -> uint32_t { return mix32(nz ? (Kc >> 1) : Kc) >> 27; };
    for (uint32_t i0 = t; i0 - t < s; i0 += GB * (uint32_t)T) {
        uint32_t Kc[GB];
#pragma unroll
        for (int u = 0; u < GB; ++u) {
            const uint32_t i = i0 + u * (uint32_t)T;
            Kc[u] = i < s ? (uint32_t)(okeys[seg0 + i] & kcmask) : 0u;
        }
#pragma unroll
        for (int u = 0; u < GB; ++u)
            if (i0 + u * (uint32_t)T < s)
                atomicAdd(&hw[wp * 32 + bin_of(Kc[u])], 1u);
    }
    __syncthreads();
    // exclusive scan in (bin, warp) order: thread t holds bin t / nwarps of
    // warp t % nwarps (32 * nwarps == T entries, one per thread)
    {
        const uint32_t bn = (uint32_t)t / nwarps, w = (uint32_t)t % nwarps;
        const uint32_t v = hw[w * 32 + bn];
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o)
                incl += y;
        }
        if (lane == 31)
            wsum2[wp] = incl;
        __syncthreads();
        uint32_t before = 0;
        for (int i = 0; i < wp; ++i)
            before += wsum2[i];
        const uint32_t ex = before + incl - v;
        hw[w * 32 + bn] = ex;                   // every thread read its v before the barrier
        if (w == 0)
            bstart[bn] = ex;
        if (t == T - 1)
            bstart[32] = ex + v;
    }
    __syncthreads();
    // scatter to tmp
    for (uint32_t i0 = t; i0 - t < s; i0 += GB * (uint32_t)T) {
        uint32_t Kc[GB], v[GB];
#pragma unroll
        for (int u = 0; u < GB; ++u) {
            const uint32_t i = i0 + u * (uint32_t)T;
            Kc[u] = i < s ? (uint32_t)(okeys[seg0 + i] & kcmask) : 0u;
            v[u] = i < s ? ovals[seg0 + i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < GB; ++u) {
            if (i0 + u * (uint32_t)T < s) {
                const uint32_t pos = atomicAdd(&hw[wp * 32 + bin_of(Kc[u])], 1u);
                tmp[pos] = ((uint64_t)Kc[u] << 32) | v[u];
            }
        }
    }
    __syncthreads();
    // bin ranges of at most SMAX entries through sv; larger bins streamed
    uint32_t *curA = reinterpret_cast<uint32_t *>(sv);    // side-A cursors of group_stream
    for (uint32_t bn = 0; bn < 32;) {
        const uint32_t nbin = bstart[bn + 1] - bstart[bn];
        if (nbin > SMAX) {
            const uint64_t *E = tmp + bstart[bn];
            if (nbin >= 65536u || !group_stream<Lay>(E, nbin, tkey, tcnt, curA, nz, b, g)) {
                // back to the segment for the general path
                const uint32_t at = left_sh;
                for (uint32_t i = t; i < nbin; i += (uint32_t)T) {
                    const uint64_t e = E[i];
                    okeys[seg0 + at + i] = runbits | (uint64_t)(uint32_t)(e >> 32);
                    ovals[seg0 + at + i] = (uint32_t)e;
                }
                __syncthreads();
                if (t == 0)
                    left_sh = at + nbin;
                __syncthreads();
            }
            ++bn;
            continue;
        }
        uint32_t be = bn + 1;
        while (be < 32 && bstart[be + 1] - bstart[bn] <= SMAX)
            ++be;
        const uint32_t n0 = bstart[bn], cnt = bstart[be] - n0;
        for (uint32_t i0 = t; i0 - t < cnt; i0 += GB * (uint32_t)T) {     // GB loads in flight
            uint64_t e[GB];
#pragma unroll
            for (int u = 0; u < GB; ++u) {
                const uint32_t i = i0 + u * (uint32_t)T;
                e[u] = i < cnt ? tmp[n0 + i] : 0ull;
            }
#pragma unroll
            for (int u = 0; u < GB; ++u)
                if (i0 + u * (uint32_t)T < cnt)
                    sv[i0 + u * (uint32_t)T] = e[u];
        }
        __syncthreads();
        if (cnt)
            group_on_chip<Lay>(sv, cnt, tkey, tcnt, nz, b, g, occ);
        bn = be;
    }
    __syncthreads();
    return left_sh;
}

// One work item of the survivor filter -- run r of the launch group and a
// block of responses [b0, b1) -- as described at the top of the file: passes
// 1-2, refinement and the on-chip grouping, for every thread of the CTA.
// `cursor` is the CTA's fill of its global segment (shared memory, kept by
// the caller across items of the same search).
//
// MB = 0: real X through the unbiased transform (Section 3.2); the keys are
// drawn from the scaled real rows Xrs (row pitch Pf floats) instead of the
// packed bits.
//
// BATCH: B responses share X and the row stream.  The keys of a run and its
// filter F are built once; pass 2, refinement and grouping then run once per
// response b (its response key c_b), and buckets carry b in their `pad`
// field.  cnz is indexed (b << rbits) | run.
template <int MB, bool BATCH>
__device__ __forceinline__ void filter_item(const FilterArgs &a, int item, uint32_t &cursor)
{
    // the launch group's arguments under their usual names
    const uint32_t *__restrict__ Xr = a.Xr;
    const int64_t Pp = a.Pp, P = a.P;
    const uint32_t *__restrict__ ybs = a.ybs;
    const int64_t Wp = a.Wp;
    const int B = a.B;
    const int64_t n = a.n, p = a.p;
    const int M = a.M;
    const uint64_t seed = a.seed;
    const int64_t l0 = a.l0;
    const int NB = a.NB, BB = a.BB, rbits = a.rbits;
    const int64_t rbase = a.rbase;
    const uint32_t mcap = a.mcap, bcap = a.bcap;
    uint32_t *__restrict__ kc_scratch = a.kc_scratch;
    void *__restrict__ seg_keys_v = a.seg_keys_v;
    uint32_t *__restrict__ seg_vals = a.seg_vals;
    const uint32_t seg_cap = a.seg_cap;
    int *__restrict__ overflow = a.overflow;
    uint8_t *__restrict__ cnz = a.cnz;
    uint32_t *__restrict__ members = a.members;
    uint32_t *__restrict__ members_count = a.members_count;
    Bucket *__restrict__ buckets = a.buckets;
    uint64_t *__restrict__ pair_counts = a.pair_counts;
    uint32_t *__restrict__ nbuckets = a.nbuckets;
    const uint64_t *__restrict__ cdf = a.cdf;
    const uint64_t wtot = a.wtot;
    const float *__restrict__ Xrs = a.Xrs;
    const int64_t Pf = a.Pf;
    const int part_max = a.part_max;
    unsigned long long *__restrict__ kept = a.kept;
    using SegKey = uint64_t;
    extern __shared__ __align__(16) uint32_t fl_smem[];
    using Lay = FlLayout<BATCH>;
    constexpr int FL_SMAX = Lay::SMAX;
    uint32_t *F = fl_smem;                                                   // [FL_FWORDS]
    uint64_t *sv = reinterpret_cast<uint64_t *>(fl_smem + Lay::OFF_SV);      // [FL_SMAX]
    uint32_t *rf = fl_smem + Lay::OFF_SV;                                    // [FL_RWORDS]
    uint32_t *kmask = fl_smem + Lay::OFF_KM;                                 // [FL_KWORDS]
    uint32_t *tkey = fl_smem + Lay::OFF_TAB;                                 // [Lay::T]
    uint32_t *tcnt = fl_smem + Lay::OFF_TAB + Lay::T;                        // [Lay::T]
    const int t = threadIdx.x;
    const int lane = t & 31, wp = t >> 5;
    __shared__ int64_t rowoff[32];      // row s_m times the row pitch
    __shared__ int64_t rowidx[32];      // row s_m
    __shared__ uint32_t c_sh;
    __shared__ uint32_t ns;             // survivors of the current (run, response)
    __shared__ uint32_t scur;           // survivor array fill after refinement
    const int T = (int)blockDim.x;      // a multiple of 32, at most FL_THREADS
    __shared__ uint32_t seg0_sh;        // first segment entry of the current (run, response)
    const GroupOut gout{members, members_count, buckets, pair_counts, nbuckets, mcap, bcap, overflow, kept + 1};
    uint32_t *kcs = kc_scratch + (int64_t)blockIdx.x * 32 * P;
    SegKey *okeys = reinterpret_cast<SegKey *>(seg_keys_v) + (int64_t)blockIdx.x * seg_cap;
    uint32_t *ovals = seg_vals + (int64_t)blockIdx.x * seg_cap;
    const uint32_t P32 = (uint32_t)P, p32 = (uint32_t)p;
    const uint32_t steps = (P32 + T - 1) / T;
    // filter F: about 16 bits per column (2^20 at most), so the load, and
    // with it the false-positive rate, does not depend on p
    int flog = 10;
    while (flog < FL_LOGF && ((int64_t)1 << flog) < 16 * p)
        ++flog;
    const int fwords = 1 << (flog - 5);
    const int fshift = 32 - (flog - 5);
    {
        const int r = item / NB;
        const int b0 = (item - r * NB) * BB;
        const int b1 = (b0 + BB < B) ? b0 + BB : B;
        const uint64_t rl = (uint64_t)(rbase + r);   // run index within the search
        for (int i = t; i < fwords; i += T)
            F[i] = 0;
        if (wp == 0) {
            int64_t s = 0;
            if (lane < M)
                s = draw_row(seed, (uint64_t)(l0 + r) * (uint64_t)M + (uint64_t)lane, n, cdf, wtot);
            rowoff[lane] = s * Pp;
            rowidx[lane] = s;
            if (!BATCH) {
                const uint32_t ybit = lane < M ? (ybs[s >> 5] >> (s & 31)) & 1u : 0u;
                const uint32_t c = __ballot_sync(FULL, ybit);
                if (lane == 0) {
                    c_sh = c;
                    cnz[rl] = (c != 0);
                }
            }
        }
        __syncthreads();

        // pass 1: keys to the scratch rows and the filter.  Rows at or past
        // MB are zero at compile time.
        {
            const bool need = BATCH || c_sh != 0;    // c == 0 keeps every column
            for (uint32_t w = t; w < P32; w += T) {
                uint32_t A[32];
                if (MB == 0) {
                    // real X, unbiased transform (Section 3.2): bit m of column
                    // 32w + cc is 1 when draw m's random binarisation of
                    // X'[s_m, j] is -1, i.e. u24 >= (X' + 1) / 2 * 2^24 with
                    // u24 the top bits of splitmix64 output (l M + m) p + j
                    // of the transform stream
#pragma unroll
                    for (int cc = 0; cc < 32; ++cc)
                        A[cc] = 0u;
                    const uint64_t col0 = 32ULL * w;
                    const uint64_t seed2 = seed + 0x632BE59BD9B4E019ULL;
                    for (int m = 0; m < M; ++m) {
                        const float *xr = Xrs + rowidx[m] * Pf + col0;
                        const uint64_t tb = ((uint64_t)(l0 + r) * (uint64_t)M + (uint64_t)m) * (uint64_t)p + col0;
#pragma unroll
                        for (int cc = 0; cc < 32; ++cc) {
                            const float g = (__ldg(xr + cc) + 1.0f) * 0.5f;
                            const uint64_t u = mix64(seed2 + (tb + (uint64_t)cc + 1ULL) * 0x9E3779B97F4A7C15ULL);
                            A[cc] |= ((float)(uint32_t)(u >> 40) < g * 16777216.0f ? 0u : 1u) << m;
                        }
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < 32; ++m)
                        A[m] = (m < MB && m < M) ? __ldg(Xr + rowoff[m] + w) : 0u;
                    transpose32(A);
                }
#pragma unroll
                for (int cc = 0; cc < 32; ++cc)
                    kcs[cc * P32 + w] = A[cc];         // bit-major: coalesced across the warp
                if (need) {
                    const uint32_t ncol = (32 * w + 32 <= p32) ? 32u : p32 - 32 * w;
                    if (ncol == 32) {                  // every word but the last
#pragma unroll
                        for (int cc = 0; cc < 32; ++cc) {
                            uint32_t word, mask;
                            bloom_pos(A[cc], fshift, word, mask);
                            atomicOr(F + word, mask);
                        }
                    } else {
#pragma unroll
                        for (int cc = 0; cc < 32; ++cc) {
                            if ((uint32_t)cc < ncol) {
                                uint32_t word, mask;
                                bloom_pos(A[cc], fshift, word, mask);
                                atomicOr(F + word, mask);
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();

        for (int b = b0; b < b1; ++b) {
            if (BATCH) {
                if (wp == 0) {
                    const int64_t s = rowidx[lane];
                    const uint32_t *ybb = ybs + (int64_t)b * Wp;
                    const uint32_t ybit = lane < M ? (ybb[s >> 5] >> (s & 31)) & 1u : 0u;
                    const uint32_t c = __ballot_sync(FULL, ybit);
                    if (lane == 0) {
                        c_sh = c;
                        cnz[((uint64_t)b << rbits) | rl] = (c != 0);
                    }
                }
            }
            if (t == 0)
                ns = 0;
            __syncthreads();
            const uint32_t c = c_sh;
            const bool nz = c != 0;
            const int tb = nz ? 31 - __clz(c) : 0;
            const uint32_t lowmask = nz ? ((1u << tb) - 1u) : 0u;
            const SegKey runbits = (SegKey)((((uint64_t)b << rbits) | rl) << M);

            // pass 2: test every column; keep bits of column word w to
            // kmask[w], and the survivors, while they fit, to the shared array
            for (uint32_t st = 0; st < steps; ++st) {
                const uint32_t w = st * T + t;
                uint32_t keep = 0;     // bit cc: column 32w + cc survives
                if (w < P32) {
                    const uint32_t valid = (32 * w + 32 <= p32) ? 0xFFFFFFFFu
                                                                : ((1u << (p32 - 32 * w)) - 1u);
                    if (!nz) {
                        keep = valid;
                    } else {
#pragma unroll
                        for (int cc = 0; cc < 32; ++cc)
                            keep += bloom_has(F, kcs[cc * P32 + w] ^ c, fshift) << cc;
                        keep &= valid;
                    }
                    kmask[w] = keep;
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
                    wbase = atomicAdd(&ns, wtot);
                wbase = __shfl_sync(FULL, wbase, 31);
                uint32_t o = wbase + incl - cnt;
                while (keep && o < (uint32_t)FL_SMAX) {
                    // two survivors per step, so that their key re-reads overlap
                    const int c0 = __ffs(keep) - 1;
                    keep &= keep - 1;
                    const bool two = keep != 0 && o + 1 < (uint32_t)FL_SMAX;
                    const int c1 = two ? __ffs(keep) - 1 : c0;
                    if (two)
                        keep &= keep - 1;
                    const uint32_t k0 = kcs[c0 * P32 + w];   // survivors only: re-read, cache-hot
                    const uint32_t k1 = kcs[c1 * P32 + w];
                    sv[o] = ((uint64_t)canon(k0, c, tb, lowmask) << 32) | (32 * w + c0);
                    if (two)
                        sv[o + 1] = ((uint64_t)canon(k1, c, tb, lowmask) << 32) | (32 * w + c1);
                    o += two ? 2u : 1u;
                }
            }
            __syncthreads();
            uint32_t s = ns;
            const uint32_t kcmask = (1u << M) - 1u;   // M <= 31 on this path
            if (t == 0)
                atomicAdd(kept, (unsigned long long)s);

            if (s > (uint32_t)FL_SMAX) {
                // refinement: a fresh filter of the survivors' keys (in the
                // survivor array's memory) with new hashes, tested again
                for (int round = 1; nz && round <= FL_ROUNDS; ++round) {
                    __syncthreads();                   // every thread has read ns
                    for (int i = t; i < FL_RWORDS; i += T)
                        rf[i] = 0;
                    if (t == 0)
                        ns = 0;
                    __syncthreads();
                    const uint32_t salt = 0x9E3779B9u * (uint32_t)round;
                    for (uint32_t w = t; w < P32; w += T) {
                        uint32_t keep = kmask[w];
                        while (keep) {                 // two keys per step
                            const int c0 = __ffs(keep) - 1;
                            keep &= keep - 1;
                            const bool two = keep != 0;
                            const int c1 = two ? __ffs(keep) - 1 : c0;
                            if (two)
                                keep &= keep - 1;
                            const uint32_t k0 = kcs[c0 * P32 + w], k1 = kcs[c1 * P32 + w];
                            uint32_t word, mask;
                            bloom_pos(mix32(k0 ^ salt), 32 - FL_LOGR, word, mask);
                            atomicOr(rf + word, mask);
                            if (two) {
                                bloom_pos(mix32(k1 ^ salt), 32 - FL_LOGR, word, mask);
                                atomicOr(rf + word, mask);
                            }
                        }
                    }
                    __syncthreads();
                    for (uint32_t st = 0; st < steps; ++st) {
                        const uint32_t w = st * T + t;
                        uint32_t keep = w < P32 ? kmask[w] : 0u;
                        uint32_t left = keep;
                        while (left) {                 // two keys per step
                            const int c0 = __ffs(left) - 1;
                            left &= left - 1;
                            const bool two = left != 0;
                            const int c1 = two ? __ffs(left) - 1 : c0;
                            if (two)
                                left &= left - 1;
                            const uint32_t k0 = kcs[c0 * P32 + w], k1 = kcs[c1 * P32 + w];
                            uint32_t word, mask;
                            bloom_pos(mix32((k0 ^ c) ^ salt), 32 - FL_LOGR, word, mask);
                            if ((rf[word] & mask) != mask)
                                keep &= ~(1u << c0);
                            bloom_pos(mix32((k1 ^ c) ^ salt), 32 - FL_LOGR, word, mask);
                            if ((rf[word] & mask) != mask)
                                keep &= ~(1u << c1);
                        }
                        if (w < P32)
                            kmask[w] = keep;
                        const uint32_t wtot = __reduce_add_sync(FULL, (uint32_t)__popc(keep));
                        if (lane == 0 && wtot)
                            atomicAdd(&ns, wtot);
                    }
                    __syncthreads();
                    const uint32_t s_new = ns;
                    const bool done = s_new <= (uint32_t)FL_SMAX || s_new > s - s / 8;
                    s = s_new;
                    if (done)
                        break;
                }
                // emit what is left: to the survivor array when it fits, else
                // to the CTA's global segment with the composite key
                const bool to_global = s > (uint32_t)FL_SMAX;
                if (t == 0) {
                    scur = 0;
                    seg0_sh = cursor;               // this run's entries start here
                }
                __syncthreads();
                for (uint32_t st = 0; st < steps; ++st) {
                    const uint32_t w = st * T + t;
                    uint32_t keep = w < P32 ? kmask[w] : 0u;
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
                        wbase = atomicAdd(to_global ? &cursor : &scur, wtot);
                    wbase = __shfl_sync(FULL, wbase, 31);
                    uint32_t o = wbase + incl - cnt;
                    auto emit = [&](uint32_t at, uint32_t key, int cc) {
                        if (to_global) {
                            if (at < seg_cap) {
                                okeys[at] = runbits | (SegKey)key;
                                ovals[at] = 32 * w + cc;
                            }
                        } else if (at < (uint32_t)FL_SMAX) {
                            sv[at] = ((uint64_t)key << 32) | (32 * w + cc);
                        }
                    };
                    while (keep) {                     // two survivors per step
                        const int c0 = __ffs(keep) - 1;
                        keep &= keep - 1;
                        const bool two = keep != 0;
                        const int c1 = two ? __ffs(keep) - 1 : c0;
                        if (two)
                            keep &= keep - 1;
                        const uint32_t k0 = kcs[c0 * P32 + w], k1 = kcs[c1 * P32 + w];
                        emit(o, canon(k0, c, tb, lowmask), c0);
                        if (two)
                            emit(o + 1, canon(k1, c, tb, lowmask), c1);
                        o += two ? 2u : 1u;
                    }
                }
                __syncthreads();
                if (to_global) {
                    // the run's entries are in the segment: grouped on chip in
                    // partitions when they fit, else left to the general path
                    if (group_from_segment<Lay>(okeys, ovals, seg0_sh, s, seg_cap, part_max, kcmask, sv, tkey,
                                                tcnt, nz, b, gout) &&
                        t == 0) {
                        cursor = seg0_sh;           // grouped on chip: the entries leave the segment
                        atomicAdd(kept + 2, 1ull);  // one more run grouped from the segment
                    }
                    continue;
                }
            }
            group_on_chip<Lay>(sv, s, tkey, tcnt, nz, b, gout);
        }
    }
}

// One CTA per run at a time: the work items of one launch group of one
// search, taken from a launch-wide counter, so a CTA that drew an expensive
// run takes fewer.  When a run keeps at most SMAX columns they are grouped
// on chip (a hash table of group keys with packed side counts; each group
// with candidates becomes a bucket, its members written side A first); a
// run that keeps more, after refinement, goes to the CTA's global segment
// and is grouped from there in hash partitions, or left for the general
// sort and join.  Spilled survivors carry ((b << rbits | run) << M) | Kc in
// 64-bit keys, run counted from the start of the search, and the per-CTA
// segments fill across launch groups until the host sorts them.
// kc_scratch holds, per CTA, the keys of its current run in bit-major order:
// kx of column 32w + cc at cc * P + w.
template <int MB, bool BATCH>
__global__ void __launch_bounds__(FL_THREADS, 1) filter_kernel(const __grid_constant__ FilterArgs a,
                                                               uint32_t *__restrict__ work)
{
    __shared__ uint32_t cursor;         // global segment fill
    __shared__ int item_sh;
    if (threadIdx.x == 0)
        cursor = a.seg_count[blockIdx.x];     // segments fill across launch groups
    for (;;) {
        if (threadIdx.x == 0)
            item_sh = (int)atomicAdd(work, 1u);
        __syncthreads();
        const int item = item_sh;           // every thread reads it before the next barrier
        if (item >= a.R * a.NB)
            break;
        filter_item<MB, BATCH>(a, item, cursor);
    }
    if (threadIdx.x == 0) {
        a.seg_count[blockIdx.x] = cursor < a.seg_cap ? cursor : a.seg_cap;
        if (cursor > a.seg_cap)
            atomicOr(a.overflow, 1);
    }
}

// The arguments of the searches of one fused launch, and the first global
// work item of each (item_start[count] = all items).
struct FusedTable {
    int count;
    int item_start[XYZ_FUSED_MAX + 1];
    FilterArgs args[XYZ_FUSED_MAX];
};
static_assert(sizeof(FusedTable) <= 32764, "the fused table fits the kernel parameter space");

// Several independent searches (one launch group each, one response, binary
// or weighted Y, the single filter) in one persistent launch: the work items
// of all of them are taken from one launch-wide counter, in search order, so
// the CTAs move on to the next search's runs as soon as the current one's
// are handed out.  Each search keeps its own buffers; a CTA's segment fill
// of a search is loaded when it takes that search's first item and stored
// when it moves on.
template <int MB>
__global__ void __launch_bounds__(FL_THREADS, 1) filter_fused_kernel(const __grid_constant__ FusedTable tab,
                                                                     uint32_t *__restrict__ work)
{
    __shared__ uint32_t cursor;
    __shared__ int item_sh, inst_sh;
    if (threadIdx.x == 0)
        inst_sh = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const int item = (int)atomicAdd(work, 1u);
            item_sh = item;
            if (item < tab.item_start[tab.count]) {
                int i = inst_sh < 0 ? 0 : inst_sh;
                while (tab.item_start[i + 1] <= item)
                    ++i;
                if (i != inst_sh) {
                    if (inst_sh >= 0) {
                        const FilterArgs &o = tab.args[inst_sh];
                        o.seg_count[blockIdx.x] = cursor < o.seg_cap ? cursor : o.seg_cap;
                        if (cursor > o.seg_cap)
                            atomicOr(o.overflow, 1);
                    }
                    cursor = tab.args[i].seg_count[blockIdx.x];
                    inst_sh = i;
                }
            }
        }
        __syncthreads();
        const int item = item_sh;
        if (item >= tab.item_start[tab.count])
            break;
        const int i = inst_sh;
        filter_item<MB, false>(tab.args[i], item - tab.item_start[i], cursor);
    }
    if (threadIdx.x == 0 && inst_sh >= 0) {
        const FilterArgs &o = tab.args[inst_sh];
        o.seg_count[blockIdx.x] = cursor < o.seg_cap ? cursor : o.seg_cap;
        if (cursor > o.seg_cap)
            atomicOr(o.overflow, 1);
    }
}

// Class of a key: bit b is the parity of the key bits m with m % 4 == b.
// The map is linear over GF(2), so class(k ^ c) = class(k) ^ class(c).
__device__ __forceinline__ uint32_t key_class(uint32_t k)
{
    uint32_t q = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
        q |= (uint32_t)(__popc(k & (0x11111111u << b)) & 1) << b;
    return q;
}

// The survivor filter for p too large for one shared-memory filter of all
// its keys (the same decisions as filter_kernel, for one response and
// M <= 28).  The keys of a run are split into 16 classes by key_class:
//
//   pass 1  build the keys (the transpose also carries the four class
//           parities, formed from the sampled row words in rows 28-31) and
//           write each to its class list, a tile of T words (32 T columns)
//           at a time, in two halves of 16 columns per word: each thread
//           counts its columns per class (a popcount of the class mask of
//           its word), one scan over the CTA's 16 x T counts gives every
//           thread its staging position per class, the keys and columns
//           are scattered into shared memory in class order, and each
//           class's part of the half-tile is copied to the end of its class
//           list with consecutive threads on consecutive entries;
//   rounds  for each class q: a fresh filter F of the class-q keys, tested
//           by the keys k of class q ^ class(c) -- exactly those with
//           k ^ c in class q, so every key k ^ c is looked up in the filter
//           that holds its class; survivors go to the CTA's segment as
//           (runbits | Kc, column).  A run with c == 0 keeps the keys
//           that occur at least twice (two filters per class).
//
// Each round's filter holds about p/16 keys, which keeps its load, and with
// it the false-positive rate, near that of filter_kernel at p/16 columns.
// The survivors of the run are then grouped on chip from the segment (hash
// partitions), or left there for the general sort when a partition bin is
// above the chip's capacity.  A class list that overflows sets overflow
// bit 4 (the host enlarges the lists and redoes the search).
template <int MB>
__global__ void __launch_bounds__(FL_THREADS, 1)
    filter_big_kernel(const uint32_t *__restrict__ Xr, int64_t Pp, int64_t P, const uint32_t *__restrict__ yb,
                      int64_t n, int64_t p, int M, uint64_t seed, int64_t l0, int R, int rbits, int64_t rbase,
                      uint32_t mcap, uint32_t bcap, uint32_t *__restrict__ lst_keys,
                      uint32_t *__restrict__ lst_cols, uint32_t lcap, void *__restrict__ seg_keys_v,
                      uint32_t *__restrict__ seg_vals, uint32_t *__restrict__ seg_count, uint32_t seg_cap,
                      int *__restrict__ overflow, uint8_t *__restrict__ cnz, uint32_t *__restrict__ members,
                      uint32_t *__restrict__ members_count, Bucket *__restrict__ buckets,
                      uint64_t *__restrict__ pair_counts, uint32_t *__restrict__ nbuckets,
                      const uint64_t *__restrict__ cdf, uint64_t wtot, int part_max, uint32_t *__restrict__ work,
                      unsigned long long *__restrict__ kept)
{
    using Lay = FlLayout<false>;
    // pass 1 staging, in the memory of the filter and survivor array (dead
    // until the rounds): one half-tile's entries (column << 32 | key, 16 T
    // of them) in class order, and the per-thread class cursors, which hold
    // the cursors of both half-tiles (low and high 16 bits).  Cursor (q, t)
    // sits at q Tp + t + 4 (t / 32), with the class stride Tp >= T + T/8 a
    // multiple of 32: the scan's 16-entry chunks and the scatter's cursor
    // accesses are then free of bank conflicts.
    constexpr int FB_STAGE = 16 * FL_THREADS;      // entries of a half-tile, 8 bytes each
    constexpr int FB_CUR = 2 * FB_STAGE;
    constexpr int FB_V = 2;                        // 16-byte list words per thread and step in the rounds
    constexpr int FB_EB = 8;                       // list entries emitted together
    constexpr int FB_EMIT = FL_FWORDS;            // rounds: per-warp buffers of passing entries
    static_assert(FB_EMIT + (FL_THREADS / 32) * FB_EB * 32 * 2 <= Lay::WORDS, "emission buffers fit");
    static_assert((4 * FB_V) % FB_EB == 0, "whole emission groups per step");
    static_assert(FB_CUR + 16 * (FL_THREADS + FL_THREADS / 8) <= Lay::WORDS,
                  "staging and cursors fit the shared memory");
    static_assert(FB_STAGE < 65536, "a half-tile's positions fit 16 bits");
    extern __shared__ __align__(16) uint32_t fl_smem[];
    uint32_t *F = fl_smem;                                                   // [FL_FWORDS], in the rounds
    uint64_t *sv = reinterpret_cast<uint64_t *>(fl_smem + Lay::OFF_SV);      // [SMAX], after the rounds
    uint32_t *occ = fl_smem + Lay::OFF_KM;                                   // [SMAX] occupied slots, grouping
    static_assert(FL_KWORDS >= Lay::SMAX, "the occupied-slot list fits its region");
    uint32_t *tkey = fl_smem + Lay::OFF_TAB;                                 // [Lay::T], after the rounds
    uint32_t *tcnt = fl_smem + Lay::OFF_TAB + Lay::T;
    uint64_t *stg = reinterpret_cast<uint64_t *>(fl_smem);                   // [16 T] staged entries
    uint32_t *cur = fl_smem + FB_CUR;                                        // [16][T + T/8] cursors
    const int t = threadIdx.x;
    const int lane = t & 31, wp = t >> 5;
    const int T = (int)blockDim.x;                 // a multiple of 32, at most FL_THREADS
    const int nwarps = T >> 5;
    const int Tp = (T + T / 8 + 31) / 32 * 32;     // class stride of the cursors (a multiple of 32 words)
    const int tt = t + 4 * wp;                     // padded place of thread t in a class
    __shared__ int64_t rowoff[32];
    __shared__ uint32_t c_sh, cursor, seg0_sh;
    __shared__ uint32_t cls_n[16];                 // fill of each class list
    __shared__ uint32_t cbase[17];                 // staging start of each class, both halves; [16]: totals
    __shared__ int64_t dstoff[16];                 // list index of staged entry i of class q: dstoff[q] + i
    __shared__ uint32_t wsum[FL_THREADS / 32];
    __shared__ int item_sh, lovf_sh;
    const GroupOut gout{members, members_count, buckets, pair_counts, nbuckets, mcap, bcap, overflow, kept + 1};
    const uint32_t P32 = (uint32_t)P, p32 = (uint32_t)p;
    const int fshift = 32 - (FL_LOGF - 5);
    const uint32_t kcmask = (1u << M) - 1u;                                  // M <= 28
    uint32_t *lk = lst_keys + (int64_t)blockIdx.x * 16 * lcap;               // [16][lcap]
    uint32_t *lc = lst_cols + (int64_t)blockIdx.x * 16 * lcap;
    uint64_t *okeys = reinterpret_cast<uint64_t *>(seg_keys_v) + (int64_t)blockIdx.x * seg_cap;
    uint32_t *ovals = seg_vals + (int64_t)blockIdx.x * seg_cap;
    if (t == 0)
        cursor = seg_count[blockIdx.x];     // segments fill across launch groups

    for (;;) {
        if (t == 0)
            item_sh = (int)atomicAdd(work, 1u);
        __syncthreads();
        const int r = item_sh;
        if (r >= R)
            break;
        const uint64_t rl = (uint64_t)(rbase + r);
        if (wp == 0) {
            int64_t srow = 0;
            if (lane < M)
                srow = draw_row(seed, (uint64_t)(l0 + r) * (uint64_t)M + (uint64_t)lane, n, cdf, wtot);
            rowoff[lane] = srow * Pp;
            const uint32_t ybit = lane < M ? (yb[srow >> 5] >> (srow & 31)) & 1u : 0u;
            const uint32_t c = __ballot_sync(FULL, ybit);
            if (lane == 0) {
                c_sh = c;
                cnz[rl] = (c != 0);
                lovf_sh = 0;
                seg0_sh = cursor;
            }
        }
        if (t < 16)
            cls_n[t] = 0;
        __syncthreads();
        const uint32_t c = c_sh;
        const bool nz = c != 0;

        // pass 1: keys with their classes, sorted into the class lists one
        // tile of T words at a time.  The sampled row words of the next
        // tile are loaded while the current tile's last half is copied out.
        uint32_t A[32];
#pragma unroll
        for (int m = 0; m < 32; ++m)
            A[m] = (t < (int)P32 && m < MB && m < M) ? __ldg(Xr + rowoff[m] + t) : 0u;
        for (uint32_t tile0 = 0; tile0 < P32; tile0 += (uint32_t)T) {
            const uint32_t w = tile0 + t;
            uint32_t Q[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int m = 0; m < MB && m < 28; ++m)
                Q[m & 3] ^= A[m];                // rows past M are zero
#pragma unroll
            for (int b = 0; b < 4; ++b)
                A[28 + b] = Q[b];
            transpose32(A);
            const uint32_t ncol = w >= P32 ? 0u : (32 * w + 32 <= p32) ? 32u : p32 - 32 * w;
            const uint32_t vm = ncol == 32 ? FULL : ((1u << ncol) - 1u);
            {
                // class masks of the word: bit cc of lo[q & 3] & hi[q >> 2]
                // is set when column cc is of class q (bits 0-1 of q from
                // Q[0..1], bits 2-3 from Q[2..3]); counts of both halves,
                // the second in the high 16 bits
                const uint32_t lo[4] = {~Q[0] & ~Q[1] & vm, Q[0] & ~Q[1] & vm, ~Q[0] & Q[1] & vm, Q[0] & Q[1] & vm};
                const uint32_t hi[4] = {~Q[2] & ~Q[3], Q[2] & ~Q[3], ~Q[2] & Q[3], Q[2] & Q[3]};
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const uint32_t mq = lo[q & 3] & hi[q >> 2];
                    cur[q * Tp + tt] = __popc(mq & 0xFFFFu) | ((uint32_t)__popc(mq >> 16) << 16);
                }
            }
            __syncthreads();
            // exclusive scan of the counts in class-major order: thread t
            // takes the chunk of the 16 consecutive counts 16t..16t+15 (one
            // class, since 16 divides T); both halves at once, since no
            // half's sum reaches 2^16
            const int cq0 = (16 * t) / T, ct0 = 16 * t - cq0 * T;     // chunk: class cq0, threads ct0..ct0+15
            uint4 *chunk = reinterpret_cast<uint4 *>(cur + cq0 * Tp + ct0 + 4 * (ct0 >> 5));
            uint32_t csum = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint4 x = chunk[i];
                csum += x.x + x.y + x.z + x.w;
            }
            uint32_t incl = csum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o)
                    incl += y;
            }
            if (lane == 31)
                wsum[wp] = incl;
            __syncthreads();
            if (wp == 0) {
                const uint32_t x = lane < nwarps ? wsum[lane] : 0u;
                uint32_t wi = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(FULL, wi, o);
                    if (lane >= o)
                        wi += y;
                }
                if (lane < nwarps)
                    wsum[lane] = wi - x;     // exclusive over warps
                if (lane == 31)
                    cbase[16] = wi;          // entries of each half
            }
            __syncthreads();
            {
                const uint32_t off = wsum[wp] + incl - csum;
                if (ct0 == 0)
                    cbase[cq0] = off;             // the chunk starts its class
                uint32_t run = off;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    uint4 x = chunk[i];
                    const uint32_t a = run, b = a + x.x, c2 = b + x.y, d = c2 + x.z;
                    run = d + x.w;
                    chunk[i] = make_uint4(a, b, c2, d);
                }
            }
            __syncthreads();
            const uint32_t col0 = 32 * w;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                // scatter this half in class order (cursor field h)
                const uint32_t hm = vm & (h ? 0xFFFF0000u : 0x0000FFFFu);
                const uint32_t inc = h ? 0x10000u : 1u;
                const bool full = hm == (h ? 0xFFFF0000u : 0x0000FFFFu);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int cc = 16 * h + i;
                    if (full || ((hm >> cc) & 1u)) {
                        uint32_t *cq = cur + (A[cc] >> 28) * Tp + tt;
                        const uint32_t cv = *cq;
                        *cq = cv + inc;
                        stg[h ? (cv >> 16) : (cv & 0xFFFFu)] = ((uint64_t)(col0 + cc) << 32) | (A[cc] & kcmask);
                    }
                }
                if (t < 16) {
                    // list space for each class part of this half
                    const uint32_t b0 = h ? (cbase[t] >> 16) : (cbase[t] & 0xFFFFu);
                    const uint32_t b1 = h ? (cbase[t + 1] >> 16) : (cbase[t + 1] & 0xFFFFu);
                    const uint32_t g = cls_n[t];
                    dstoff[t] = (int64_t)t * lcap + g - b0;
                    if ((uint64_t)g + (b1 - b0) > lcap)
                        lovf_sh = 1;
                    else
                        cls_n[t] = g + (b1 - b0);
                }
                if (h == 1) {
                    // the sampled row words of the next tile, in flight
                    // during the copy-out
                    const uint32_t wn = w + (uint32_t)T;
#pragma unroll
                    for (int m = 0; m < 32; ++m)
                        A[m] = (wn < P32 && m < MB && m < M) ? __ldg(Xr + rowoff[m] + wn) : 0u;
                }
                __syncthreads();
                if (!lovf_sh) {
                    // to the class lists, consecutive threads on consecutive
                    // entries; a thread's entries are in increasing class
                    const uint32_t tot = h ? (cbase[16] >> 16) : (cbase[16] & 0xFFFFu);
                    uint32_t q = 0;
                    uint32_t nxt = h ? (cbase[1] >> 16) : (cbase[1] & 0xFFFFu);
                    for (uint32_t i = t; i < tot; i += (uint32_t)T) {
                        while (i >= nxt) {           // q <= 15: i < the total
                            ++q;
                            nxt = h ? (cbase[q + 1] >> 16) : (cbase[q + 1] & 0xFFFFu);
                        }
                        const uint64_t e = stg[i];
                        const int64_t g = dstoff[q] + i;
                        lk[g] = (uint32_t)e;
                        lc[g] = (uint32_t)(e >> 32);
                    }
                }
                __syncthreads();                 // the staging is reused by the next half
            }
        }
        __syncthreads();
        if (lovf_sh) {
            if (t == 0)
                atomicOr(overflow, 4);       // the host enlarges the class lists and redoes the search
            continue;
        }
        const int tb = nz ? 31 - __clz(c) : 0;
        const uint32_t lowmask = nz ? ((1u << tb) - 1u) : 0u;
        const uint64_t runbits = rl << M;

        // entries of class q2 that pass (all of them when c == 0) to the
        // segment with their columns.  The whole CTA walks the class list in
        // 16-byte words (four keys, and the same word of the columns), each
        // thread FB_V words at a time (independent loads in flight; the
        // list's memory runs to a multiple of 16 bytes, and keys past its
        // fill are masked).  A warp gathers its passing entries (column,
        // key) in its shared buffer and writes them to the segment with
        // consecutive lanes, after one reservation.
        uint64_t *wbuf = reinterpret_cast<uint64_t *>(fl_smem + FB_EMIT) + wp * (FB_EB * 32);
        auto emit_class = [&](uint32_t q2, const uint32_t *Ft, int fs) {
            const uint32_t n2 = cls_n[q2] < lcap ? cls_n[q2] : lcap;
            const uint32_t n4 = (n2 + 3) >> 2;
            const uint4 *lkq = reinterpret_cast<const uint4 *>(lk + (int64_t)q2 * lcap);
            const uint4 *lcq = reinterpret_cast<const uint4 *>(lc + (int64_t)q2 * lcap);
            for (uint32_t j0 = t; j0 - t < n4; j0 += FB_V * (uint32_t)T) {
                uint32_t k[4 * FB_V], cl[4 * FB_V];
#pragma unroll
                for (int u = 0; u < FB_V; ++u) {
                    const uint32_t j = j0 + u * (uint32_t)T;
                    const uint4 v = j < n4 ? __ldcg(lkq + j) : make_uint4(0u, 0u, 0u, 0u);
                    const uint4 w = j < n4 ? __ldcg(lcq + j) : make_uint4(0u, 0u, 0u, 0u);
                    k[4 * u] = v.x;
                    k[4 * u + 1] = v.y;
                    k[4 * u + 2] = v.z;
                    k[4 * u + 3] = v.w;
                    cl[4 * u] = w.x;
                    cl[4 * u + 1] = w.y;
                    cl[4 * u + 2] = w.z;
                    cl[4 * u + 3] = w.w;
                }
                uint32_t pm = 0;           // bit 4u + x: key x of word j0 + u T passes
#pragma unroll
                for (int e = 0; e < 4 * FB_V; ++e) {
                    const uint32_t i = 4 * (j0 + (e >> 2) * (uint32_t)T) + (e & 3);
                    if (i < n2 && bloom_has3(Ft, k[e] ^ c, fs))
                        pm |= 1u << e;
                }
#pragma unroll
                for (int e0 = 0; e0 < 4 * FB_V; e0 += FB_EB) {
                    const uint32_t pe = (pm >> e0) & ((1u << FB_EB) - 1u);
                    const uint32_t cnt = __popc(pe);
                    uint32_t incl = cnt;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(FULL, incl, o);
                        if (lane >= o)
                            incl += y;
                    }
                    const uint32_t wt = __shfl_sync(FULL, incl, 31);
                    if (wt == 0)
                        continue;
                    uint32_t o = incl - cnt;
#pragma unroll
                    for (int u = 0; u < FB_EB; ++u) {
                        const int e = e0 + u;
                        if ((pe >> u) & 1u)
                            wbuf[o++] = ((uint64_t)cl[e] << 32) | k[e];
                    }
                    uint32_t base = 0;
                    if (lane == 0)
                        base = atomicAdd(&cursor, wt);
                    base = __shfl_sync(FULL, base, 0);
                    __syncwarp();
                    for (uint32_t e = lane; e < wt; e += 32) {
                        const uint64_t v = wbuf[e];
                        const uint32_t at = base + e;
                        if (at < seg_cap) {
                            okeys[at] = runbits | canon((uint32_t)v, c, tb, lowmask);
                            ovals[at] = (uint32_t)(v >> 32);
                        }
                    }
                    __syncwarp();
                }
            }
        };
        // keys of class q into the round's filter(s), FB_V 16-byte words per
        // thread and step; ins(key) does the insert
        auto insert_class = [&](uint32_t q, auto ins) {
            const uint32_t nq = cls_n[q] < lcap ? cls_n[q] : lcap;
            const uint32_t n4 = (nq + 3) >> 2;
            const uint4 *lkq = reinterpret_cast<const uint4 *>(lk + (int64_t)q * lcap);
            for (uint32_t j0 = t; j0 - t < n4; j0 += FB_V * (uint32_t)T) {
                uint4 v[FB_V];
#pragma unroll
                for (int u = 0; u < FB_V; ++u) {
                    const uint32_t j = j0 + u * (uint32_t)T;
                    v[u] = j < n4 ? __ldcg(lkq + j) : make_uint4(0u, 0u, 0u, 0u);
                }
#pragma unroll
                for (int u = 0; u < FB_V; ++u) {
                    const uint32_t i = 4 * (j0 + u * (uint32_t)T);
                    if (i < nq)
                        ins(v[u].x);
                    if (i + 1 < nq)
                        ins(v[u].y);
                    if (i + 2 < nq)
                        ins(v[u].z);
                    if (i + 3 < nq)
                        ins(v[u].w);
                }
            }
        };
        if (!nz) {
            // c == 0: a column pairs only with an equal key, so only keys
            // that occur at least twice can be in a candidate.  Per class a
            // filter of the keys seen once (F1) and one of the keys seen
            // again (F2): an insert that finds all its bits already set in F1
            // sets them in F2, and the class's keys are tested against F2.
            // No false negatives: the inserts of two equal keys touch the same
            // word with the same mask, the atomics order them, and the later
            // sees the earlier's bits.
            uint32_t *F1 = F, *F2 = F + FL_FWORDS / 2;
            const int fs2 = fshift + 1;                 // half the words each
            for (uint32_t q = 0; q < 16; ++q) {
                for (int i = t; i < FL_FWORDS / 4; i += T)
                    reinterpret_cast<uint4 *>(F)[i] = make_uint4(0u, 0u, 0u, 0u);
                __syncthreads();
                insert_class(q, [&](uint32_t key) {
                    uint32_t word, mask;
                    bloom_pos3(key, fs2, word, mask);
                    if ((atomicOr(F1 + word, mask) & mask) == mask)
                        atomicOr(F2 + word, mask);
                });
                __syncthreads();
                emit_class(q, F2, fs2);
                __syncthreads();
            }
        } else {
            const uint32_t cq = key_class(c);
            for (uint32_t q = 0; q < 16; ++q) {
                for (int i = t; i < FL_FWORDS / 4; i += T)
                    reinterpret_cast<uint4 *>(F)[i] = make_uint4(0u, 0u, 0u, 0u);
                __syncthreads();
                insert_class(q, [&](uint32_t key) {
                    uint32_t word, mask;
                    bloom_pos3(key, fshift, word, mask);
                    atomicOr(F + word, mask);
                });
                __syncthreads();
                emit_class(q ^ cq, F, fshift);
                __syncthreads();
            }
        }
        __syncthreads();
        const uint32_t seg0 = seg0_sh, s = cursor - seg0;
        if (t == 0)
            atomicAdd(kept, (unsigned long long)s);
        __syncthreads();                     // every thread has read the cursor
        // the keys list is dead after the rounds: the run's entries are
        // sorted by bin there
        uint32_t left = part_max > 0
            ? group_segment_sorted<Lay>(okeys, ovals, seg0, s, seg_cap, kcmask, runbits, sv, tkey, tcnt, nz, 0,
                                        gout, reinterpret_cast<uint64_t *>(lk), 8 * lcap, occ)
            : GS_NONE;
        if (left == GS_NONE)
            left = s;
        else if (t == 0 && s > (uint32_t)Lay::SMAX)
            atomicAdd(kept + 2, 1ull);       // one more run grouped from the segment in several passes
        __syncthreads();
        if (t == 0)
            cursor = seg0 + left;            // what the chip could not group stays for the general path
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

size_t filter_smem_bytes(bool batch)
{
    return (size_t)(batch ? FlLayout<true>::WORDS : FlLayout<false>::WORDS) * 4;
}

int64_t filter_run_cap() { return FlLayout<false>::SMAX; }

// Threads per filter CTA: the passes give each thread whole 32-column words,
// so a multiple of 32 between 640 and 1024 that wastes the fewest thread
// slots in the last round over the P words (the largest among near ties).
int filter_threads(int64_t P)
{
    int best = FL_THREADS;
    double best_eff = 0.0;
    for (int T = FL_THREADS; T >= 640; T -= 32) {
        const int64_t rounds = (P + T - 1) / T;
        const double eff = (double)P / (double)(rounds * T);
        if (eff > best_eff + 0.01) {
            best_eff = eff;
            best = T;
        }
    }
    return best;
}

int filter_grid()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 152;
}

size_t filter_scratch_words(int64_t p) { return (size_t)filter_grid() * 32 * (size_t)((p + 31) / 32); }

bool filter_big_supported(int64_t p, int M) { return M >= 1 && M <= 28 && p >= 2 && p <= ((int64_t)1 << 27); }

uint32_t filter_big_lcap(int64_t p)
{
    // a class list holds p / 16 keys on average, but skewed data fill some
    // classes far more: columns of low minor frequency share a few keys with
    // few bits set, whose classes are the few of even parities (every
    // all-zero key is in class 0).  Room for p / 4 first, plus some slack
    // for small p.
    const int64_t l = (p + 3) / 4 + 512;
    return (uint32_t)((l + 15) / 16 * 16);
}

uint32_t filter_big_lcap_max(int64_t p)
{
    // every key of a run in one class
    return (uint32_t)((p + 512 + 15) / 16 * 16);
}

size_t filter_big_list_words(int64_t p, uint32_t lcap)
{
    (void)p;
    return (size_t)filter_grid() * 16 * (size_t)lcap;
}

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
                          int64_t *launches, int part_max, uint32_t *work, unsigned long long *kept,
                          FilterArgs *defer)
{
    FilterArgs a;
    a.Xr = pk.Xr;
    a.Pp = pk.Pp;
    a.P = pk.P;
    a.ybs = ybs;
    a.Wp = pk.Wp;
    a.B = B;
    a.n = pk.n;
    a.p = pk.p;
    a.M = M;
    a.seed = seed;
    a.l0 = l0;
    a.R = R;
    a.NB = NB;
    a.BB = BB;
    a.rbits = rbits;
    a.rbase = rbase;
    a.mcap = mcap;
    a.bcap = bcap;
    a.kc_scratch = kc_scratch;
    a.seg_keys_v = seg_keys;
    a.seg_vals = seg_vals;
    a.seg_count = seg_count;
    a.seg_cap = seg_cap;
    a.overflow = overflow;
    a.cnz = cnz;
    a.members = members;
    a.members_count = members_count;
    a.buckets = buckets;
    a.pair_counts = pair_counts;
    a.nbuckets = nbuckets;
    a.cdf = pk.cdf;
    a.wtot = pk.wtotal;
    a.Xrs = pk.Xrs;
    a.Pf = pk.Pf;
    a.part_max = part_max;
    a.kept = kept;
    if (defer) {
        *defer = a;
        return cudaSuccess;
    }
    const bool batch = B > 1;
    const size_t smem = filter_smem_bytes(batch);
    using KernT = void (*)(const FilterArgs, uint32_t *);
    KernT kern;
    if (batch)
        kern = M <= 8 ? filter_kernel<8, true> : M <= 16 ? filter_kernel<16, true>
               : M <= 24 ? filter_kernel<24, true> : filter_kernel<32, true>;
    else if (pk.Xrs)
        kern = filter_kernel<0, false>;        // real X, unbiased transform
    else
        kern = M <= 8 ? filter_kernel<8, false> : M <= 16 ? filter_kernel<16, false>
               : M <= 24 ? filter_kernel<24, false> : filter_kernel<32, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    kern<<<grid, pk.filter_threads > 0 ? pk.filter_threads : filter_threads(pk.P), smem, s>>>(a, work);
    *launches += 1;
    return cudaGetLastError();
}

int fused_key_class(int M)
{
    return M <= 16 ? 16 : M <= 24 ? 24 : 32;
}

cudaError_t launch_filter_fused(const FilterArgs *args, int count, int key_class, int grid, uint32_t *work,
                                cudaStream_t s, int64_t *launches)
{
    if (count < 1 || count > XYZ_FUSED_MAX)
        return cudaErrorInvalidValue;
    FusedTable tab;
    std::memset(&tab, 0, sizeof(tab));
    tab.count = count;
    tab.item_start[0] = 0;
    for (int i = 0; i < count; ++i) {
        if (args[i].B != 1 || args[i].Xrs || fused_key_class(args[i].M) != key_class)
            return cudaErrorInvalidValue;
        tab.args[i] = args[i];
        tab.item_start[i + 1] = tab.item_start[i] + args[i].R * args[i].NB;
    }
    using KernT = void (*)(const FusedTable, uint32_t *);
    const KernT kern = key_class == 16 ? filter_fused_kernel<16>
                       : key_class == 24 ? filter_fused_kernel<24> : filter_fused_kernel<32>;
    const size_t smem = filter_smem_bytes(false);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    kern<<<grid, FL_THREADS, smem, s>>>(tab, work);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_filter_big(const Packed &pk, int M, uint64_t seed, int64_t l0, int R, int rbits, int64_t rbase,
                              int grid, uint32_t mcap, uint32_t bcap, uint32_t *lst_keys, uint32_t *lst_cols,
                              uint32_t lcap, uint64_t *seg_keys, uint32_t *seg_vals, uint32_t *seg_count,
                              uint32_t seg_cap, int *overflow, uint8_t *cnz, uint32_t *members,
                              uint32_t *members_count, Bucket *buckets, uint64_t *pair_counts, uint32_t *nbuckets,
                              cudaStream_t s, int64_t *launches, int part_max, uint32_t *work,
                              unsigned long long *kept)
{
    const size_t smem = filter_smem_bytes(false);
    using KernT = void (*)(const uint32_t *, int64_t, int64_t, const uint32_t *, int64_t, int64_t, int, uint64_t,
                           int64_t, int, int, int64_t, uint32_t, uint32_t, uint32_t *, uint32_t *, uint32_t, void *,
                           uint32_t *, uint32_t *, uint32_t, int *, uint8_t *, uint32_t *, uint32_t *, Bucket *,
                           uint64_t *, uint32_t *, const uint64_t *, uint64_t, int, uint32_t *,
                           unsigned long long *);
    const KernT kern = M <= 8 ? filter_big_kernel<8> : M <= 16 ? filter_big_kernel<16>
                       : M <= 24 ? filter_big_kernel<24> : filter_big_kernel<32>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    kern<<<grid, pk.filter_threads > 0 ? pk.filter_threads : filter_threads(pk.P), smem, s>>>(pk.Xr, pk.Pp, pk.P, pk.yb, pk.n, pk.p, M, seed, l0, R, rbits, rbase,
                                                  mcap, bcap, lst_keys, lst_cols, lcap, seg_keys, seg_vals, seg_count,
                                                  seg_cap, overflow, cnz, members, members_count, buckets,
                                                  pair_counts, nbuckets, pk.cdf, pk.wtotal, part_max, work, kept);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace xyz
