// Per-run survivor filter for the equal-pairs search (Algorithm 2 steps
// 3-4): filter_kernel for M <= 31 when p is small enough for one
// shared-memory filter of a run's keys, filter_big_kernel (further down)
// for larger p with the keys split into 16 linear classes.
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
};

// Groups the s <= SMAX survivors (Kc << 32 | j) in sv on chip: a hash table
// of group keys with packed side counts (tkey / tcnt); each group with
// candidates becomes a bucket (response b in its pad) and its members are
// written side A first.  Called by every thread of the CTA.
template <class Lay>
__device__ __forceinline__ void group_on_chip(uint64_t *sv, uint32_t s, uint32_t *tkey, uint32_t *tcnt, bool nz,
                                              int b, const GroupOut &g)
{
    __shared__ uint32_t mbase_sh, bbase_sh;
    __shared__ uint32_t wsum[FL_THREADS / 32];
    const int t = threadIdx.x, T = (int)blockDim.x;
    const int lane = t & 31, wp = t >> 5, nwarps = T >> 5;
    uint32_t *members = g.members;
    Bucket *buckets = g.buckets;
    uint64_t *pair_counts = g.pair_counts;
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
    __syncthreads();
    // phase I: insert group keys, count sides (A high half, B low
    // half); keep (side, slot, j)
    for (uint32_t i = t; i < s; i += T) {
        const uint64_t e = sv[i];
        const uint32_t Kc = (uint32_t)(e >> 32);
        const uint32_t g = nz ? (Kc >> 1) : Kc;
        const uint32_t side = nz ? (Kc & 1u) : 0u;
        uint32_t slot = (g * 0x9E3779B1u) >> (32 - tlog);
        for (int probe = 0; probe < tsize; ++probe) {    // s < tsize: always ends
            const uint32_t old = atomicCAS(&tkey[slot], FL_EMPTY, g);
            if (old == FL_EMPTY || old == g)
                break;
            slot = (slot + 1) & (tsize - 1);
        }
        atomicAdd(&tcnt[slot], side ? 1u : 0x10000u);
        sv[i] = ((uint64_t)((side << 31) | slot) << 32) | (uint32_t)e;
    }
    __syncthreads();
    // phase II: groups with candidates -> buckets; one global atomic
    // pair per (run, response) reserves their space.  Afterwards
    // tkey / tcnt of a bucket's slot are the end cursors of its sides
    // A / B, and tcnt is FL_EMPTY for a slot without a bucket.
    {
        // each thread owns a contiguous range of slots; the value of
        // a slot is members << 16 | 1 when its group yields a bucket
        const int per = (tsize + T - 1) / T;
        const int s0 = t * per < tsize ? t * per : tsize;
        const int s1 = s0 + per < tsize ? s0 + per : tsize;
        auto slot_value = [&](int slot) -> uint32_t {
            if (tkey[slot] == FL_EMPTY)
                return 0u;
            const uint32_t nA = tcnt[slot] >> 16, nB = tcnt[slot] & 0xFFFFu;
            const bool ok = nz ? (nA > 0 && nB > 0) : (nA > 1);
            return ok ? ((nA + nB) << 16) | 1u : 0u;
        };
        uint32_t mysum = 0;
        for (int slot = s0; slot < s1; ++slot)
            mysum += slot_value(slot);
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
            }
        }
        __syncthreads();
        if (mbase_sh == 0xFFFFFFFFu)
            return;          // the host grows the space and redoes the search
        uint32_t run_off = before + incl - mysum;
        for (int slot = s0; slot < s1; ++slot) {
            const uint32_t v = slot_value(slot);
            if (v) {
                const uint32_t nA = tcnt[slot] >> 16, nB = tcnt[slot] & 0xFFFFu;
                const uint32_t base = mbase_sh + (run_off >> 16);
                const uint32_t bi = bbase_sh + (run_off & 0xFFFFu);
                buckets[bi] = Bucket{base, nA, nz ? nB : 0u, (uint32_t)b};
                pair_counts[bi] = nz ? (uint64_t)nA * nB : (uint64_t)nA * (nA - 1) / 2;
                tkey[slot] = base + nA;          // end of side A: cursor counts down
                tcnt[slot] = base + nA + nB;     // end of side B
            } else {
                tcnt[slot] = FL_EMPTY;
            }
            run_off += v;
        }
    }
    __syncthreads();
    // phase III: members, side A first
    for (uint32_t i = t; i < s; i += T) {
        const uint64_t e = sv[i];
        const uint32_t hi = (uint32_t)(e >> 32);
        const uint32_t slot = hi & 0x7FFFFFFFu;
        if (tcnt[slot] == FL_EMPTY)
            continue;
        const uint32_t pos = atomicSub((hi >> 31) ? &tcnt[slot] : &tkey[slot], 1u) - 1u;
        members[pos] = (uint32_t)e;
    }
    __syncthreads();
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
    for (uint32_t i = t; i < s; i += T) {
        const uint32_t Kc = (uint32_t)(okeys[seg0 + i] & kcmask);
        atomicAdd(&hist[mix32(nz ? (Kc >> 1) : Kc) >> 27], 1u);
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
        for (uint32_t i = t; i < s; i += T) {
            const uint32_t Kc = (uint32_t)(okeys[seg0 + i] & kcmask);
            const uint32_t bn = mix32(nz ? (Kc >> 1) : Kc) >> 27;
            if (bn >= blo && bn < bhi)
                sv[atomicAdd(&scur, 1u)] = ((uint64_t)Kc << 32) | ovals[seg0 + i];
        }
        __syncthreads();
        group_on_chip<Lay>(sv, scur, tkey, tcnt, nz, b, g);
    }
    return true;
}

// One CTA per run at a time (passes 1-2 as described at the top of the
// file).  When the run keeps at most FL_SMAX columns they are grouped on
// chip: a hash table of group keys with packed side counts, each group
// with candidates becomes a bucket (bucket and member space reserved with
// one global atomic pair per run) and its members are written side A first.
// A run that keeps more, after refinement (for example every column of a run
// whose c is 0), goes to the CTA's global segment instead, for the general
// sort and join.  Spilled survivors carry ((b << rbits | run) << M) | Kc in
// 64-bit keys, run counted from the start of the search, and the per-CTA
// segments fill across launch groups until the host sorts them.  kc_scratch
// holds, per CTA, the keys of its current run in bit-major order: kx of
// column 32w + cc at cc * P + w.
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
__global__ void __launch_bounds__(FL_THREADS, 1)
    filter_kernel(const uint32_t *__restrict__ Xr, int64_t Pp, int64_t P,
                  const uint32_t *__restrict__ ybs, int64_t Wp, int B, int64_t n, int64_t p, int M,
                  uint64_t seed, int64_t l0, int R, int NB, int BB, int rbits, int64_t rbase,
                  uint32_t mcap, uint32_t bcap, uint32_t *__restrict__ kc_scratch,
                  void *__restrict__ seg_keys_v, uint32_t *__restrict__ seg_vals,
                  uint32_t *__restrict__ seg_count, uint32_t seg_cap, int *__restrict__ overflow,
                  uint8_t *__restrict__ cnz, uint32_t *__restrict__ members,
                  uint32_t *__restrict__ members_count, Bucket *__restrict__ buckets,
                  uint64_t *__restrict__ pair_counts, uint32_t *__restrict__ nbuckets,
                  const uint64_t *__restrict__ cdf, uint64_t wtot, const float *__restrict__ Xrs,
                  int64_t Pf, int part_max, uint32_t *__restrict__ work)
{
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
    __shared__ uint32_t cursor;         // global segment fill
    __shared__ uint32_t ns;             // survivors of the current (run, response)
    __shared__ uint32_t scur;           // survivor array fill after refinement
    const int T = (int)blockDim.x;      // a multiple of 32, at most FL_THREADS
    __shared__ uint32_t seg0_sh;        // first segment entry of the current (run, response)
    const GroupOut gout{members, members_count, buckets, pair_counts, nbuckets, mcap, bcap, overflow};
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
    if (t == 0)
        cursor = seg_count[blockIdx.x];     // segments fill across launch groups

    // work item = (run r, block of responses [b0, b1)); the keys of the run
    // and its filter are built once per item.  Items are taken from a
    // launch-wide counter, so a CTA that drew an expensive run takes fewer.
    __shared__ int item_sh;
    for (;;) {
        if (t == 0)
            item_sh = (int)atomicAdd(work, 1u);
        __syncthreads();
        const int item = item_sh;           // every thread reads it before the next barrier
        if (item >= R * NB)
            break;
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
                        t == 0)
                        cursor = seg0_sh;           // grouped on chip: the entries leave the segment
                    continue;
                }
            }
            group_on_chip<Lay>(sv, s, tkey, tcnt, nz, b, gout);
        }
    }
    if (t == 0) {
        seg_count[blockIdx.x] = cursor < seg_cap ? cursor : seg_cap;
        if (cursor > seg_cap)
            atomicOr(overflow, 1);
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
//           append each to its class: each warp stages its keys per class
//           in shared memory (the filter and survivor array are free until
//           the rounds) and moves them to the CTA's class lists 16 at a
//           time, so the lists are written in whole sectors;
//   rounds  for each class q: a fresh filter F of the class-q keys, tested
//           by the keys k of class q ^ class(c) -- exactly those with
//           k ^ c in class q, so every key k ^ c is looked up in the filter
//           that holds its class; survivors go to the CTA's segment as
//           (runbits | Kc, j).
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
                      const uint64_t *__restrict__ cdf, uint64_t wtot, int part_max, uint32_t *__restrict__ work)
{
    using Lay = FlLayout<false>;
    constexpr int FB_WARPS = FL_THREADS / 32;
    constexpr uint32_t FB_BUF = 48;                // staged entries per warp and class
    constexpr uint32_t FB_NONE = 0xFFFFFFFFu;      // padding key (real keys have M <= 28 bits)
    static_assert(2 * FB_WARPS * 16 * (int)FB_BUF <= Lay::OFF_KM, "staging fits the filter and survivor array");
    static_assert(FB_WARPS * 16 <= FL_KWORDS, "staged counts fit the keep-mask region");
    extern __shared__ __align__(16) uint32_t fl_smem[];
    uint32_t *F = fl_smem;                                                   // [FL_FWORDS], in the rounds
    uint64_t *sv = reinterpret_cast<uint64_t *>(fl_smem + Lay::OFF_SV);      // [SMAX], after the rounds
    uint32_t *tkey = fl_smem + Lay::OFF_TAB;                                 // [Lay::T], after the rounds
    uint32_t *tcnt = fl_smem + Lay::OFF_TAB + Lay::T;
    const int t = threadIdx.x;
    const int lane = t & 31, wp = t >> 5;
    const int T = (int)blockDim.x;
    // pass 1 staging: per warp and class FB_BUF keys and columns, and counts
    uint32_t *mk = fl_smem + wp * 16 * FB_BUF;
    uint32_t *mc = fl_smem + FB_WARPS * 16 * FB_BUF + wp * 16 * FB_BUF;
    uint32_t *mw = fl_smem + Lay::OFF_KM + wp * 16;
    __shared__ int64_t rowoff[32];
    __shared__ uint32_t c_sh, cursor, seg0_sh;
    __shared__ uint32_t cls_n[16];                 // fill of each class list
    __shared__ int item_sh, lovf_sh;
    const GroupOut gout{members, members_count, buckets, pair_counts, nbuckets, mcap, bcap, overflow};
    const uint32_t P32 = (uint32_t)P, p32 = (uint32_t)p;
    const uint32_t steps = (P32 + T - 1) / T;
    const int fshift = 32 - (FL_LOGF - 5);
    const uint32_t kcmask = (1u << M) - 1u;                                  // M <= 28
    uint32_t *lk = lst_keys + (int64_t)blockIdx.x * 16 * lcap;               // [16][lcap]
    uint32_t *lc = lst_cols + (int64_t)blockIdx.x * 16 * lcap;
    uint64_t *okeys = reinterpret_cast<uint64_t *>(seg_keys_v) + (int64_t)blockIdx.x * seg_cap;
    uint32_t *ovals = seg_vals + (int64_t)blockIdx.x * seg_cap;
    if (t == 0)
        cursor = seg_count[blockIdx.x];     // segments fill across launch groups

    // the first 16 staged entries of class q (cntq staged) to the class list;
    // the rest move down.  Executed by the whole warp.
    auto flush16 = [&](uint32_t q, uint32_t cntq) {
        uint32_t pos = 0;
        if (lane == 0)
            pos = atomicAdd(&cls_n[q], 16u);
        pos = __shfl_sync(FULL, pos, 0);
        if (pos + 16 <= lcap) {
            if (lane < 16) {
                lk[(int64_t)q * lcap + pos + lane] = mk[q * FB_BUF + lane];
                lc[(int64_t)q * lcap + pos + lane] = mc[q * FB_BUF + lane];
            }
        } else if (lane == 0) {
            lovf_sh = 1;
        }
        const uint32_t rest = cntq - 16;         // <= 32
        uint32_t ek = 0, ec = 0;
        if ((uint32_t)lane < rest) {
            ek = mk[q * FB_BUF + 16 + lane];
            ec = mc[q * FB_BUF + 16 + lane];
        }
        __syncwarp();
        if ((uint32_t)lane < rest) {
            mk[q * FB_BUF + lane] = ek;
            mc[q * FB_BUF + lane] = ec;
        }
        if (lane == 0)
            mw[q] = rest;
        __syncwarp();
    };

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
        if (lane < 16)
            mw[lane] = 0;
        if (t < 16)
            cls_n[t] = 0;
        __syncthreads();
        const uint32_t c = c_sh;
        const bool nz = c != 0;

        // pass 1: keys with their classes, staged per warp and class
        for (uint32_t st = 0; st < steps; ++st) {
            const uint32_t w = st * T + t;
            const bool wv = w < P32;
            uint32_t A[32];
#pragma unroll
            for (int m = 0; m < 32; ++m)
                A[m] = (wv && m < MB && m < M) ? __ldg(Xr + rowoff[m] + w) : 0u;
            uint32_t Q[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int m = 0; m < MB && m < 28; ++m)
                Q[m & 3] ^= A[m];                // rows past M are zero
#pragma unroll
            for (int b = 0; b < 4; ++b)
                A[28 + b] = Q[b];
            transpose32(A);
            const uint32_t ncol = !wv ? 0u : (32 * w + 32 <= p32) ? 32u : p32 - 32 * w;
#pragma unroll
            for (int cc = 0; cc < 32; ++cc) {
                // room for this step's appends: no class above 16 staged
                for (;;) {
                    uint32_t full = __ballot_sync(FULL, lane < 16 && mw[lane] > 16);
                    if (!full)
                        break;
                    while (full) {
                        const uint32_t q = __ffs(full) - 1;
                        full &= full - 1;
                        flush16(q, mw[q]);
                    }
                }
                if ((uint32_t)cc < ncol) {
                    const uint32_t q = A[cc] >> 28;
                    const uint32_t slot = atomicAdd(&mw[q], 1u);     // < FB_BUF
                    mk[q * FB_BUF + slot] = A[cc] & kcmask;
                    mc[q * FB_BUF + slot] = 32 * w + cc;
                }
                __syncwarp();
            }
        }
        // what is still staged, the last entries of a class padded to 16
        for (uint32_t q = 0; q < 16; ++q) {
            uint32_t left = mw[q];
            while (left >= 16) {
                flush16(q, left);
                left = mw[q];
            }
            if (left > 0) {
                if ((uint32_t)lane >= left && lane < 16) {
                    mk[q * FB_BUF + lane] = FB_NONE;
                    mc[q * FB_BUF + lane] = 0;
                }
                __syncwarp();
                flush16(q, 16);
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
        // segment, warp-aggregated; the whole CTA walks the class list
        auto emit_class = [&](uint32_t q2, bool test) {
            const uint32_t n2 = cls_n[q2] < lcap ? cls_n[q2] : lcap;
            for (uint32_t i0 = 0; i0 < n2; i0 += T) {
                const uint32_t i = i0 + t;
                bool pass = false;
                uint32_t k = 0;
                if (i < n2) {
                    k = lk[(int64_t)q2 * lcap + i];
                    pass = k != FB_NONE && (!test || bloom_has(F, k ^ c, fshift));
                }
                const uint32_t bal = __ballot_sync(FULL, pass);
                if (bal == 0)
                    continue;
                uint32_t base = 0;
                if (lane == 0)
                    base = atomicAdd(&cursor, (uint32_t)__popc(bal));
                base = __shfl_sync(FULL, base, 0);
                if (pass) {
                    const uint32_t o = base + __popc(bal & ((1u << lane) - 1u));
                    if (o < seg_cap) {
                        okeys[o] = runbits | canon(k, c, tb, lowmask);
                        ovals[o] = lc[(int64_t)q2 * lcap + i];
                    }
                }
            }
        };
        if (!nz) {
            // c == 0: every column survives
            for (uint32_t q = 0; q < 16; ++q)
                emit_class(q, false);
        } else {
            const uint32_t cq = key_class(c);
            for (uint32_t q = 0; q < 16; ++q) {
                for (int i = t; i < FL_FWORDS; i += T)
                    F[i] = 0;
                __syncthreads();
                const uint32_t nq = cls_n[q] < lcap ? cls_n[q] : lcap;
                for (uint32_t i = t; i < nq; i += T) {
                    const uint32_t k = lk[(int64_t)q * lcap + i];
                    if (k != FB_NONE) {
                        uint32_t word, mask;
                        bloom_pos(k, fshift, word, mask);
                        atomicOr(F + word, mask);
                    }
                }
                __syncthreads();
                emit_class(q ^ cq, true);
                __syncthreads();
            }
        }
        __syncthreads();
        const uint32_t seg0 = seg0_sh, s = cursor - seg0;
        __syncthreads();                     // every thread has read the cursor
        if (group_from_segment<Lay>(okeys, ovals, seg0, s, seg_cap, part_max, kcmask, sv, tkey, tcnt, nz, 0,
                                    gout) &&
            t == 0)
            cursor = seg0;                   // grouped on chip: the entries leave the segment
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
    // a class list holds p / 16 keys on average: room for 1.5 times that,
    // plus the padding of every warp's last flush (< 16 per warp)
    const int64_t l = (3 * p + 31) / 32 + 16 * (FL_THREADS / 32);
    return (uint32_t)((l + 15) / 16 * 16);
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
                          int64_t *launches, int part_max, uint32_t *work)
{
    const bool batch = B > 1;
    const size_t smem = filter_smem_bytes(batch);
    using KernT = void (*)(const uint32_t *, int64_t, int64_t, const uint32_t *, int64_t, int, int64_t,
                           int64_t, int, uint64_t, int64_t, int, int, int, int, int64_t, uint32_t, uint32_t,
                           uint32_t *, void *, uint32_t *, uint32_t *, uint32_t, int *, uint8_t *,
                           uint32_t *, uint32_t *, Bucket *, uint64_t *, uint32_t *, const uint64_t *,
                           uint64_t, const float *, int64_t, int, uint32_t *);
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
    kern<<<grid, filter_threads(pk.P), smem, s>>>(pk.Xr, pk.Pp, pk.P, ybs, pk.Wp, B, pk.n, pk.p, M, seed, l0, R,
                                        NB, BB, rbits, rbase, mcap, bcap, kc_scratch, seg_keys, seg_vals,
                                        seg_count, seg_cap, overflow, cnz, members, members_count,
                                        buckets, pair_counts, nbuckets, pk.cdf, pk.wtotal, pk.Xrs, pk.Pf,
                                        part_max, work);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_filter_big(const Packed &pk, int M, uint64_t seed, int64_t l0, int R, int rbits, int64_t rbase,
                              int grid, uint32_t mcap, uint32_t bcap, uint32_t *lst_keys, uint32_t *lst_cols,
                              uint32_t lcap, uint64_t *seg_keys, uint32_t *seg_vals, uint32_t *seg_count,
                              uint32_t seg_cap, int *overflow, uint8_t *cnz, uint32_t *members,
                              uint32_t *members_count, Bucket *buckets, uint64_t *pair_counts, uint32_t *nbuckets,
                              cudaStream_t s, int64_t *launches, int part_max, uint32_t *work)
{
    const size_t smem = filter_smem_bytes(false);
    using KernT = void (*)(const uint32_t *, int64_t, int64_t, const uint32_t *, int64_t, int64_t, int, uint64_t,
                           int64_t, int, int, int64_t, uint32_t, uint32_t, uint32_t *, uint32_t *, uint32_t, void *,
                           uint32_t *, uint32_t *, uint32_t, int *, uint8_t *, uint32_t *, uint32_t *, Bucket *,
                           uint64_t *, uint32_t *, const uint64_t *, uint64_t, int, uint32_t *);
    const KernT kern = M <= 8 ? filter_big_kernel<8> : M <= 16 ? filter_big_kernel<16>
                       : M <= 24 ? filter_big_kernel<24> : filter_big_kernel<32>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    kern<<<grid, filter_threads(pk.P), smem, s>>>(pk.Xr, pk.Pp, pk.P, pk.yb, pk.n, pk.p, M, seed, l0, R, rbits, rbase,
                                                  mcap, bcap, lst_keys, lst_cols, lcap, seg_keys, seg_vals, seg_count,
                                                  seg_cap, overflow, cnz, members, members_count, buckets,
                                                  pair_counts, nbuckets, pk.cdf, pk.wtotal, part_max, work);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace xyz
