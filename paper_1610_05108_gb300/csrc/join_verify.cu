// K4 join, K5 verify, K6 unique, K7 pair sampler.
//
// Join (Section 2.2, Figure 2): after the sort, the entries of one run with
// one canonical key form a group; a group with entries on both sides (or,
// for a run whose response key c is 0, with at least two entries) yields
// the Cartesian product of its sides as candidates.  One thread per sorted
// entry detects group heads; a head whose successor is in the same group
// finds the group end by galloping and the side split by binary search, and
// appends one bucket with its pair count.  Singleton groups -- almost every
// entry -- cost three coalesced key reads.
//
// Verify (the verification step of Algorithm 2): candidate t of the launch group is decoded to
// (bucket, a, b) through the exclusive scan of the bucket pair counts, so
// every thread gets one candidate regardless of how skewed the buckets are.
// The agreement is a_jk = sum_w popc(~(Xc_j[w] ^ Xc_k[w] ^ yb[w])): bit i of
// the xor is 1 exactly when Y_i != X_ij X_ik, and padding bits contribute 0.
#include "xyz_internal.cuh"

namespace xyz {
namespace {

constexpr int JV_THREADS = 256;

template <typename K>
__device__ __forceinline__ K group_of(K key, int sh) { return key >> sh; }

template <typename K>
__global__ void __launch_bounds__(JV_THREADS)
    join_kernel(const K *__restrict__ keys, int64_t N, int M, int rbits, int runbits,
                const uint8_t *__restrict__ cnz, Bucket *__restrict__ buckets,
                uint64_t *__restrict__ pair_counts, uint32_t *__restrict__ nbuckets)
{
    const int resp_shift = M + runbits;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const K ki = keys[i];
        const int r = rbits > 0 ? (int)(ki >> M) : 0;
        const int sh = cnz[r] ? 1 : 0;
        const K gi = group_of(ki, sh);
        // Entries of other runs never share a group value: the run index sits
        // above the M >= sh key bits, so equal (key >> sh) implies equal run.
        if (i > 0 && group_of(keys[i - 1], sh) == gi)
            continue;                                   // not a head
        if (i + 1 >= N || group_of(keys[i + 1], sh) != gi)
            continue;                                   // singleton group
        int64_t good = i + 1, bad = N, step = 1;
        while (true) {
            int64_t probe = good + step;
            if (probe >= N)
                break;
            if (group_of(keys[probe], sh) == gi) {
                good = probe;
                step <<= 1;
            } else {
                bad = probe;
                break;
            }
        }
        while (bad - good > 1) {
            int64_t mid = good + (bad - good) / 2;
            if (group_of(keys[mid], sh) == gi)
                good = mid;
            else
                bad = mid;
        }
        const int64_t end = bad;
        uint32_t nA, nB;
        uint64_t pairs;
        if (sh) {
            int64_t a = i, b = end;                      // first side-B entry
            while (a < b) {
                int64_t mid = a + (b - a) / 2;
                if (keys[mid] & (K)1)
                    b = mid;
                else
                    a = mid + 1;
            }
            nA = (uint32_t)(a - i);
            nB = (uint32_t)(end - a);
            if (nA == 0 || nB == 0)
                continue;
            pairs = (uint64_t)nA * nB;
        } else {
            nA = (uint32_t)(end - i);
            nB = 0;
            pairs = (uint64_t)nA * (nA - 1) / 2;
        }
        uint32_t b = atomicAdd(nbuckets, 1u);
        const uint32_t resp = resp_shift < (int)(8 * sizeof(K)) ? (uint32_t)(ki >> resp_shift) : 0u;
        buckets[b] = Bucket{(uint32_t)i, nA, nB, resp};
        pair_counts[b] = pairs;
    }
}

__device__ __forceinline__ int agree_cols(const uint32_t *__restrict__ Xc, int64_t Wp,
                                          const uint32_t *__restrict__ yb, int64_t j, int64_t k)
{
    const uint4 *cj = reinterpret_cast<const uint4 *>(Xc + j * Wp);
    const uint4 *ck = reinterpret_cast<const uint4 *>(Xc + k * Wp);
    const uint4 *y4 = reinterpret_cast<const uint4 *>(yb);
    int a = 0;
    const int64_t nq = Wp >> 2;
    for (int64_t q = 0; q < nq; ++q) {
        uint4 x = __ldg(cj + q), z = __ldg(ck + q), y = __ldg(y4 + q);
        a += __popc(~(x.x ^ z.x ^ y.x)) + __popc(~(x.y ^ z.y ^ y.y)) +
             __popc(~(x.z ^ z.z ^ y.z)) + __popc(~(x.w ^ z.w ^ y.w));
    }
    return a;
}

// Verification with eight lanes per candidate: each warp decodes 32
// consecutive candidates (one per lane), then in eight steps handles four of
// them at a time, the eight lanes of a group reading consecutive 16-byte
// pieces of the two columns (fully used 128-byte segments) and summing their
// popcounts with shuffles.  Each lane keeps its pieces of the response bits
// in registers across the steps.
// VQ: response pieces per lane held in registers (columns up to VQ * 1024 rows)

// Weighted agreement of one 32-row word (Section 3.1): sum over the agreeing
// rows of their fixed-point weights, from the weights' bit planes of that
// word (plane b holds bit b of q_i for the word's 32 rows).
__device__ __forceinline__ int32_t word_weight(const uint32_t *__restrict__ planes, int64_t w, uint32_t g)
{
    const uint32_t *pl = planes + w * XYZ_WPLANES;
    int32_t s = 0;
#pragma unroll
    for (int b = 0; b < XYZ_WPLANES; ++b)
        s += __popc(g & __ldg(pl + b)) << b;
    return s;                     // <= 32 (2^25 - 1) < 2^31
}

template <bool BATCH, bool WEIGHTED, int VQ>
__global__ void __launch_bounds__(JV_THREADS, (VQ == 2 && !WEIGHTED) ? 5 : (!WEIGHTED ? 3 : 1))   // 5: 48, 3: 80 registers
    verify_kernel(const uint32_t *__restrict__ Xc, int64_t Wp, const uint32_t *__restrict__ yb,
                  const Bucket *__restrict__ buckets, const uint64_t *__restrict__ pair_off,
                  const uint32_t *__restrict__ nbuckets, const uint64_t *__restrict__ total_pairs,
                  const uint32_t *__restrict__ vals, int64_t amin, int kbits,
                  uint64_t *__restrict__ rec_keys, uint32_t *__restrict__ rec_agree,
                  uint32_t *__restrict__ nrec, uint32_t rec_cap, const int *__restrict__ abort_flag,
                  const uint32_t *__restrict__ planes, int64_t wQ, double kq,
                  const uint32_t *__restrict__ bstart, int64_t bstart_cap, int *__restrict__ verr)
{
    // WEIGHTED (real response, Section 3.1): yb holds the signs of Y; a
    // candidate passes when (double)(2 S - Q) >= kappa * Q, S the weight sum
    // of its agreeing rows (the records still carry the agreement count).
    // abort_flag (may be null): bit 2 set means the producer of the buckets
    // ran out of space after reserving some of them, so their entries are not
    // all written; the whole launch group is then skipped (and redone).
    if (abort_flag && (*(volatile const int *)abort_flag & 2))
        return;
    // BATCH: yb holds one response-bit row of Wp words per response; a
    // bucket's pad names its response, which is also the top field of the
    // record key (resp << 2 kbits | j << kbits | k).
    const uint32_t nb = *nbuckets;
    const uint64_t T = *total_pairs;
    const int lane = threadIdx.x & 31;
    const int sub = lane & 7;
    const int nq = (int)(Wp >> 2);
    const uint4 *y4 = reinterpret_cast<const uint4 *>(yb);
    uint4 yr[VQ];
#pragma unroll
    for (int i = 0; i < VQ; ++i) {
        const int q = sub + 8 * i;
        yr[i] = q < nq ? __ldg(y4 + q) : make_uint4(0, 0, 0, 0);
    }
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // Each warp takes 32 consecutive candidates; the bucket of the first comes
    // from the block starts (else lane 0's binary search).
    for (uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); t0 < T; t0 += stride) {
        uint32_t base = 0;
        if (bstart && (int64_t)(t0 >> 5) < bstart_cap) {
            base = bstart[t0 >> 5];        // bucket of candidate t0, precomputed
        } else {
            if (lane == 0) {
                uint32_t lo = 0, hi = nb;      // pair_off[lo] <= t0 < pair_off[hi] (reading T for [nb])
                while (hi - lo > 1) {
                    uint32_t mid = lo + (hi - lo) / 2;
                    if (pair_off[mid] <= t0)
                        lo = mid;
                    else
                        hi = mid;
                }
                base = lo;
            }
            base = __shfl_sync(0xffffffffu, base, 0);
        }
        const uint64_t t = t0 + lane;
        bool valid = t < T;
        // Bucket of each lane's candidate.  32 consecutive candidates span
        // buckets base .. base + 31 (each holds >= 1), so lane i reads the
        // start of bucket base + 1 + i (one coalesced load); a start at
        // offset d in 1..31 of the block sets bit d, and a lane's bucket is
        // base plus the bits at or below its offset.
        const uint32_t bi = base + 1u + (uint32_t)lane;
        const uint64_t po = bi < nb ? pair_off[bi] : ~0ULL;
        const uint64_t d = po - t0;
        const uint32_t mark = __reduce_or_sync(0xffffffffu, d < 32 ? (1u << d) : 0u);
        uint32_t j = 0, k = 0, resp = 0;
        if (valid) {
            const uint32_t lo = base + __popc(mark & (0xFFFFFFFFu >> (31 - lane)));
            const Bucket B = buckets[lo];
            const uint64_t u = t - pair_off[lo];
            // self-check: the offset must lie inside the bucket before any of
            // its members is read; a miss is reported, never dereferenced
            const uint64_t np = B.nB ? (uint64_t)B.nA * B.nB : (uint64_t)B.nA * (B.nA - 1) / 2;
            if (u >= np) {
                valid = false;
                if (verr)
                    atomicOr(verr, 2);
            }
            resp = B.pad;
            if (!valid) {
                // nothing to read
            } else if (B.nB) {
                uint64_t ia = u / B.nB, ib = u - ia * B.nB;
                j = vals[B.start + ia];
                k = vals[B.start + B.nA + ib];
            } else {
                // u -> (x, y), x > y, u = x(x-1)/2 + y
                uint64_t x = (uint64_t)((1.0 + sqrt(1.0 + 8.0 * (double)u)) * 0.5);
                while (x * (x - 1) / 2 > u)
                    --x;
                while ((x + 1) * x / 2 <= u)
                    ++x;
                uint64_t y = u - x * (x - 1) / 2;
                j = vals[B.start + x];
                k = vals[B.start + y];
            }
        }
        int agree = 0;
        int64_t wsum = 0;
#pragma unroll
        for (int st = 0; st < 8; ++st) {
            const int cidx = 4 * st + (lane >> 3);           // candidate of this lane's group
            const uint32_t jj = __shfl_sync(0xffffffffu, j, cidx);
            const uint32_t kk = __shfl_sync(0xffffffffu, k, cidx);
            const bool vv = __shfl_sync(0xffffffffu, (int)valid, cidx) != 0;
            const uint32_t rr = BATCH ? __shfl_sync(0xffffffffu, resp, cidx) : 0u;
            int part = 0;
            int64_t wpart = 0;
            if (vv) {
                const uint4 *cj = reinterpret_cast<const uint4 *>(Xc + (int64_t)jj * Wp);
                const uint4 *ck = reinterpret_cast<const uint4 *>(Xc + (int64_t)kk * Wp);
                const uint4 *yq = BATCH ? reinterpret_cast<const uint4 *>(yb + (int64_t)rr * Wp) : y4;
#pragma unroll
                for (int i = 0; i < VQ; ++i) {
                    const int q = sub + 8 * i;
                    if (q < nq) {
                        const uint4 x = __ldg(cj + q), z = __ldg(ck + q);
                        const uint4 y = BATCH ? __ldg(yq + q) : yr[i];
                        const uint32_t g0 = ~(x.x ^ z.x ^ y.x), g1 = ~(x.y ^ z.y ^ y.y);
                        const uint32_t g2 = ~(x.z ^ z.z ^ y.z), g3 = ~(x.w ^ z.w ^ y.w);
                        part += __popc(g0) + __popc(g1) + __popc(g2) + __popc(g3);
                        if (WEIGHTED)
                            wpart += (int64_t)word_weight(planes, 4 * q, g0) + word_weight(planes, 4 * q + 1, g1) +
                                     (int64_t)word_weight(planes, 4 * q + 2, g2) + word_weight(planes, 4 * q + 3, g3);
                    }
                }
                for (int q = sub + 8 * VQ; q < nq; q += 8) {
                    const uint4 x = __ldg(cj + q), z = __ldg(ck + q), y = __ldg(yq + q);
                    const uint32_t g0 = ~(x.x ^ z.x ^ y.x), g1 = ~(x.y ^ z.y ^ y.y);
                    const uint32_t g2 = ~(x.z ^ z.z ^ y.z), g3 = ~(x.w ^ z.w ^ y.w);
                    part += __popc(g0) + __popc(g1) + __popc(g2) + __popc(g3);
                    if (WEIGHTED)
                        wpart += (int64_t)word_weight(planes, 4 * q, g0) + word_weight(planes, 4 * q + 1, g1) +
                                 (int64_t)word_weight(planes, 4 * q + 2, g2) + word_weight(planes, 4 * q + 3, g3);
                }
            }
            part += __shfl_xor_sync(0xffffffffu, part, 4);
            part += __shfl_xor_sync(0xffffffffu, part, 2);
            part += __shfl_xor_sync(0xffffffffu, part, 1);
            const int got = __shfl_sync(0xffffffffu, part, 8 * (lane & 3));
            if ((lane >> 2) == st)
                agree = got;
            if (WEIGHTED) {
                wpart += __shfl_xor_sync(0xffffffffu, wpart, 4);
                wpart += __shfl_xor_sync(0xffffffffu, wpart, 2);
                wpart += __shfl_xor_sync(0xffffffffu, wpart, 1);
                const int64_t wgot = __shfl_sync(0xffffffffu, wpart, 8 * (lane & 3));
                if ((lane >> 2) == st)
                    wsum = wgot;
            }
        }
        const bool pass = WEIGHTED ? (double)(2 * wsum - wQ) >= kq : agree >= amin;
        if (valid && pass) {
            uint32_t idx = atomicAdd(nrec, 1u);
            if (idx < rec_cap) {
                uint32_t lo_c = j < k ? j : k, hi_c = j < k ? k : j;
                rec_keys[idx] = ((uint64_t)resp << (2 * kbits)) | ((uint64_t)lo_c << kbits) | hi_c;
                rec_agree[idx] = (uint32_t)agree;
            }
        }
    }
}

// For every block of 32 consecutive candidates, the bucket holding its first
// candidate: bucket b writes the blocks that start in [pair_off[b],
// pair_off[b+1]), so every block below bstart_cap gets exactly one writer.
// abort_flag as in verify_kernel: when the producer ran out of bucket space
// its bucket count passes the arrays, and nothing is read.
__global__ void block_start_kernel(const uint64_t *__restrict__ pair_off, const uint32_t *__restrict__ nbuckets,
                                   const uint64_t *__restrict__ total_pairs, uint32_t *__restrict__ bstart,
                                   int64_t bstart_cap, const int *__restrict__ abort_flag)
{
    if (abort_flag && (*(volatile const int *)abort_flag & 2))
        return;
    const uint32_t nb = *nbuckets;
    const uint64_t T = *total_pairs;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += stride) {
        // the scan leaves pair_off[nb] unwritten: the last bucket ends at T
        const uint64_t lo = pair_off[b], hi = b + 1 < nb ? pair_off[b + 1] : T;
        uint64_t k1 = (hi + 31) >> 5;
        if (k1 > (uint64_t)bstart_cap)
            k1 = (uint64_t)bstart_cap;
        for (uint64_t k = (lo + 31) >> 5; k < k1; ++k)
            bstart[k] = (uint32_t)b;
    }
}

__global__ void unique_flags_kernel(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ nrec,
                                    int64_t cap, uint32_t *__restrict__ flags)
{
    int64_t N = *nrec;
    if (N > cap)
        N = cap;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
        flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void unique_scatter_kernel(const uint64_t *__restrict__ keys,
                                      const uint32_t *__restrict__ agree,
                                      const uint32_t *__restrict__ nrec, int64_t cap,
                                      const uint32_t *__restrict__ flags,
                                      const uint32_t *__restrict__ pos, int kbits, int64_t n,
                                      PairOut *__restrict__ out, uint32_t *__restrict__ resp)
{
    int64_t N = *nrec;
    if (N > cap)
        N = cap;
    const uint64_t kmask = (kbits >= 64) ? ~0ULL : ((1ULL << kbits) - 1ULL);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        if (!flags[i])
            continue;
        uint64_t key = keys[i];
        PairOut o;
        o.j = (int32_t)((key >> kbits) & kmask);
        o.k = (int32_t)(key & kmask);
        o.agree = (int32_t)agree[i];
        o.strength = (float)((double)(2 * (int64_t)agree[i] - n) / (double)n);
        out[pos[i]] = o;
        if (resp)
            resp[pos[i]] = (uint32_t)(key >> (2 * kbits));
    }
}

// The union of a small record set (at most UQ_SMALL records) in one CTA:
// bitonic sort of (key, agree) in shared memory, then the first record of
// every key is written to its place; same result as the sort + unique pair.
constexpr int UQ_SMALL = 2048;
constexpr int UQ_THREADS = 1024;

__global__ void __launch_bounds__(UQ_THREADS)
    unique_small_kernel(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ agree, int N, int kbits,
                        int64_t n, PairOut *__restrict__ out, uint32_t *__restrict__ nout,
                        uint32_t *__restrict__ resp)
{
    __shared__ uint64_t sk[UQ_SMALL];
    __shared__ uint32_t sa[UQ_SMALL];
    __shared__ uint32_t wsum[UQ_THREADS / 32];
    const int t = threadIdx.x;
    int size = 1;
    while (size < N)
        size <<= 1;
    for (int i = t; i < size; i += UQ_THREADS) {
        sk[i] = i < N ? keys[i] : ~0ULL;
        sa[i] = i < N ? agree[i] : 0u;
    }
    __syncthreads();
    for (int k = 2; k <= size; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = t; i < size; i += UQ_THREADS) {
                const int l = i ^ jj;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const uint64_t a = sk[i], b = sk[l];
                    if ((a > b) == up) {
                        sk[i] = b;
                        sk[l] = a;
                        const uint32_t x = sa[i];
                        sa[i] = sa[l];
                        sa[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    // first record of each key: flag, block-wide exclusive scan (two per thread)
    const int i0 = 2 * t, i1 = 2 * t + 1;
    const uint32_t f0 = (i0 < N && (i0 == 0 || sk[i0] != sk[i0 - 1])) ? 1u : 0u;
    const uint32_t f1 = (i1 < N && sk[i1] != sk[i1 - 1]) ? 1u : 0u;
    const uint32_t mine = f0 + f1;
    const int lane = t & 31, wp = t >> 5;
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += y;
    }
    if (lane == 31)
        wsum[wp] = incl;
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < UQ_THREADS / 32; ++w) {
        before += w < wp ? wsum[w] : 0u;
        total += wsum[w];
    }
    uint32_t pos = before + incl - mine;
    const uint64_t kmask = (kbits >= 64) ? ~0ULL : ((1ULL << kbits) - 1ULL);
    for (int q = 0; q < 2; ++q) {
        const int i = q ? i1 : i0;
        if (q ? f1 : f0) {
            const uint64_t key = sk[i];
            PairOut o;
            o.j = (int32_t)((key >> kbits) & kmask);
            o.k = (int32_t)(key & kmask);
            o.agree = (int32_t)sa[i];
            o.strength = (float)((double)(2 * (int64_t)sa[i] - n) / (double)n);
            out[pos] = o;
            if (resp)
                resp[pos] = (uint32_t)(key >> (2 * kbits));
            ++pos;
        }
    }
    if (t == 0)
        *nout = total;
}

__global__ void agree_pairs_kernel(const uint32_t *__restrict__ Xc, int64_t Wp,
                                   const uint32_t *__restrict__ yb, const int32_t *__restrict__ j,
                                   const int32_t *__restrict__ k, int64_t count,
                                   int32_t *__restrict__ agree)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride)
        agree[t] = agree_cols(Xc, Wp, yb, j[t], k[t]);
}

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Pair number t uses splitmix64 outputs 2t and 2t+1 of `seed`: j uniform on
// [0, p), k uniform on [0, p) \ {j}.
__global__ void sample_pairs_kernel(const uint32_t *__restrict__ Xc, int64_t Wp,
                                    const uint32_t *__restrict__ yb, int64_t p, uint64_t seed,
                                    int64_t count, int32_t *__restrict__ jo,
                                    int32_t *__restrict__ ko, int32_t *__restrict__ agree)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride) {
        uint64_t u1 = mix64(seed + (uint64_t)(2 * t + 1) * 0x9E3779B97F4A7C15ULL);
        uint64_t u2 = mix64(seed + (uint64_t)(2 * t + 2) * 0x9E3779B97F4A7C15ULL);
        int64_t j = (int64_t)__umul64hi(u1, (uint64_t)p);
        int64_t k = (int64_t)__umul64hi(u2, (uint64_t)(p - 1));
        if (k >= j)
            ++k;
        jo[t] = (int32_t)j;
        ko[t] = (int32_t)k;
        agree[t] = agree_cols(Xc, Wp, yb, j, k);
    }
}

unsigned grid_for(int64_t work, int threads, int64_t max_blocks)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1)
        b = 1;
    if (b > max_blocks)
        b = max_blocks;
    return (unsigned)b;
}

int g_sm_count = 0;
int64_t max_resident_blocks()
{
    if (!g_sm_count) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count <= 0)
            g_sm_count = 152;
    }
    return (int64_t)g_sm_count * 8;
}

// One block per resident slot of the kernel on every SM: the grid-stride
// loops then finish in a single wave, with no half-filled second one.
template <typename Kern>
unsigned resident_grid(Kern kernel, int cap_per_sm = 0)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, JV_THREADS, 0) != cudaSuccess || per_sm < 1)
        per_sm = 4;
    if (cap_per_sm > 0 && cap_per_sm < per_sm)
        per_sm = cap_per_sm;
    return (unsigned)(max_resident_blocks() / 8 * per_sm);
}

template <typename K>
cudaError_t join_impl(const K *keys, int64_t N, int M, int rbits, int runbits, const uint8_t *cnz,
                      Bucket *buckets, uint64_t *pair_counts, uint32_t *nbuckets, cudaStream_t s,
                      int64_t *launches)
{
    if (N <= 0)
        return cudaSuccess;
    join_kernel<K><<<grid_for(N, JV_THREADS, 1 << 20), JV_THREADS, 0, s>>>(
        keys, N, M, rbits, runbits, cnz, buckets, pair_counts, nbuckets);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_join32(const uint32_t *keys, int64_t N, int M, int rbits, const uint8_t *cnz,
                          Bucket *buckets, uint64_t *pair_counts, uint32_t *nbuckets,
                          cudaStream_t s, int64_t *launches)
{
    return join_impl<uint32_t>(keys, N, M, rbits, rbits, cnz, buckets, pair_counts, nbuckets, s,
                               launches);
}

cudaError_t launch_join64(const uint64_t *keys, int64_t N, int M, int rbits, const uint8_t *cnz,
                          Bucket *buckets, uint64_t *pair_counts, uint32_t *nbuckets,
                          cudaStream_t s, int64_t *launches, int runbits)
{
    return join_impl<uint64_t>(keys, N, M, rbits, runbits < 0 ? rbits : runbits, cnz, buckets,
                               pair_counts, nbuckets, s, launches);
}

cudaError_t launch_verify(const Packed &pk, const Bucket *buckets, const uint64_t *pair_off,
                          const uint32_t *nbuckets, const uint64_t *total_pairs,
                          const uint32_t *vals, int64_t amin, int kbits, uint64_t *rec_keys,
                          uint32_t *rec_agree, uint32_t *nrec, uint32_t rec_cap, cudaStream_t s,
                          int64_t *launches, const uint32_t *ybs, const int *abort_flag, uint32_t *bstart,
                          int64_t bstart_cap, int *verr)
{
    if (pk.Xcs && !ybs)       // real X (unbiased transform): real inner products
        return launch_verify_real(pk, buckets, pair_off, nbuckets, total_pairs, vals, kbits, rec_keys,
                                  rec_agree, nrec, rec_cap, s, launches, abort_flag);
    if (bstart && bstart_cap > 0) {
        block_start_kernel<<<(unsigned)max_resident_blocks(), JV_THREADS, 0, s>>>(pair_off, nbuckets, total_pairs,
                                                                               bstart, bstart_cap, abort_flag);
        *launches += 1;
    } else {
        bstart = nullptr;
    }
    // response pieces held in registers: 2 per lane covers columns of up to
    // 2048 rows (16 pieces of 16 bytes), 4 up to 4096; longer columns read
    // the rest from memory
    const bool short_cols = pk.Wp <= 64;
    if (ybs) {
        auto k = short_cols ? verify_kernel<true, false, 2> : verify_kernel<true, false, 4>;
        k<<<resident_grid(k, pk.verify_bpsm), JV_THREADS, 0, s>>>(pk.Xc, pk.Wp, ybs, buckets, pair_off, nbuckets, total_pairs,
                                                  vals, amin, kbits, rec_keys, rec_agree, nrec, rec_cap,
                                                  abort_flag, nullptr, 0, 0.0, bstart, bstart_cap, verr);
    } else if (pk.cdf) {
        auto k = short_cols ? verify_kernel<false, true, 2> : verify_kernel<false, true, 4>;
        k<<<resident_grid(k, pk.verify_bpsm), JV_THREADS, 0, s>>>(pk.Xc, pk.Wp, pk.yb, buckets, pair_off, nbuckets, total_pairs,
                                                  vals, amin, kbits, rec_keys, rec_agree, nrec, rec_cap,
                                                  abort_flag, pk.planes, (int64_t)pk.wtotal, pk.wkq, bstart,
                                                  bstart_cap, verr);
    } else {
        auto k = short_cols ? verify_kernel<false, false, 2> : verify_kernel<false, false, 4>;
        k<<<resident_grid(k, pk.verify_bpsm), JV_THREADS, 0, s>>>(pk.Xc, pk.Wp, pk.yb, buckets, pair_off, nbuckets, total_pairs,
                                                  vals, amin, kbits, rec_keys, rec_agree, nrec, rec_cap,
                                                  abort_flag, nullptr, 0, 0.0, bstart, bstart_cap, verr);
    }
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_unique(const uint64_t *rec_keys, const uint32_t *rec_agree, const uint32_t *nrec,
                          int64_t cap, int kbits, int64_t n, uint32_t *flags, uint32_t *pos,
                          void *scan_temp, PairOut *out, uint32_t *nout, cudaStream_t s,
                          int64_t *launches, uint32_t *resp)
{
    if (cap <= 0)
        return cudaSuccess;
    unsigned g = grid_for(cap, JV_THREADS, max_resident_blocks());
    unique_flags_kernel<<<g, JV_THREADS, 0, s>>>(rec_keys, nrec, cap, flags);
    *launches += 1;
    cudaError_t e = scan_u32_dev(flags, pos, nrec, cap, nout, scan_temp, s, launches);
    if (e != cudaSuccess)
        return e;
    unique_scatter_kernel<<<g, JV_THREADS, 0, s>>>(rec_keys, rec_agree, nrec, cap, flags, pos, kbits,
                                                   n, out, resp);
    *launches += 1;
    return cudaGetLastError();
}

int64_t unique_small_cap() { return UQ_SMALL; }

cudaError_t launch_unique_small(const uint64_t *rec_keys, const uint32_t *rec_agree, int64_t N, int kbits,
                                int64_t n, PairOut *out, uint32_t *nout, cudaStream_t s, int64_t *launches,
                                uint32_t *resp)
{
    if (N < 1 || N > UQ_SMALL)
        return cudaErrorInvalidValue;
    unique_small_kernel<<<1, UQ_THREADS, 0, s>>>(rec_keys, rec_agree, (int)N, kbits, n, out, nout, resp);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_agree_pairs(const Packed &pk, const int32_t *j, const int32_t *k, int64_t count,
                               int32_t *agree, cudaStream_t s, int64_t *launches)
{
    if (count <= 0)
        return cudaSuccess;
    agree_pairs_kernel<<<grid_for(count, JV_THREADS, max_resident_blocks()), JV_THREADS, 0, s>>>(
        pk.Xc, pk.Wp, pk.yb, j, k, count, agree);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_sample_pairs(const Packed &pk, int64_t count, uint64_t seed, int32_t *j,
                                int32_t *k, int32_t *agree, cudaStream_t s, int64_t *launches)
{
    if (count <= 0)
        return cudaSuccess;
    sample_pairs_kernel<<<grid_for(count, JV_THREADS, max_resident_blocks()), JV_THREADS, 0, s>>>(
        pk.Xc, pk.Wp, pk.yb, pk.p, seed, count, j, k, agree);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace xyz
