// Internal declarations shared by the CUDA translation units of libxyz.
// Nothing here is part of the public ABI (include/xyz.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace xyz {

// ------------------------------------------------------------ error state

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);

#define XYZ_CUDA_TRY(expr)                                                         \
    do {                                                                           \
        cudaError_t _e = (expr);                                                   \
        if (_e != cudaSuccess)                                                     \
            return ::xyz::fail(3, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

// ------------------------------------------------------------- layouts
//
// Packed X, resident for the life of a context:
//   Xc [p][Wp] uint32  column bits, bit i%32 of word i/32 is (X_ij == -1);
//                      Wp = round_up(ceil(n/32), 4) so a column is whole
//                      16-byte vectors; padding bits are 0.
//   yb [Wp]    uint32  response bits (Y_i == -1); padding bits are 1, so a
//                      padding position never counts as an agreement:
//                      ~(0 ^ 0 ^ 1) = 0.
//   Xr [n][Pp] uint32  row bits, bit j%32 of word j/32 is (X_ij == -1);
//                      Pp = round_up(ceil(p/32), 8) so a row is whole
//                      32-byte sectors; padding bits are 0.

struct Packed {
    int64_t n = 0, p = 0;
    int64_t W = 0, Wp = 0;   // words per column (used, padded)
    int64_t P = 0, Pp = 0;   // words per row (used, padded)
    uint32_t *Xc = nullptr;
    uint32_t *Xr = nullptr;
    uint32_t *yb = nullptr;
    // real response (Section 3.1): weighted rows and weighted verification;
    // null cdf = binary response
    const uint64_t *cdf = nullptr;     // [n] cumulative fixed-point weights
    uint64_t wtotal = 0;               // sum of the weights, cdf[n - 1]
    const uint32_t *planes = nullptr;  // [Wp][XYZ_WPLANES] bit planes of the weights per word
    double wkq = 0.0;                  // kappa * wtotal of the current search
    double wscale = 0.0;               // strength = (2S - Q) * wscale (0: divide by Q)
    // real X through the unbiased transform (Section 3.2); null = binary X
    const float *Xrs = nullptr;        // [n][Pf] rows of X' = X / nu_i (padding 0)
    int64_t Pf = 0;                    // row pitch in floats, a multiple of 32
    const float *Xcs = nullptr;        // [p][Wf] columns of X' (padding 0)
    int64_t Wf = 0;                    // column pitch in floats, a multiple of 32
    const double *ysd = nullptr;       // [Wf] Y' = Y nu_i^2 (padding 0), then [Wf] floats of it
    double rkq = 0.0;                  // pass: sum_i Y'_i X'_ij X'_ik >= rkq
    double rnorm = 0.0;                // ||Y'||_1 (reported strength = dot / rnorm)
    // launch shapes (xyz_set_tiles; 0 = the default rule); results never
    // depend on them
    int filter_threads = 0;            // threads per filter CTA
    int verify_bpsm = 0;               // verification blocks per SM
};

constexpr int XYZ_WPLANES = 25;        // weights are integers in [0, 2^24]

// One group of equal keys that yields candidates.  Entries [start, start+nA)
// of the sorted arrays are side A, [start+nA, start+nA+nB) side B; nB == 0
// marks a group of a run whose response key c is 0, where every unordered
// pair inside the nA entries is a candidate.
struct Bucket {
    uint32_t start;
    uint32_t nA;
    uint32_t nB;
    uint32_t pad;
};

// Arguments of the single-filter survivor kernel for one launch group of
// one search (see filter.cu); an array of them describes the instances of a
// fused launch over several searches.
struct FilterArgs {
    const uint32_t *Xr;
    int64_t Pp, P;
    const uint32_t *ybs;
    int64_t Wp;
    int B;
    int64_t n, p;
    int M;
    uint64_t seed;
    int64_t l0;
    int R, NB, BB, rbits;
    int64_t rbase;
    uint32_t mcap, bcap;
    uint32_t *kc_scratch;
    void *seg_keys_v;
    uint32_t *seg_vals, *seg_count;
    uint32_t seg_cap;
    int *overflow;
    uint8_t *cnz;
    uint32_t *members, *members_count;
    Bucket *buckets;
    uint64_t *pair_counts;
    uint32_t *nbuckets;
    const uint64_t *cdf;
    uint64_t wtot;
    const float *Xrs;
    int64_t Pf;
    int part_max;
    unsigned long long *kept;
};

// At most this many searches share one fused filter launch (their
// arguments travel as one kernel parameter of about 18 KB).
constexpr int XYZ_FUSED_MAX = 64;

// ------------------------------------------------------ kernel launchers
// Each returns cudaError_t of its launch(es); `launches` is incremented by
// the number of kernels launched.

cudaError_t launch_pack(const int8_t *dX, const int8_t *dY, const Packed &pk, int *bad_flag,
                        cudaStream_t s, int64_t *launches);
cudaError_t launch_pack_y(const int8_t *dY, const Packed &pk, int *bad_flag, cudaStream_t s,
                          int64_t *launches);

// Keys of runs [l0, l0+R) into keys[r*p + j] (composite, see keys.cu) and
// vals[r*p + j] = j; cnz[r] = 1 when the run's response key c != 0.
// raw_kx/raw_c (nullable) receive the plain keys of run l0 (R must be 1).
cudaError_t launch_keybuild32(const Packed &pk, int M, uint64_t seed, int64_t l0, int R, int rbits,
                              uint32_t *keys, uint32_t *vals, uint8_t *cnz, uint64_t *raw_kx,
                              uint64_t *raw_c, cudaStream_t s, int64_t *launches);
cudaError_t launch_keybuild64(const Packed &pk, int M, uint64_t seed, int64_t l0, int R, int rbits,
                              uint64_t *keys, uint32_t *vals, uint8_t *cnz, uint64_t *raw_kx,
                              uint64_t *raw_c, cudaStream_t s, int64_t *launches);

// LSD radix sort of (key, value) pairs on bits [0, bits).  Ping-pongs
// between (k0, v0) and (k1, v1); *in_alt is set when the result is in
// (k1, v1).  temp must hold radix_temp_bytes(N).
size_t radix_temp_bytes(int64_t N);
cudaError_t radix_sort32(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, int64_t N, int bits,
                         void *temp, bool *in_alt, cudaStream_t s, int64_t *launches);
cudaError_t radix_sort64(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int64_t N, int bits,
                         void *temp, bool *in_alt, cudaStream_t s, int64_t *launches);
int radix_passes(int bits);

// Exclusive scans with the element count read from device memory
// (count_dev) and at most `cap` elements.
size_t scan_temp_bytes(int64_t cap);
cudaError_t scan_u64_dev(const uint64_t *in, uint64_t *out, const uint32_t *count_dev, int64_t cap,
                         uint64_t *total_out, uint64_t *total_accum, void *temp, cudaStream_t s,
                         int64_t *launches);
cudaError_t scan_u32_dev(const uint32_t *in, uint32_t *out, const uint32_t *count_dev, int64_t cap,
                         uint32_t *total_out, void *temp, cudaStream_t s, int64_t *launches);

// Equal-key groups of a sorted chunk -> buckets + per-bucket pair counts.
// Keys are ((resp << runbits | run) << M) | Kc with rbits = bits above M;
// a bucket's `pad` gets resp (0 when rbits == runbits).
cudaError_t launch_join32(const uint32_t *keys, int64_t N, int M, int rbits, const uint8_t *cnz,
                          Bucket *buckets, uint64_t *pair_counts, uint32_t *nbuckets,
                          cudaStream_t s, int64_t *launches);
cudaError_t launch_join64(const uint64_t *keys, int64_t N, int M, int rbits, const uint8_t *cnz,
                          Bucket *buckets, uint64_t *pair_counts, uint32_t *nbuckets,
                          cudaStream_t s, int64_t *launches, int runbits = -1);

// Verify every candidate of the buckets; append passing (key, agree)
// records, key = j * 2^kbits + k with j < k.  verr (may be null) gets bit 2
// when a candidate's offset is not inside the bucket its lookup found (an
// internal error; the candidate is skipped, none of its members is read).
cudaError_t launch_verify(const Packed &pk, const Bucket *buckets, const uint64_t *pair_off,
                          const uint32_t *nbuckets, const uint64_t *total_pairs,
                          const uint32_t *vals, int64_t amin, int kbits, uint64_t *rec_keys,
                          uint32_t *rec_agree, uint32_t *nrec, uint32_t rec_cap, cudaStream_t s,
                          int64_t *launches, const uint32_t *ybs = nullptr,
                          const int *abort_flag = nullptr, uint32_t *bstart = nullptr,
                          int64_t bstart_cap = 0, int *verr = nullptr);

// Sorted records -> unique xyz pairs (device array), count in *nout.
struct PairOut {
    int32_t j, k, agree;
    float strength;
};
// the union of at most unique_small_cap() records (N known on the host) in
// one CTA; the same output as radix_sort64 + launch_unique
int64_t unique_small_cap();
cudaError_t launch_unique_small(const uint64_t *rec_keys, const uint32_t *rec_agree, int64_t N, int kbits,
                                int64_t n, PairOut *out, uint32_t *nout, cudaStream_t s, int64_t *launches,
                                uint32_t *resp = nullptr);
cudaError_t launch_unique(const uint64_t *rec_keys, const uint32_t *rec_agree, const uint32_t *nrec,
                          int64_t cap, int kbits, int64_t n, uint32_t *flags, uint32_t *pos,
                          void *scan_temp, PairOut *out, uint32_t *nout, cudaStream_t s,
                          int64_t *launches, uint32_t *resp = nullptr);

// Agreement of explicit pairs.
cudaError_t launch_agree_pairs(const Packed &pk, const int32_t *j, const int32_t *k, int64_t count,
                               int32_t *agree, cudaStream_t s, int64_t *launches);
// Agreement of pairs drawn uniformly from the splitmix64 stream of `seed`.
cudaError_t launch_sample_pairs(const Packed &pk, int64_t count, uint64_t seed, int32_t *j,
                                int32_t *k, int32_t *agree, cudaStream_t s, int64_t *launches);

// Partitioned grouping (group.cu), used for M <= 31.
int part_bits(int64_t p);
int part_blocks(int64_t p);
bool part_supported(int64_t p, int M);
size_t part_seg_words(int64_t p, int R);
cudaError_t launch_keybuild_part(const Packed &pk, int M, uint64_t seed, int64_t l0, int R,
                                 uint64_t *ents, uint32_t *seg, uint8_t *cnz, cudaStream_t s,
                                 int64_t *launches);
cudaError_t launch_group(const Packed &pk, int R, const uint64_t *ents, const uint32_t *seg,
                         const uint8_t *cnz, uint32_t *members, uint32_t *members_count,
                         Bucket *buckets, uint64_t *pair_counts, uint32_t *nbuckets, int *err,
                         cudaStream_t s, int64_t *launches);

// Per-run survivor filter (filter.cu), used for M <= 31 and moderate p.
bool filter_supported(int64_t p, int M);
// The class-split filter (filter_big_kernel) for one response and M <= 28
// at any p up to 2^27: per-CTA lists of lcap entries for each of 16 classes.
bool filter_big_supported(int64_t p, int M);
uint32_t filter_big_lcap(int64_t p);
uint32_t filter_big_lcap_max(int64_t p);
size_t filter_big_list_words(int64_t p, uint32_t lcap);
cudaError_t launch_filter_big(const Packed &pk, int M, uint64_t seed, int64_t l0, int R, int rbits, int64_t rbase,
                              int grid, uint32_t mcap, uint32_t bcap, uint32_t *lst_keys, uint32_t *lst_cols,
                              uint32_t lcap, uint64_t *seg_keys, uint32_t *seg_vals, uint32_t *seg_count,
                              uint32_t seg_cap, int *overflow, uint8_t *cnz, uint32_t *members,
                              uint32_t *members_count, Bucket *buckets, uint64_t *pair_counts, uint32_t *nbuckets,
                              cudaStream_t s, int64_t *launches, int part_max, uint32_t *work,
                              unsigned long long *kept);
int filter_grid();
size_t filter_scratch_words(int64_t p);
int64_t filter_run_cap();
// ybs: B response-bit rows of Wp words (B = 1: the context's own).  Runs
// [l0, l0 + R) of a search whose first run is l0 - rbase, as R * NB work
// items of one run and a block of BB responses; spilled survivors
// go to the per-CTA segments as ((b << rbits | run) << M | Kc, j) and the
// segments fill across launch groups (reset with launch_seg_reset, joined
// with launch_compact).  overflow bit 1: a segment overflowed; bit 2: the
// member/bucket space (mcap/bcap) did.  A run whose survivors pass the
// on-chip capacity is grouped on chip in at most part_max hash partitions
// of its group keys when they fit (0: never; it then always spills).  work:
// a zeroed counter from which the CTAs take their work items.  defer: when
// not null, the launch's arguments are stored there and nothing is launched
// (for launch_filter_fused).
cudaError_t launch_filter(const Packed &pk, const uint32_t *ybs, int B, int M, uint64_t seed,
                          int64_t l0, int R, int NB, int BB, int rbits, int64_t rbase, int grid,
                          uint32_t mcap, uint32_t bcap, uint32_t *kc_scratch, uint64_t *seg_keys,
                          uint32_t *seg_vals, uint32_t *seg_count, uint32_t seg_cap, int *overflow,
                          uint8_t *cnz, uint32_t *members, uint32_t *members_count, Bucket *buckets,
                          uint64_t *pair_counts, uint32_t *nbuckets, cudaStream_t s,
                          int64_t *launches, int part_max, uint32_t *work, unsigned long long *kept,
                          FilterArgs *defer = nullptr);
// Searches of one key class (fused_key_class of their M: 16, 24 or 32) in one
// persistent launch of `grid` CTAs of the largest filter CTA size (results
// do not depend on it): args as recorded by
// launch_filter with `defer` (one launch group each, B = 1, binary X); the
// CTAs take the work items of all of them, in order, from the zeroed
// counter `work`.  Every search's buffers must be sized for `grid` CTAs.
int fused_key_class(int M);
cudaError_t launch_filter_fused(const FilterArgs *args, int count, int key_class, int grid, uint32_t *work,
                                cudaStream_t s, int64_t *launches);
cudaError_t launch_seg_reset(uint32_t *seg_count, cudaStream_t s, int64_t *launches);
cudaError_t launch_compact(const uint64_t *seg_keys, const uint32_t *seg_vals,
                           const uint32_t *seg_count, uint32_t seg_cap, int nseg, uint64_t *out_keys,
                           uint32_t *out_vals, uint32_t *total, cudaStream_t s, int64_t *launches);

// Host-side helpers shared by the API files.
int64_t amin_rule(int64_t n, double kappa);

// Real response (weights.cu): fixed-point weights q, sign bits, bit planes,
// inclusive cdf and total of a device array of n doubles; maxbits / bad let
// the host reject a response that is all zero or not finite.
size_t weights_scan_bytes(int64_t n);
cudaError_t launch_prepare_weights(const double *dY, int64_t n, int64_t Wp, uint64_t *q, uint32_t *yb,
                                   uint32_t *planes, uint64_t *cdf, uint64_t *total,
                                   unsigned long long *maxbits, int *bad, void *scan_tmp, cudaStream_t s,
                                   int64_t *launches);
// sign transform of a real X (count entries) to -1 / +1, zeros by a fair coin
cudaError_t launch_sign_transform(const float *dX, int64_t count, uint64_t coin_seed, int8_t *out, int *bad,
                                  cudaStream_t s, int64_t *launches);
// Real X, unbiased transform (realx.cu).
cudaError_t launch_unbiased_scale(const float *dX, int64_t n, int64_t p, int64_t Pf, int64_t Wf, float *Xrs,
                                  float *Xcs, float *nu, unsigned *bad, cudaStream_t s, int64_t *launches);
cudaError_t launch_unbiased_y(const double *dY, const float *nu, int64_t n, int64_t Wf, double *yprime,
                              double *ysd, cudaStream_t s, int64_t *launches);
cudaError_t launch_verify_real(const Packed &pk, const Bucket *buckets, const uint64_t *pair_off,
                               const uint32_t *nbuckets, const uint64_t *total_pairs, const uint32_t *vals,
                               int kbits, uint64_t *rec_keys, uint32_t *rec_agree, uint32_t *nrec,
                               uint32_t rec_cap, cudaStream_t s, int64_t *launches, const int *abort_flag);
cudaError_t launch_real_strengths(const Packed &pk, PairOut *out, const uint32_t *nout, int64_t cap,
                                  cudaStream_t s, int64_t *launches);
// Y -> -Y on the response sign bits of the valid rows
cudaError_t launch_flip_signs(const Packed &pk, cudaStream_t s, int64_t *launches);
// weighted strengths (2 S - Q) / Q of the first *nout output pairs
cudaError_t launch_weighted_strengths(const Packed &pk, PairOut *out, const uint32_t *nout, int64_t cap,
                                      cudaStream_t s, int64_t *launches);

// Exhaustive screen (brute.cu): records (j << kbits | k, a) of every pair
// j < k with a >= amin; blocks = brute_tiles(p).
int64_t brute_tiles(int64_t p);
cudaError_t launch_brute(const Packed &pk, int64_t amin, int kbits, uint64_t *rec_keys,
                         uint32_t *rec_agree, uint32_t *nrec, uint32_t rec_cap, cudaStream_t s,
                         int64_t *launches);

}  // namespace xyz

struct xyz_ctx;

namespace xyz {
const Packed *ctx_packed(const xyz_ctx *c);
cudaStream_t ctx_stream(const xyz_ctx *c);
int ctx_device(const xyz_ctx *c);
int view_create(int device, xyz_ctx **out);
void view_target(xyz_ctx *view, const xyz_ctx *base, uint32_t *yb);
int64_t ctx_device_bytes(const xyz_ctx *c);
xyz_ctx *ctx_sizing_copy(const xyz_ctx *c);
void ctx_sizing_update(xyz_ctx *dst, const xyz_ctx *src);
void ctx_sizing_free(xyz_ctx *c);
int64_t ctx_slice_growth(const xyz_ctx *view, const xyz_ctx *base, int64_t runs, int M);
int pack_response(xyz_ctx *c, const int8_t *Y, uint32_t *yb_dev);

}  // namespace xyz
