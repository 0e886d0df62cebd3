/*
 * xyz.h -- C ABI of the GB300 binary xyz interaction search.
 *
 * The library finds column pairs (j, k) of a +-1 matrix X whose product
 * X_j o X_k has a large inner product with a +-1 response Y:
 *
 *     keep (j, k), j < k, with  Y^T (X_j o X_k) / n  >=  kappa
 *
 * (eq. 1 of Thanei, Meinshausen & Shah, "The xyz algorithm for fast
 * interaction search in high-dimensional data", with the >= of Algorithm 2
 * step 5), without screening all p(p-1)/2 pairs: it runs the final xyz
 * algorithm (Algorithm 2, Section 2.2) with minimal subsampling.  Every step
 * runs in CUDA kernels for sm_103a; the host code only validates, plans and
 * launches.
 *
 * Conventions used by every entry point
 *   - X is n x p, column-major, int8: X[j*n + i] = X_ij, each entry -1 or +1.
 *     Y has n int8 entries, each -1 or +1.  Indices are 0-based.
 *   - "Agreement" a_jk = #{ i : Y_i = X_ij X_ik }  (eq. def_gamma: the
 *     interaction strength is gamma_jk = a_jk / n and, by eq. equiv,
 *     Y^T(X_j o X_k)/n = 2 gamma_jk - 1 = (2 a_jk - n) / n).
 *   - kappa in [-1, 1]; a pair passes when (double)(2a - n) >= kappa * (double)n
 *     (one IEEE double multiply), i.e. a >= xyz_amin(n, kappa).
 *   - Row subsets: run l draws M rows i.i.d. uniform on {0..n-1} WITH
 *     replacement (eq. projR, subsampling class).  Draw number t = l*M + m of
 *     a search with seed s is u = splitmix64 output t from state s, i.e.
 *     mix(s + (t+1) * 0x9E3779B97F4A7C15) with the splitmix64 finaliser of
 *     Steele, Lea & Flood (2014), and the row is floor(u * n / 2^64).
 *   - A candidate of run l is an unordered pair j != k that agrees on every
 *     sampled row: X_{s j} = Y_s X_{s k} for all sampled s (the projection
 *     and equal-pairs steps of Algorithm 2; equality of the projections
 *     x_j = z_k happens exactly then, see the remark on minimal subsampling
 *     in Section 2).
 *   - Results are deterministic: they depend only on (X, Y, M, L, kappa,
 *     seed), never on tuning, chunking or batching.
 *
 * Errors: every int-returning call returns XYZ_OK (0) or one of the codes
 * below; on error no output is written and xyz_last_error() returns a
 * message (thread-local, valid until the next call on that thread).
 *
 * Ownership: the library copies what it needs from inputs before returning;
 * callers may free inputs immediately.  Arrays the library returns through
 * `**` out-parameters are allocated by it and released with xyz_free_pairs()
 * (or xyz_free() for non-pair arrays).  A context owns its device memory and
 * its CUDA stream and is not re-entrant: one thread at a time per context.
 */
#ifndef XYZ_H
#define XYZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define XYZ_OK 0
#define XYZ_EINVAL 1      /* bad argument: sizes, null pointer, entry not +-1, M, L, kappa */
#define XYZ_ENOMEM 2      /* host or device allocation failed, or over a memory budget */
#define XYZ_ECUDA 3       /* a CUDA call failed (the message names it) */
#define XYZ_ETIMEDOUT 4   /* a bounded wait gave up (device-side, or xyz_server_wait) */
#define XYZ_ECANCELED 5   /* a served request was cancelled */
#define XYZ_EAGAIN 6      /* a served request is not finished yet */

#define XYZ_MAX_M 64      /* keys hold one bit per sampled row */

typedef struct xyz_ctx xyz_ctx;

/* One reported interaction: columns j < k, agreement a_jk and the
 * kappa-scale strength (2 a_jk - n) / n = Y^T(X_j o X_k)/n (eq. equiv). */
typedef struct xyz_pair {
    int32_t j;
    int32_t k;
    int32_t agree;
    float strength;
} xyz_pair;

/* Counters of the last search on a context (observability only). */
typedef struct xyz_stats {
    int64_t runs;             /* runs executed */
    int64_t chunks;           /* launch groups the runs were split into */
    int64_t runs_per_chunk;   /* runs sorted together in one launch group */
    int64_t candidates;       /* sum over runs of |E_l| (unordered pairs) */
    int64_t buckets;          /* equal-key groups holding >= 1 candidate */
    int64_t passing;          /* verified pairs before the union over runs */
    int64_t unique_pairs;     /* |I| returned */
    int64_t sort_passes;      /* radix passes per launch group */
    int64_t key_bits;         /* bits sorted per launch group */
    int64_t gpu_launches;     /* kernels launched by the last call */
    double ms_keys;           /* device time per stage, summed over launches */
    double ms_sort;           /*   (filled only when timing is enabled) */
    double ms_join;
    double ms_verify;
    double ms_dedup;
    double ms_total;          /* device time from first to last kernel */
    int64_t launches_keys;    /* launches per stage */
    int64_t launches_sort;
    int64_t launches_join;
    int64_t launches_verify;
    int64_t launches_dedup;
    int64_t survivors;        /* entries that reached the sort (all of them without the filter) */
    int64_t filter_kept;      /* columns kept by the survivor filter, summed over runs (0 without it) */
    int64_t attempts;         /* 1, plus one for every redo after a buffer grew */
    int64_t bucket_members;   /* columns in buckets grouped on chip, summed over runs (spilled runs excluded) */
    int64_t segment_grouped_runs; /* runs past one on-chip grouping, grouped on chip from the segment
                                     in several passes (hash partitions or bins) instead of the sort */
} xyz_stats;

/* ---------------------------------------------------------------- context */

/* the form-Z step of Algorithm 2 ("form Z"): copy X and Y to the device and pack them
 * into bit columns (for verification), bit rows (for key building) and the
 * response bits; Z is never materialised (its bits are X's bits xor Y's).
 * X: host pointer, n*p int8, column-major.  Y: host pointer, n int8.
 * n >= 1, 2 <= p < 2^31, n < 2^31.  Any entry other than -1/+1 gives
 * XYZ_EINVAL.  On success *out owns all device state.  When both buffers
 * are page-locked host memory mapped into the device's address space (for
 * example cudaHostAlloc or torch's pin_memory), the pack kernel reads them
 * in place -- one pass over X, no staging copy; pageable buffers are copied
 * to the device first.  Either way X and Y are not referenced after return. */
int xyz_create(const int8_t *X, const int8_t *Y, int64_t n, int64_t p, xyz_ctx **out);

/* Same as xyz_create with X and Y already in device memory (e.g. torch
 * tensors).  `stream` is a cudaStream_t (NULL: the library makes its own);
 * all later work of the context is ordered on it.  The caller keeps
 * ownership of dX/dY, which are not referenced after return. */
int xyz_create_dev(const int8_t *dX, const int8_t *dY, int64_t n, int64_t p, void *stream,
                   xyz_ctx **out);

/* Real-valued X by the sign transform of Section 3.2: X~_ij = sgn(X_ij),
 * an entry that is exactly 0 getting a fair coin (the top bit of splitmix64
 * output j*n + i from state coin_seed, so the transform is reproducible).
 * X: n x p column-major float (copied before the call returns); NaN gives
 * XYZ_EINVAL.  The context holds the binary X~ and the response +1 until
 * xyz_set_y / xyz_set_y_real; with a real Y the search computes the
 * sign-transform strength of Section 3.2,
 * 1/2 + sum_i Y_i sgn(X_ij) sgn(X_ik) / (2 ||Y||_1). */
int xyz_create_sign(const float *X, int64_t n, int64_t p, uint64_t coin_seed, xyz_ctx **out);

/* Real-valued X by the unbiased transform of Section 3.2.  Rows are scaled,
 * nu_i = max_j |X_ij|, X'_ij = X_ij / nu_i (float; a row of zeros stays 0),
 * Y'_i = Y_i nu_i^2, and the search draws rows with probability
 * |Y'_i| / ||Y'||_1 (fixed point as xyz_set_y_real), binarises every drawn
 * entry afresh with P(X~ = +1) = (X'_ij + 1)/2 (u24 < (X' + 1)/2 * 2^24, u24
 * the top 24 bits of splitmix64 output (l M + m) p + j from state
 * seed + 0x632BE59BD9B4E019), and keeps a candidate when the real inner
 * product sum_i Y'_i X'_ij X'_ik (float, eight partial sums per candidate)
 * is >= kappa ||Y'||_1 -- by the proposition on the unbiased transform its
 * strength gamma^g_jk >= (1 + kappa)/2.  Results: agree = -1, strength =
 * sum_i Y'_i X'_ij X'_ik / ||Y'||_1.  X: n x p column-major float, Y: n
 * doubles (copied; NaN in X or an unusable Y' gives XYZ_EINVAL).  Searches
 * need M <= 31 and p <= 262144; a new response goes through xyz_set_y_real
 * (which scales it); binary responses, batched search, the exhaustive screen,
 * xyz_search_abs and xyz_kkt_screen are XYZ_EINVAL on such a context. */
int xyz_create_unbiased(const float *X, const double *Y, int64_t n, int64_t p, xyz_ctx **out);

/* Replace the response Y (host pointer, n int8) of an existing context,
 * keeping packed X resident (Section 4 calls xyz repeatedly on one X with
 * changing responses). */
int xyz_set_y(xyz_ctx *ctx, const int8_t *Y);

/* xyz_set_y with Y in device memory. */
int xyz_set_y_dev(xyz_ctx *ctx, const int8_t *dY);

/* Real-valued response (Section 3.1, continuous Y with binary X): the rows
 * of a run are drawn with probability |Y_i| / ||Y||_1, Z = sgn(Y) o X
 * (sgn(0) = +1), and a candidate passes when Y^T(X_j o X_k) >= kappa ||Y||_1,
 * i.e. its |Y|-weighted agreement gamma~_jk >= (1 + kappa)/2.  The weights
 * are used in fixed point, exactly on every step: with max|Y_i| = f 2^e
 * (f in [0.5, 1)), q_i = floor(|Y_i| 2^(24-e) + 1/2) and Q = sum q_i; the
 * weighted draw t is the least i with q_0 + ... + q_i > floor(u Q / 2^64),
 * u the splitmix64 output t; a pair passes when (double)(2 S - Q) >=
 * kappa * (double)Q with S the weight sum of the rows where
 * sgn(Y_i) = X_ij X_ik.  Results report agree = the count of those rows and
 * strength = (2 S - Q) / Q.  Y: n doubles, finite, not all zero (else
 * XYZ_EINVAL, context unchanged).  The context stays in this mode until the
 * next xyz_set_y(_dev).  Batched search and the exhaustive screen take
 * binary responses only (XYZ_EINVAL in this mode). */
int xyz_set_y_real(xyz_ctx *ctx, const double *Y);
int xyz_set_y_real_dev(xyz_ctx *ctx, const double *dY);

/* Release a context and its device memory.  NULL is ignored. */
void xyz_destroy(xyz_ctx *ctx);

/* Message of the last failed call on this thread ("" if none). */
const char *xyz_last_error(void);

/* n, p and the device bytes held by the context. */
int xyz_info(const xyz_ctx *ctx, int64_t *n, int64_t *p, int64_t *device_bytes);

/* ----------------------------------------------------------------- search */

/* Algorithm 2 (final xyz): for runs l = 0..L-1 draw M rows, hash every
 * column of X and Z to its M sampled bits, group equal keys (Section 2.2,
 * equal-pairs search by sorting, Figure 2), verify each candidate exactly
 * and keep it when a_jk >= xyz_amin(n, kappa); return the union over runs.
 * L >= 1, 0 <= M <= 64, kappa finite in [-1, 1].  M = 0 makes every pair a
 * candidate (the brute-force search).  *pairs gets *npairs records sorted by
 * (j, k), each pair once; free with xyz_free_pairs (NULL when *npairs = 0). */
int xyz_search(xyz_ctx *ctx, int32_t L, int32_t M, double kappa, uint64_t seed,
               xyz_pair **pairs, int64_t *npairs);

/* Runs [l0, l1) of the search above (same seed stream), for sharding runs
 * across devices or processes: the union of the results of disjoint ranges
 * covering [0, L) equals xyz_search(L).  0 <= l0 < l1. */
int xyz_search_range(xyz_ctx *ctx, int64_t l0, int64_t l1, int32_t M, double kappa,
                     uint64_t seed, xyz_pair **pairs, int64_t *npairs);

/* Batched search (many responses on one resident X, as Section 4's repeated
 * calls with changing responses need): for each of B responses (Ys: host
 * array of B rows of n int8, row b = response b) the same search as
 * xyz_search(L, M, kappa, seed) with that response.  All responses share the
 * row stream, so each run's keys of X are built once.  *pairs gets all
 * results, response b's at [offsets[b], offsets[b+1]) sorted by (j, k);
 * offsets: caller array of B + 1.  Results are identical to B separate
 * searches.  B >= 1; other arguments as xyz_search. */
int xyz_search_batch(xyz_ctx *ctx, const int8_t *Ys, int32_t B, int32_t L, int32_t M, double kappa,
                     uint64_t seed, xyz_pair **pairs, int64_t *offsets);

/* xyz_search_batch with the responses in device memory. */
int xyz_search_batch_dev(xyz_ctx *ctx, const int8_t *dYs, int32_t B, int32_t L, int32_t M,
                         double kappa, uint64_t seed, xyz_pair **pairs, int64_t *offsets);

/* Absolute-value search: the pairs with |Y^T(X_j o X_k)| / n >= kappa
 * (|.| / ||Y||_1 for a real response), found as Section 4 does, by running
 * the search with Y and with -Y (same rows, same seed) and uniting the two
 * results.  Pairs are reported for +Y: agree counts the rows agreeing with
 * Y and strength is signed (negative for the pairs found through -Y).  Each
 * pair once, sorted by (j, k).  Arguments and errors as xyz_search. */
int xyz_search_abs(xyz_ctx *ctx, int32_t L, int32_t M, double kappa, uint64_t seed, xyz_pair **pairs,
                   int64_t *npairs);

/* The interaction half of the KKT check of the Lasso active-set strategy
 * (Section 4, the KKT check of Algorithm 3): with a real residual r (n doubles, e.g.
 * Y - X_A beta_A - W_B theta_B, centred), the pairs with
 * |r^T (X_j o X_k)| / n > lambda, searched with Y set to +r and to -r.  The
 * context switches to the real response r (as xyz_set_y_real).  In the
 * fixed-point form of xyz_set_y_real the test is |2 S - Q| >= t with
 * t = floor(lambda * n * 2^(24 - e)) + 1.  Results: agree as for +r, and
 * strength = r^T (X_j o X_k) / n from the fixed-point weights (signed).
 * lambda >= 0 and finite, else XYZ_EINVAL. */
int xyz_kkt_screen(xyz_ctx *ctx, const double *r, double lambda, int32_t L, int32_t M, uint64_t seed,
                   xyz_pair **pairs, int64_t *npairs);

/* Operating-point autotuner: eq. bestM chooses M from the paper's cost model
 * (Section 2.3); this measures this implementation's cost instead.  For
 * each M in [M_lo, M_hi] it takes L = xyz_runs_for_recall(gamma^M, recall)
 * (eq. L_choice), times two short searches on the device (trial_runs and a
 * quarter of it; CUDA events on the context's stream), fits time = a + b*runs
 * and predicts the full search.  With a table, the two best predictions
 * (when under 200 ms) are then timed as full searches and the faster one
 * wins.  *M_best / *L_best / *ms_best get the chosen point.  table
 * (optional, 3*(M_hi - M_lo + 1) doubles) gets (M, L, ms) rows: measured for
 * the confirmed points, predicted for the rest, < 0 where L is out of range.  Searches on the context's data;
 * results of later searches never depend on it.  0 < gamma < 1,
 * 0 < recall < 1, 1 <= M_lo <= M_hi <= 64, trial_runs >= 8, else XYZ_EINVAL. */
int xyz_autotune_M(xyz_ctx *ctx, double kappa, double gamma, double recall, int32_t M_lo, int32_t M_hi,
                   uint64_t seed, int64_t trial_runs, int32_t *M_best, int64_t *L_best, double *ms_best,
                   double *table);

/* Launch shapes of the search on the survivor-filter path (no counterpart
 * in the paper).  Results never depend on them. */
typedef struct xyz_tiles {
    int32_t filter_threads;        /* threads per filter CTA: a multiple of 32 in [512, 1024];
                                      0 = chosen from p (least waste in the last round) */
    int32_t verify_blocks_per_sm;  /* verification blocks per SM, 1 or more; 0 = as many as fit */
    int64_t group_runs;            /* runs per launch group, 1 or more; 0 = the default rule */
} xyz_tiles;

/* Sets the launch shapes of later searches on ctx (XYZ_EINVAL for values
 * out of range; all zero restores the defaults). */
int xyz_set_tiles(xyz_ctx *ctx, const xyz_tiles *tiles);

/* Picks the launch shapes by measurement, one after another: the filter's
 * CTA size among {default, 640, 768, 896, 1024}, then the launch-group size
 * among {default, 1/2, 1/4 of it} (at least 2 runs per SM), then the
 * verification's blocks per SM among {as many as fit, 2, 1}; each candidate
 * is timed (CUDA events) on a search of trial_runs runs with (M, kappa) after
 * one warm-up search.  The best shapes are set on ctx and returned in *best,
 * with their time in *ms_best.  trial_runs >= 8, kappa finite in [-1, 1],
 * 0 <= M <= 31 (the filter path), else XYZ_EINVAL. */
int xyz_autotune_tiles(xyz_ctx *ctx, int32_t M, double kappa, uint64_t seed, int64_t trial_runs, xyz_tiles *best,
                       double *ms_best);

/* Many independent searches at once, each on its own context (instances of
 * different n and p): search i is xyz_search(ctxs[i], L[i], M[i],
 * kappa[i], seed[i]) and its result is identical to that call.  The launch
 * groups of all searches are captured into one CUDA graph, forked over the
 * contexts' streams so that they run concurrently, and launched once; the
 * searches of one launch group on the single-filter path share one
 * persistent filter launch per key class (xyz_set_fused_filter).  Each
 * search then finishes (spilled runs, union) on its own stream.  Results go
 * to one array: search i owns (*pairs)[offsets[i] .. offsets[i+1]); offsets
 * has count + 1 entries.  Contexts must be distinct, on one device, with
 * their own streams (XYZ_EINVAL otherwise). */
int xyz_search_many(xyz_ctx **ctxs, int32_t count, const int32_t *L, const int32_t *M, const double *kappa,
                    const uint64_t *seed, xyz_pair **pairs, int64_t *offsets);

/* Exhaustive screen: every pair j < k with (2a - n) >= kappa*n, i.e. I* of
 * eq. 1 under the >= reading -- the comparator the search is measured
 * against and the M = 0 case of Algorithm 2 (one empty key, every pair a
 * candidate).  O(p^2 n / 32) word operations on the GPU (a tiled popcount
 * over the packed columns); output as xyz_search. */
int xyz_brute_force(xyz_ctx *ctx, double kappa, xyz_pair **pairs, int64_t *npairs);

void xyz_free_pairs(xyz_pair *pairs);
void xyz_free(void *ptr);

/* Counters (and, with timing on, per-stage device times) of the last search. */
int xyz_get_stats(const xyz_ctx *ctx, xyz_stats *out);

/* Record CUDA events around every stage of later searches (0 = off). */
int xyz_set_timing(xyz_ctx *ctx, int enable);

/* Tuning: at most `entries` sorted keys (runs x p) per launch group; one run
 * per group when entries < p.  The filter path, which sorts only a few
 * percent of the columns, puts up to 64 x entries / p runs (at most 16384)
 * in a group.  Results never depend on it.  Default 2^25. */
int xyz_set_chunk_entries(xyz_ctx *ctx, int64_t entries);

/* Tuning: 1 (default) lets searches drop, per run, the columns that cannot
 * be in any candidate pair before grouping: with one shared-memory filter
 * of the run's keys when M <= 31 and p <= 262144, and otherwise -- one
 * binary response, M <= 28, p <= 2^27 -- with the keys split into 16
 * linear classes, one filter per class in turn.  2 uses the class-split
 * form wherever it applies (also at small p); 0 groups every column.
 * XYZ_EINVAL for other values.  Results never depend on it. */
int xyz_set_filter(xyz_ctx *ctx, int enable);

/* Tuning (filter path): runs whose survivors do not fit on chip are grouped
 * through a sort, once per `groups` launch groups (0, the default: once per
 * search; the library lowers it by itself when the spill buffers would pass
 * about 2^27 entries).  groups >= 0.  Results never depend on it. */
int xyz_set_spill_flush(xyz_ctx *ctx, int64_t groups);

/* Tuning (filter path): a run with more survivors than one on-chip grouping
 * holds is grouped on chip in up to max_parts passes, each over the
 * survivors whose group key hashes into one range of 32 bins (a group never
 * straddles two); a run that needs more passes, or has a single bin above
 * the capacity, goes through the sort as above.  The class-split filter
 * (p > 262144, or xyz_set_filter(ctx, 2)) instead sorts a run's survivors by
 * bin once and groups every bin on chip -- a bin above the capacity from
 * global memory, when its distinct group keys fit the on-chip table -- so
 * there only 0 versus nonzero matters.  0 sends every such run to the sort.
 * 0 <= max_parts <= 32, default 32.  Results never depend on it. */
int xyz_set_onchip_partitions(xyz_ctx *ctx, int32_t max_parts);

/* Tuning (xyz_search_many): 1 (default) lets this context's search share a
 * fused filter launch with the other searches of the call -- one persistent
 * grid whose CTAs take the runs of all of them from one counter -- when the
 * search is one launch group on the single-filter path (M <= 31,
 * p <= 262144, binary X; at most 64 searches per launch, one launch per key
 * class M <= 16, <= 24, <= 31).  0 keeps its filter a launch of its own.
 * XYZ_EINVAL for other values.  Results never depend on it. */
int xyz_set_fused_filter(xyz_ctx *ctx, int enable);

/* --------------------------------------------------- parity / observability */

/* Keys of run `run` (the projection step of Algorithm 2 with the integer reading of the
 * projection): kx[j] = sum_m bit(X_{s_m j}) 2^m with bit(v) = 1 iff v = -1,
 * for j < p, and c = sum_m bit(Y_{s_m}) 2^m, so that the Z-key of column k is
 * kx[k] xor c.  kx: host array of p uint64; c: host pointer. */
int xyz_run_keys(xyz_ctx *ctx, int32_t M, uint64_t seed, int64_t run, uint64_t *kx, uint64_t *c);

/* Candidate set E_run (the equal-pairs step of Algorithm 2) as unordered pairs j < k,
 * sorted; *jk gets 2*count int32 (j0,k0,j1,k1,...), free with xyz_free. */
int xyz_run_candidates(xyz_ctx *ctx, int32_t M, uint64_t seed, int64_t run, int32_t **jk,
                       int64_t *count);

/* Exact agreement a_jk (eq. def_gamma) of `count` given pairs, computed on
 * the device by popcount over the packed columns.  j, k, agree: host arrays
 * of `count` int32; 0 <= j, k < p. */
int xyz_agree(xyz_ctx *ctx, const int32_t *j, const int32_t *k, int64_t count, int32_t *agree);

/* Agreement of `count` pairs drawn uniformly among all unordered pairs j != k
 * (splitmix64 stream of `seed`), for the plug-in estimate of
 * sum_{j,k} gamma_jk^M in eq. bestM.  j_out, k_out, agree: host arrays. */
int xyz_sample_agree(xyz_ctx *ctx, int64_t count, uint64_t seed, int32_t *j_out, int32_t *k_out,
                     int32_t *agree);

/* ---------------------------------------------------- planner (host only) */

/* Least agreement count that passes kappa (n + 1 when none can). */
int64_t xyz_amin(int64_t n, double kappa);

/* eq. eta: probability that a pair of strength gamma (in [0,1]) is found in
 * L runs of M rows: 1 - (1 - gamma^M)^L. */
double xyz_eta(double gamma, int32_t M, int64_t L);

/* eq. L_choice: least L with 1 - (1 - beta)^L >= eta, where beta is the
 * single-run retention probability (gamma^M for minimal subsampling).
 * Returns -1 for beta <= 0 or eta outside (0, 1). */
int64_t xyz_runs_for_recall(double beta, double eta);

/* eq. bestM with the plug-in estimate of Section 2.3: minimise over
 * M = 1..max_M the cost  -(M p + p log p + n S(M)) / log(1 - gamma^M),
 * where S(M) = sum_{j != k} gamma_jk^M is estimated as p(p-1) times the mean
 * of (agree/n)^M over `count` sampled pairs.  Writes the minimiser to *M_out
 * and the minimum to *cost_out (may be NULL).  gamma in (0, 1). */
int xyz_best_M(int64_t n, int64_t p, double gamma, const int32_t *agree, int64_t count,
               int32_t max_M, int32_t *M_out, double *cost_out);

/* M with gamma_0 = p^(-1/M) closest to gamma0 (Section 5.2 sets gamma_0
 * near 0.55): round(log p / log(1/gamma0)), at least 1. */
int32_t xyz_M_for_gamma0(int64_t p, double gamma0);

/* ------------------------------------------------------ measured peaks */

/* Throughputs of the instruction classes the integer kernels are made of,
 * measured on the current device (the paper has no counterpart: these are
 * the denominators of the rooflines reported for this implementation). */
typedef struct xyz_peaks {
    double alu_ops_per_s;     /* lop3.b32 (integer ALU pipe: logic, shifts, byte permutes) */
    double iadd_ops_per_s;    /* add.u32 */
    double popc_ops_per_s;    /* popc.b32 */
    double sm_mhz;            /* mean SM clock during the probes (clock64 cycles / elapsed time) */
    int32_t sms;              /* streaming multiprocessors */
} xyz_peaks;

/* Runs the three probes on the current device: per SM 1024 threads with 8
 * independent chains of one instruction each, about 1-2 ms per launch, timed
 * with CUDA events on the default stream (each probe's second launch is the
 * measured one).  Allocates a few KB of device memory for the duration of
 * the call.  XYZ_EINVAL for a null pointer, XYZ_ECUDA on a CUDA error. */
int xyz_probe_peaks(xyz_peaks *out);

/* --------------------------------------- allocation-free candidate set */

/* Limits of xyz_run_candidates_noalloc. */
#define XYZ_NOALLOC_MAX_P 16384      /* columns of X */
#define XYZ_NOALLOC_MAX_PAIRS 32768  /* candidates of the requested run */

/* The paper has no counterpart to this entry point.  It returns the same
 * candidate set as xyz_run_candidates, for callers that cannot allocate
 * device memory at the time they ask (their device memory is owned by another
 * allocator, or they cannot afford cudaMalloc's device-wide synchronisation).
 * It allocates nothing: its scratch is a fixed array inside the library of
 * about 2.3 MB that every GPU which loads the library keeps until the process
 * exits.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with the context's device current), so make the first
 * call before beginning any stream capture on that device.  Calls share the
 * array: calls that overlap on the GPU race and must be serialised.  The
 * cached address is that of the device's primary context: after a
 * cudaDeviceReset of the device, do not call this entry point on it again in
 * the same process.  The caller's current device is restored on return.
 * Binary and real-valued (xyz_set_y_real) responses are taken, whatever
 * search ran on the context before; contexts of real X built by
 * xyz_create_unbiased are refused (XYZ_EINVAL).
 * ctx: a context with p <= XYZ_NOALLOC_MAX_P (else XYZ_EINVAL).  jk: host array
 * of 2*cap int32 that receives the pairs (j0,k0,j1,k1,...), j < k, sorted;
 * *count gets their number.  A run with more than XYZ_NOALLOC_MAX_PAIRS or
 * more than cap candidates gives XYZ_ENOMEM and writes nothing. */
int xyz_run_candidates_noalloc(xyz_ctx *ctx, int32_t M, uint64_t seed, int64_t run, int32_t *jk,
                               int64_t cap, int64_t *count);

/* ------------------------------------------------------------- server */

/* A search server: the search as a request loop.  The paper screens one X
 * against several responses (the scaling experiment of Section 5.2 builds
 * responses of strength 0.7, 0.8 and 0.9 for each X); here each such search
 * is a request.  Datasets (packed X and a
 * default response) stay resident on the device; requests carry their own
 * response, L, M, kappa and seed.  Requests are admitted in arrival order
 * while the device memory in use stays within hbm_budget_bytes: the
 * resident datasets, the workers' workspaces as measured after their last
 * slice, and for each admitted request a reservation sized at admission --
 * its packed response (when it has its own) plus the growth its slices may
 * cause in every worker's workspace, by the library's own workspace sizing
 * for a search of slice_runs runs at the request's M (buffers that a search
 * grows on overflow count at their starting size).  The others wait (the
 * oldest waiting request is admitted whenever nothing is running, so none
 * waits forever).  Admitted requests are cut into slices of slice_runs runs,
 * and `workers` threads -- each with its own CUDA stream and workspace --
 * take slices round-robin over all admitted requests (continuous batching
 * at run granularity).  Each slice is a search over its run range, whose
 * results are deduplicated and sorted on the device; a request's result is
 * the merge of its slices' sorted results, each pair once, which equals
 * xyz_search(L, M, kappa, seed) on its (X, Y) exactly, whatever else is
 * being served.  All xyz_server_* calls are thread-safe. */
typedef struct xyz_server xyz_server;

typedef struct xyz_server_stats {
    int64_t completed;        /* requests finished with a result */
    int64_t canceled;         /* requests cancelled */
    int64_t failed;           /* requests that ended with an error */
    int64_t queued;           /* waiting for admission now */
    int64_t active;           /* admitted, not finished, now */
    int64_t device_bytes;     /* device memory counted against the budget now */
    int64_t budget_bytes;     /* the budget */
    double p50_ms;            /* median submit-to-finish latency of completed requests */
    double p99_ms;            /* 99th percentile of the same (linear interpolation) */
    double pairs_screened;    /* sum of p(p-1)/2 over completed requests */
    double elapsed_ms;        /* first submit to last completion */
} xyz_server_stats;

/* workers in [1, 64]; hbm_budget_bytes > 0; slice_runs >= 1.  Uses the
 * current CUDA device. */
int xyz_server_create(int32_t workers, int64_t hbm_budget_bytes, int64_t slice_runs, xyz_server **out);
/* Make X (and default response Y) resident; same layout and checks as
 * xyz_create.  XYZ_ENOMEM when the datasets would exceed the budget. */
int xyz_server_add_dataset(xyz_server *srv, const int8_t *X, const int8_t *Y, int64_t n, int64_t p,
                           int32_t *dataset);
/* Queue a search of `dataset` with response Y (n int8 +-1, copied before the
 * call returns; NULL = the dataset's default response).  *request gets an id
 * for wait/poll/cancel. */
int xyz_server_submit(xyz_server *srv, int32_t dataset, const int8_t *Y, int32_t L, int32_t M,
                      double kappa, uint64_t seed, int64_t *request);
/* Block until the request ends or timeout_ms passes (< 0: no limit).  On
 * XYZ_OK the request is retired and *pairs / *npairs / *latency_ms get its
 * result (sorted by (j, k), free with xyz_free_pairs) and its submit-to-finish
 * time; XYZ_ETIMEDOUT leaves it running; XYZ_ECANCELED / an error code retire
 * it. */
int xyz_server_wait(xyz_server *srv, int64_t request, int64_t timeout_ms, xyz_pair **pairs,
                    int64_t *npairs, double *latency_ms);
/* As xyz_server_wait with no waiting: XYZ_EAGAIN while the request runs. */
int xyz_server_poll(xyz_server *srv, int64_t request, xyz_pair **pairs, int64_t *npairs,
                    double *latency_ms);
/* Cancel a queued or running request (slices already on the GPU finish;
 * no new ones start).  Its wait/poll then returns XYZ_ECANCELED. */
int xyz_server_cancel(xyz_server *srv, int64_t request);
int xyz_server_get_stats(xyz_server *srv, xyz_server_stats *out);
/* Stops the workers after their current slice and frees everything. */
void xyz_server_destroy(xyz_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* XYZ_H */
