/*
 * Plain CPU oracle for the binary xyz interaction search
 * (Thanei, Meinshausen & Shah, "The xyz algorithm for fast interaction
 * search in high-dimensional data", Section 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library calls this file.  It is
 * loaded by the tests, by __graft_entry__.smoke() and by the CPU-baseline leg
 * of bench.py, and by nothing else.  It shares no code, header, table or
 * helper with the CUDA path; the only thing the two sides have in common is
 * the seeded synthetic input they are handed.
 *
 * Everything is written for clarity, not speed: int8 loops over the +-1
 * data, qsort for the equal-pairs search, one run at a time.
 *
 * Data convention (both sides): X is n x p, column-major int8
 * (X[j*n + i] = X_ij, entries -1 or +1); Y is n int8 entries -1 or +1.
 * Column and row indices are 0-based.
 *
 * Readings of the paper taken here (where it is silent or ambiguous):
 *   R1  rows of a run are drawn i.i.d. uniform on {0..n-1} WITH replacement
 *       (subsampling with replacement, Section 2, eq. projR and class (b);
 *       the retention probability gamma^M of Section 2.3 holds exactly only
 *       with replacement).
 *   R2  the random stream is a counter-based splitmix64 (Steele, Lea & Flood
 *       2014): draw t of a search with seed s is mix(s + (t+1)*0x9E3779B97F4A7C15)
 *       with t = run*M + m, and the row is floor(u * n / 2^64).
 *   R3  the projection R of eq. projR with F = U[0,1] (Algorithm 2's projection of the sampled rows)
 *       makes x_j = z_k exactly when X_{i_m j} = Z_{i_m k} for every sampled
 *       row (Section 2, the remark after the definition of the classes);
 *       keys are therefore the M sampled bits, bit(v) = 1 iff v = -1.
 *       orc_project_real() computes the paper's real projection as well, so
 *       the tests can check that both give the same equal pairs.
 *   R4  the diagonal j = k is not an interaction; candidates are reported as
 *       unordered pairs j < k (the model of eq. inter_mod sums over j < k).
 *   R5  the verification keeps gamma_jk >= gamma (Algorithm 2's check of the equal pairs), in
 *       kappa form: keep (2a - n) >= kappa*n, with a the agreement count of
 *       eq. def_gamma.  a_min is the least integer a in [0, n] with
 *       (double)(2a - n) >= kappa * (double)n (one IEEE double multiply).
 *   R6  the output of a search is the union over runs, each pair once,
 *       sorted by (j, k), with its exact integer agreement count.
 *
 * Parity unpinned: the splitmix64 row stream beyond its published first
 * outputs is a project convention; it is pinned only by agreement with the
 * CUDA path.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- stream */

/* splitmix64 output function (Steele, Lea & Flood 2014): finaliser applied to
 * a Weyl sequence with increment 0x9E3779B97F4A7C15. */
static uint64_t orc_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output number t (0-based) of the splitmix64 generator started at state
 * `seed`: the state after t+1 increments, finalised. */
uint64_t orc_splitmix64_at(uint64_t seed, uint64_t t)
{
    return orc_mix64(seed + (t + 1) * 0x9E3779B97F4A7C15ULL);
}

/* Reading R1/R2: the M row indices i_1..i_M of run `run`, i.i.d. uniform on
 * {0..n-1} with replacement (eq. projR, subsampling class). */
void orc_draw_rows(uint64_t seed, int64_t run, int32_t M, int64_t n,
                   int64_t *rows)
{
    for (int32_t m = 0; m < M; m++) {
        uint64_t u = orc_splitmix64_at(seed, (uint64_t)run * (uint64_t)M + (uint64_t)m);
        unsigned __int128 prod = (unsigned __int128)u * (unsigned __int128)(uint64_t)n;
        rows[m] = (int64_t)(uint64_t)(prod >> 64);
    }
}

/* ------------------------------------------------------------- strengths */

/* eq. def_gamma: a_jk = sum_i 1{Y_i = X_ij X_ik}; gamma_jk = a_jk / n. */
int64_t orc_agree(const int8_t *X, const int8_t *Y, int64_t n,
                  int64_t j, int64_t k)
{
    int64_t a = 0;
    for (int64_t i = 0; i < n; i++) {
        int prod = (int)X[j * n + i] * (int)X[k * n + i];
        if ((int)Y[i] == prod)
            a++;
    }
    return a;
}

/* a_jk for `count` given pairs (j[t], k[t]), one by one. */
void orc_agree_pairs(const int8_t *X, const int8_t *Y, int64_t n, const int32_t *j,
                     const int32_t *k, int64_t count, int32_t *out)
{
    for (int64_t t = 0; t < count; t++)
        out[t] = (int32_t)orc_agree(X, Y, n, j[t], k[t]);
}

/* Reading R5: least a in [0, n] with (double)(2a - n) >= kappa * (double)n;
 * n + 1 when no a qualifies (then nothing passes). */
int64_t orc_amin(int64_t n, double kappa)
{
    double rhs = kappa * (double)n;
    for (int64_t a = 0; a <= n; a++) {
        if ((double)(2 * a - n) >= rhs)
            return a;
    }
    return n + 1;
}

/* Input check shared by the entry points below: entries must be -1 or +1. */
int orc_check_pm1(const int8_t *v, int64_t count)
{
    for (int64_t i = 0; i < count; i++)
        if (v[i] != 1 && v[i] != -1)
            return 0;
    return 1;
}

/* eq. inter_search1 with the >= reading (R5): every pair j < k with
 * a_jk >= a_min, by looping over all p(p-1)/2 pairs (the naive O(np^2)
 * search of the Introduction).  Writes up to `cap` triples (j, k, a) and
 * returns how many pairs qualify. */
int64_t orc_brute_force(const int8_t *X, const int8_t *Y, int64_t n, int64_t p,
                        double kappa, int32_t *out, int64_t cap)
{
    int64_t amin = orc_amin(n, kappa);
    int64_t cnt = 0;
    for (int64_t j = 0; j < p; j++) {
        for (int64_t k = j + 1; k < p; k++) {
            int64_t a = orc_agree(X, Y, n, j, k);
            if (a >= amin) {
                if (cnt < cap) {
                    out[3 * cnt + 0] = (int32_t)j;
                    out[3 * cnt + 1] = (int32_t)k;
                    out[3 * cnt + 2] = (int32_t)a;
                }
                cnt++;
            }
        }
    }
    return cnt;
}

/* ------------------------------------------------------------ projection */

/* Reading R3: x_j = sum_m 2^m bit(X_{i_m j}), z_k = sum_m 2^m bit(Z_{i_m k})
 * with Z_ik = Y_i X_ik (Algorithm 2's product of Y with X) and bit(v) = 1 iff v = -1.
 * Two columns get equal keys exactly when they agree on every sampled row. */
void orc_keys(const int8_t *X, const int8_t *Y, int64_t n, int64_t p,
              const int64_t *rows, int32_t M, uint64_t *x, uint64_t *z)
{
    for (int64_t j = 0; j < p; j++) {
        uint64_t kx = 0, kz = 0;
        for (int32_t m = 0; m < M; m++) {
            int64_t i = rows[m];
            int xv = X[j * n + i];
            int zv = (int)Y[i] * xv;
            if (xv == -1)
                kx |= (uint64_t)1 << m;
            if (zv == -1)
                kz |= (uint64_t)1 << m;
        }
        x[j] = kx;
        z[j] = kz;
    }
}

/* The paper's own projection (eq. projR, the projection step of Algorithm 2):
 * R_i = sum_m D_m 1{i_m = i}, x = X^T R, z = Z^T R, in double precision.
 * D holds the M weights (drawn from U[0,1] by the caller). */
void orc_project_real(const int8_t *X, const int8_t *Y, int64_t n, int64_t p,
                      const int64_t *rows, int32_t M, const double *D,
                      double *x, double *z)
{
    double *R = (double *)calloc((size_t)n, sizeof(double));
    for (int32_t m = 0; m < M; m++)
        R[rows[m]] += D[m];
    for (int64_t j = 0; j < p; j++) {
        double sx = 0.0, sz = 0.0;
        for (int64_t i = 0; i < n; i++) {
            if (R[i] == 0.0)
                continue;
            sx += (double)X[j * n + i] * R[i];
            sz += (double)((int)Y[i] * (int)X[j * n + i]) * R[i];
        }
        x[j] = sx;
        z[j] = sz;
    }
    free(R);
}

/* --------------------------------------------------- equal-pairs search */

/* One point of the concatenation (x, z) in R^{2p}: its value, its colour
 * (0 = from x, 1 = from z) and its index. */
typedef struct {
    uint64_t v;
    int32_t colour;
    int32_t idx;
} orc_point;

static int orc_point_cmp(const void *pa, const void *pb)
{
    const orc_point *a = (const orc_point *)pa, *b = (const orc_point *)pb;
    if (a->v != b->v)
        return a->v < b->v ? -1 : 1;
    if (a->colour != b->colour)
        return a->colour - b->colour;
    return a->idx - b->idx;
}

typedef struct {
    double v;
    int32_t colour;
    int32_t idx;
} orc_rpoint;

static int orc_rpoint_cmp(const void *pa, const void *pb)
{
    const orc_rpoint *a = (const orc_rpoint *)pa, *b = (const orc_rpoint *)pb;
    if (a->v != b->v)
        return a->v < b->v ? -1 : 1;
    if (a->colour != b->colour)
        return a->colour - b->colour;
    return a->idx - b->idx;
}

/* the equal-pairs step of Algorithm 2 by the procedure of Section 2.2 (Figure 2): sort the 2p
 * values of (x, z), walk the distinct values, and wherever both colours are
 * present record the Cartesian product {j : x_j = v} x {k : z_k = v}.
 * Writes up to `cap` ORDERED pairs (j, k) with x_j = z_k (the diagonal
 * included) and returns their number. */
int64_t orc_equal_pairs(const uint64_t *x, const uint64_t *z, int64_t p,
                        int32_t *out, int64_t cap)
{
    orc_point *pts = (orc_point *)malloc((size_t)(2 * p) * sizeof(orc_point));
    for (int64_t j = 0; j < p; j++) {
        pts[j].v = x[j];
        pts[j].colour = 0;
        pts[j].idx = (int32_t)j;
        pts[p + j].v = z[j];
        pts[p + j].colour = 1;
        pts[p + j].idx = (int32_t)j;
    }
    qsort(pts, (size_t)(2 * p), sizeof(orc_point), orc_point_cmp);
    int64_t cnt = 0;
    int64_t s = 0;
    while (s < 2 * p) {
        int64_t e = s;
        while (e < 2 * p && pts[e].v == pts[s].v)
            e++;
        /* points [s, e) share one value; x-colour first (sort order) */
        int64_t mid = s;
        while (mid < e && pts[mid].colour == 0)
            mid++;
        for (int64_t a = s; a < mid; a++) {
            for (int64_t b = mid; b < e; b++) {
                if (cnt < cap) {
                    out[2 * cnt + 0] = pts[a].idx;
                    out[2 * cnt + 1] = pts[b].idx;
                }
                cnt++;
            }
        }
        s = e;
    }
    free(pts);
    return cnt;
}

/* The same walk over the paper's real-valued projections, with exact
 * floating-point equality as in the equal-pairs step of Algorithm 2. */
int64_t orc_equal_pairs_real(const double *x, const double *z, int64_t p,
                             int32_t *out, int64_t cap)
{
    orc_rpoint *pts = (orc_rpoint *)malloc((size_t)(2 * p) * sizeof(orc_rpoint));
    for (int64_t j = 0; j < p; j++) {
        pts[j].v = x[j];
        pts[j].colour = 0;
        pts[j].idx = (int32_t)j;
        pts[p + j].v = z[j];
        pts[p + j].colour = 1;
        pts[p + j].idx = (int32_t)j;
    }
    qsort(pts, (size_t)(2 * p), sizeof(orc_rpoint), orc_rpoint_cmp);
    int64_t cnt = 0;
    int64_t s = 0;
    while (s < 2 * p) {
        int64_t e = s;
        while (e < 2 * p && pts[e].v == pts[s].v)
            e++;
        int64_t mid = s;
        while (mid < e && pts[mid].colour == 0)
            mid++;
        for (int64_t a = s; a < mid; a++) {
            for (int64_t b = mid; b < e; b++) {
                if (cnt < cap) {
                    out[2 * cnt + 0] = pts[a].idx;
                    out[2 * cnt + 1] = pts[b].idx;
                }
                cnt++;
            }
        }
        s = e;
    }
    free(pts);
    return cnt;
}

/* ---------------------------------------------------------------- sets */

typedef struct {
    int32_t j, k, a;
} orc_triple;

static int orc_triple_cmp(const void *pa, const void *pb)
{
    const orc_triple *a = (const orc_triple *)pa, *b = (const orc_triple *)pb;
    if (a->j != b->j)
        return a->j < b->j ? -1 : 1;
    if (a->k != b->k)
        return a->k < b->k ? -1 : 1;
    return 0;
}

/* Sort triples by (j, k) and keep one per pair; returns the new count. */
static int64_t orc_sort_unique(orc_triple *t, int64_t cnt)
{
    if (cnt == 0)
        return 0;
    qsort(t, (size_t)cnt, sizeof(orc_triple), orc_triple_cmp);
    int64_t u = 1;
    for (int64_t i = 1; i < cnt; i++) {
        if (t[i].j != t[u - 1].j || t[i].k != t[u - 1].k)
            t[u++] = t[i];
    }
    return u;
}

typedef struct {
    orc_triple *v;
    int64_t n, cap;
} orc_vec;

static void orc_vec_push(orc_vec *vec, int32_t j, int32_t k, int32_t a)
{
    if (vec->n == vec->cap) {
        vec->cap = vec->cap ? 2 * vec->cap : 1024;
        vec->v = (orc_triple *)realloc(vec->v, (size_t)vec->cap * sizeof(orc_triple));
    }
    vec->v[vec->n].j = j;
    vec->v[vec->n].k = k;
    vec->v[vec->n].a = a;
    vec->n++;
}

/* Candidate set E_l of run `run` (the projection and equal-pairs steps of Algorithm 2) as unordered pairs
 * j < k (reading R4), sorted, each once.  The ordered pairs (j, k) and (k, j)
 * of the equal-pairs walk name the same unordered pair. */
static int64_t orc_rows_candidates(const int8_t *X, const int8_t *Y, int64_t n,
                                   int64_t p, const int64_t *rows, int32_t M,
                                   orc_vec *vec)
{
    uint64_t *x = (uint64_t *)malloc((size_t)p * sizeof(uint64_t));
    uint64_t *z = (uint64_t *)malloc((size_t)p * sizeof(uint64_t));
    orc_keys(X, Y, n, p, rows, M, x, z);
    int64_t ne = orc_equal_pairs(x, z, p, NULL, 0);
    int32_t *pairs = (int32_t *)malloc((size_t)(ne > 0 ? ne : 1) * 2 * sizeof(int32_t));
    orc_equal_pairs(x, z, p, pairs, ne);
    int64_t first = vec->n;
    for (int64_t e = 0; e < ne; e++) {
        int32_t j = pairs[2 * e], k = pairs[2 * e + 1];
        if (j == k)
            continue;
        orc_vec_push(vec, j < k ? j : k, j < k ? k : j, 0);
    }
    int64_t added = orc_sort_unique(vec->v + first, vec->n - first);
    vec->n = first + added;
    free(pairs);
    free(z);
    free(x);
    return added;
}

static int64_t orc_run_candidates(const int8_t *X, const int8_t *Y, int64_t n,
                                  int64_t p, int32_t M, uint64_t seed,
                                  int64_t run, orc_vec *vec)
{
    int64_t *rows = (int64_t *)malloc((size_t)(M > 0 ? M : 1) * sizeof(int64_t));
    orc_draw_rows(seed, run, M, n, rows);
    int64_t added = orc_rows_candidates(X, Y, n, p, rows, M, vec);
    free(rows);
    return added;
}

/* E_l of one run as unordered pairs (j, k), j < k, sorted by (j, k).
 * Writes up to `cap` pairs and returns their number. */
int64_t orc_candidates(const int8_t *X, const int8_t *Y, int64_t n, int64_t p,
                       int32_t M, uint64_t seed, int64_t run,
                       int32_t *out, int64_t cap)
{
    orc_vec vec = {0, 0, 0};
    int64_t cnt = orc_run_candidates(X, Y, n, p, M, seed, run, &vec);
    for (int64_t i = 0; i < cnt && i < cap; i++) {
        out[2 * i + 0] = vec.v[i].j;
        out[2 * i + 1] = vec.v[i].k;
    }
    free(vec.v);
    return cnt;
}

/* Algorithm 2 over runs [l0, l1): for each run draw the rows, build keys,
 * find E_l, and add to I the pairs of E_l with a_jk >= a_min (R5); return
 * I sorted by (j, k) with the agreement counts (R6).  Writes up to `cap`
 * triples (j, k, a) and returns |I|.  The full search is l0 = 0, l1 = L. */
int64_t orc_xyz_range(const int8_t *X, const int8_t *Y, int64_t n, int64_t p,
                      int64_t l0, int64_t l1, int32_t M, double kappa,
                      uint64_t seed, int32_t *out, int64_t cap)
{
    int64_t amin = orc_amin(n, kappa);
    orc_vec found = {0, 0, 0};
    orc_vec cand = {0, 0, 0};
    for (int64_t l = l0; l < l1; l++) {
        cand.n = 0;
        int64_t ne = orc_run_candidates(X, Y, n, p, M, seed, l, &cand);
        for (int64_t e = 0; e < ne; e++) {
            int32_t j = cand.v[e].j, k = cand.v[e].k;
            int64_t a = orc_agree(X, Y, n, j, k);
            if (a >= amin)
                orc_vec_push(&found, j, k, (int32_t)a);
        }
    }
    int64_t u = orc_sort_unique(found.v, found.n);
    for (int64_t i = 0; i < u && i < cap; i++) {
        out[3 * i + 0] = found.v[i].j;
        out[3 * i + 1] = found.v[i].k;
        out[3 * i + 2] = found.v[i].a;
    }
    free(found.v);
    free(cand.v);
    return u;
}

int64_t orc_xyz(const int8_t *X, const int8_t *Y, int64_t n, int64_t p,
                int32_t L, int32_t M, double kappa, uint64_t seed,
                int32_t *out, int64_t cap)
{
    return orc_xyz_range(X, Y, n, p, 0, L, M, kappa, seed, out, cap);
}

/* ------------------------------------------------- continuous response */

/* Section 3.1, continuous Y with binary X.  Z_ij = sgn(Y_i) X_ij, the rows of
 * a run are drawn i.i.d. with P(i) proportional to |Y_i|, and the strength of
 * (j, k) is the weighted agreement sum_{i : sgn(Y_i) = X_ij X_ik} |Y_i| over
 * ||Y||_1; in kappa form Y^T(X_j o X_k) / ||Y||_1 = 2 gamma~_jk - 1.
 *
 * Readings taken here:
 *   R9   the weights are used in fixed point.  With m = max_i |Y_i| written
 *        m = f 2^e, f in [0.5, 1), q_i = floor(|Y_i| 2^(24 - e) + 1/2), an
 *        integer in [0, 2^24]; Q = sum_i q_i.  sgn(0) = +1 (such a row has
 *        weight 0 and is never drawn).  The relative error of any weighted
 *        sum is below 2^-24 max|Y| / mean|Y|.
 *   R10  the weighted draw t of a search with seed s: u = splitmix64 output t
 *        (R2), r = floor(u Q / 2^64), and the row is the least i with
 *        q_0 + ... + q_i > r.  With equal weights this is the draw of R2.
 *   R11  a candidate passes when (double)(2 S_jk - Q) >= kappa (double)Q,
 *        S_jk = sum_{i : sgn(Y_i) = X_ij X_ik} q_i (one IEEE multiply, as R5).
 */

/* R9: fixed-point weights q and signs (+1 / -1) of a real response.  Returns
 * 0, or -1 when an entry is not finite or every entry is 0. */
int orc_quantize_y(const double *Y, int64_t n, int64_t *q, int8_t *sgn)
{
    double m = 0.0;
    for (int64_t i = 0; i < n; i++) {
        if (!isfinite(Y[i]))
            return -1;
        double a = fabs(Y[i]);
        if (a > m)
            m = a;
    }
    if (m == 0.0)
        return -1;
    int e = 0;
    frexp(m, &e);
    for (int64_t i = 0; i < n; i++) {
        q[i] = (int64_t)floor(ldexp(fabs(Y[i]), 24 - e) + 0.5);
        sgn[i] = Y[i] < 0.0 ? (int8_t)-1 : (int8_t)1;
    }
    return 0;
}

/* R10: the M rows of run `run`, drawn with probability q_i / Q. */
void orc_draw_rows_weighted(const int64_t *q, int64_t n, uint64_t seed,
                            int64_t run, int32_t M, int64_t *rows)
{
    uint64_t Q = 0;
    for (int64_t i = 0; i < n; i++)
        Q += (uint64_t)q[i];
    for (int32_t m = 0; m < M; m++) {
        uint64_t u = orc_splitmix64_at(seed, (uint64_t)run * (uint64_t)M + (uint64_t)m);
        uint64_t r = (uint64_t)(((unsigned __int128)u * (unsigned __int128)Q) >> 64);
        uint64_t c = 0;
        int64_t row = n - 1;
        for (int64_t i = 0; i < n; i++) {
            c += (uint64_t)q[i];
            if (c > r) {
                row = i;
                break;
            }
        }
        rows[m] = row;
    }
}

/* Weighted agreement of (j, k): returns the count of rows with
 * sgn(Y_i) = X_ij X_ik and writes their weight sum S_jk. */
int64_t orc_weighted_agree(const int8_t *X, const int8_t *sgn, const int64_t *q,
                           int64_t n, int64_t j, int64_t k, int64_t *S)
{
    int64_t a = 0, w = 0;
    for (int64_t i = 0; i < n; i++) {
        if ((int)X[j * n + i] * (int)X[k * n + i] == (int)sgn[i]) {
            a++;
            w += q[i];
        }
    }
    *S = w;
    return a;
}

/* Algorithm 2 with the modifications of Section 3.1 over runs [l0, l1):
 * weighted rows (R10), keys of X and Z = sgn(Y) o X, candidates as in the
 * binary search, kept by R11.  Writes up to `cap` triples (j, k, a) and
 * their S to `wsum`, sorted by (j, k), each pair once; returns the count.
 * -1 when Y is not usable (R9). */
int64_t orc_xyz_weighted_range(const int8_t *X, const double *Y, int64_t n, int64_t p,
                               int64_t l0, int64_t l1, int32_t M, double kappa,
                               uint64_t seed, int32_t *out, int64_t *wsum, int64_t cap)
{
    int64_t *q = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int8_t *sgn = (int8_t *)malloc((size_t)n);
    if (orc_quantize_y(Y, n, q, sgn) != 0) {
        free(q);
        free(sgn);
        return -1;
    }
    int64_t Q = 0;
    for (int64_t i = 0; i < n; i++)
        Q += q[i];
    int64_t *rows = (int64_t *)malloc((size_t)(M > 0 ? M : 1) * sizeof(int64_t));
    orc_vec found = {0, 0, 0};
    orc_vec cand = {0, 0, 0};
    for (int64_t l = l0; l < l1; l++) {
        cand.n = 0;
        orc_draw_rows_weighted(q, n, seed, l, M, rows);
        int64_t ne = orc_rows_candidates(X, sgn, n, p, rows, M, &cand);
        for (int64_t e = 0; e < ne; e++) {
            int32_t j = cand.v[e].j, k = cand.v[e].k;
            int64_t S = 0;
            int64_t a = orc_weighted_agree(X, sgn, q, n, j, k, &S);
            if ((double)(2 * S - Q) >= kappa * (double)Q)
                orc_vec_push(&found, j, k, (int32_t)a);
        }
    }
    int64_t u = orc_sort_unique(found.v, found.n);
    for (int64_t i = 0; i < u && i < cap; i++) {
        out[3 * i + 0] = found.v[i].j;
        out[3 * i + 1] = found.v[i].k;
        out[3 * i + 2] = found.v[i].a;
        orc_weighted_agree(X, sgn, q, n, found.v[i].j, found.v[i].k, &wsum[i]);
    }
    free(found.v);
    free(cand.v);
    free(rows);
    free(sgn);
    free(q);
    return u;
}

/* Every pair j < k passing R11, by looping over all pairs (the exhaustive
 * screen with the weighted strength).  Output as orc_xyz_weighted_range. */
int64_t orc_brute_force_weighted(const int8_t *X, const double *Y, int64_t n, int64_t p,
                                 double kappa, int32_t *out, int64_t *wsum, int64_t cap)
{
    int64_t *q = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int8_t *sgn = (int8_t *)malloc((size_t)n);
    if (orc_quantize_y(Y, n, q, sgn) != 0) {
        free(q);
        free(sgn);
        return -1;
    }
    int64_t Q = 0;
    for (int64_t i = 0; i < n; i++)
        Q += q[i];
    int64_t cnt = 0;
    for (int64_t j = 0; j < p; j++) {
        for (int64_t k = j + 1; k < p; k++) {
            int64_t S = 0;
            int64_t a = orc_weighted_agree(X, sgn, q, n, j, k, &S);
            if ((double)(2 * S - Q) >= kappa * (double)Q) {
                if (cnt < cap) {
                    out[3 * cnt + 0] = (int32_t)j;
                    out[3 * cnt + 1] = (int32_t)k;
                    out[3 * cnt + 2] = (int32_t)a;
                    wsum[cnt] = S;
                }
                cnt++;
            }
        }
    }
    free(sgn);
    free(q);
    return cnt;
}

/* -------------------------------------------- absolute value, Lasso screen */

/* Section 4 runs the search with Y set to each of +r and -r to find the
 * pairs with |r^T (X_j o X_k)| above a threshold.  The KKT check of
 * The KKT check of Algorithm 3 keeps the pairs with |r^T (X_j o X_k)| / n > lambda.
 *
 * Reading R12: with the fixed-point weights of R9 (q_i = floor(|r_i|
 * 2^(24-e) + 1/2)), r^T (X_j o X_k) is taken as (2 S_jk - Q) 2^(e-24), so the
 * strict test becomes the integer rule |2 S_jk - Q| >= t with
 * t = floor(ldexp(lambda * (double)n, 24 - e)) + 1. */
int64_t orc_kkt_threshold(const double *r, int64_t n, double lambda)
{
    double m = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double a = fabs(r[i]);
        if (a > m)
            m = a;
    }
    int e = 0;
    frexp(m, &e);
    return (int64_t)floor(ldexp(lambda * (double)n, 24 - e)) + 1;
}

/* The KKT violators V by the naive loop over all pairs, with R12: writes
 * triples (j, k, a) and the signed integer 2 S - Q to `d`. */
int64_t orc_kkt_brute(const int8_t *X, const double *r, int64_t n, int64_t p,
                      double lambda, int32_t *out, int64_t *d, int64_t cap)
{
    int64_t *q = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int8_t *sgn = (int8_t *)malloc((size_t)n);
    if (orc_quantize_y(r, n, q, sgn) != 0) {
        free(q);
        free(sgn);
        return -1;
    }
    int64_t Q = 0;
    for (int64_t i = 0; i < n; i++)
        Q += q[i];
    const int64_t t = orc_kkt_threshold(r, n, lambda);
    int64_t cnt = 0;
    for (int64_t j = 0; j < p; j++) {
        for (int64_t k = j + 1; k < p; k++) {
            int64_t S = 0;
            int64_t a = orc_weighted_agree(X, sgn, q, n, j, k, &S);
            int64_t v = 2 * S - Q;
            if (v >= t || -v >= t) {
                if (cnt < cap) {
                    out[3 * cnt + 0] = (int32_t)j;
                    out[3 * cnt + 1] = (int32_t)k;
                    out[3 * cnt + 2] = (int32_t)a;
                    d[cnt] = v;
                }
                cnt++;
            }
        }
    }
    free(sgn);
    free(q);
    return cnt;
}

/* The xyz form of the same check (Section 4): the continuous-response
 * search with Y = +r and with Y = -r, each keeping sign * (2 S - Q) >= t,
 * united; output as orc_kkt_brute, sorted by (j, k), each pair once. */
int64_t orc_kkt_xyz(const int8_t *X, const double *r, int64_t n, int64_t p, int64_t L,
                    int32_t M, double lambda, uint64_t seed, int32_t *out, int64_t *d, int64_t cap)
{
    int64_t *q = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int8_t *sgn = (int8_t *)malloc((size_t)n);
    int8_t *neg = (int8_t *)malloc((size_t)n);
    if (orc_quantize_y(r, n, q, sgn) != 0) {
        free(q);
        free(sgn);
        free(neg);
        return -1;
    }
    for (int64_t i = 0; i < n; i++)
        neg[i] = (int8_t)-sgn[i];
    int64_t Q = 0;
    for (int64_t i = 0; i < n; i++)
        Q += q[i];
    const int64_t t = orc_kkt_threshold(r, n, lambda);
    int64_t *rows = (int64_t *)malloc((size_t)(M > 0 ? M : 1) * sizeof(int64_t));
    orc_vec found = {0, 0, 0};
    orc_vec cand = {0, 0, 0};
    for (int side = 0; side < 2; side++) {
        const int8_t *s8 = side ? neg : sgn;
        for (int64_t l = 0; l < L; l++) {
            cand.n = 0;
            orc_draw_rows_weighted(q, n, seed, l, M, rows);
            int64_t ne = orc_rows_candidates(X, s8, n, p, rows, M, &cand);
            for (int64_t e = 0; e < ne; e++) {
                int32_t j = cand.v[e].j, k = cand.v[e].k;
                int64_t S = 0;
                int64_t a = orc_weighted_agree(X, sgn, q, n, j, k, &S);
                int64_t v = 2 * S - Q;
                if ((side ? -v : v) >= t)
                    orc_vec_push(&found, j, k, (int32_t)a);
            }
        }
    }
    int64_t u = orc_sort_unique(found.v, found.n);
    for (int64_t i = 0; i < u && i < cap; i++) {
        out[3 * i + 0] = found.v[i].j;
        out[3 * i + 1] = found.v[i].k;
        out[3 * i + 2] = found.v[i].a;
        int64_t S = 0;
        orc_weighted_agree(X, sgn, q, n, found.v[i].j, found.v[i].k, &S);
        d[i] = 2 * S - Q;
    }
    free(found.v);
    free(cand.v);
    free(rows);
    free(neg);
    free(sgn);
    free(q);
    return u;
}

/* ------------------------------------------------------ continuous X */

/* Section 3.2, the sign transform: X~_ij = sgn(X_ij), with a fair coin for
 * an entry that is exactly 0.  Reading R14: the coin of entry (i, j) is the
 * top bit of splitmix64 output t = j*n + i from state coin_seed (1 -> -1), so
 * the transform is reproducible.  Returns 0, or -1 on a NaN. */
int orc_sign_transform(const float *X, int64_t n, int64_t p, uint64_t coin_seed, int8_t *out)
{
    for (int64_t t = 0; t < n * p; t++) {
        float x = X[t];
        if (x != x)
            return -1;
        if (x < 0.0f)
            out[t] = -1;
        else if (x > 0.0f)
            out[t] = 1;
        else
            out[t] = (orc_splitmix64_at(coin_seed, (uint64_t)t) >> 63) ? (int8_t)-1 : (int8_t)1;
    }
    return 0;
}

/* Section 3.2, the unbiased transform.
 *
 * Reading R15: rows are scaled first, nu_i = max_j |X_ij| (float),
 * X'_ij = X_ij / nu_i (float division; a row of zeros stays 0) and
 * Y'_i = Y_i nu_i^2 (double), so X' lies in [-1, 1] and Proposition
 * "unbiased" applies to (Y', X').  The search is the continuous-response
 * search of R9-R11 on Y' with the random binary X~ of each draw: for draw
 * m of run l (row i = s_{l,m}) and column j, X~ = +1 with probability
 * g(X'_ij) = (X'_ij + 1) / 2, decided by u24 < g 2^24 with u24 the top 24
 * bits of splitmix64 output t = (l M + m) p + j from state
 * seed + 0x632BE59BD9B4E019 (a stream separate from the rows'); every draw
 * transforms independently.  Keys: bit m of column j is 1 iff X~ = -1.
 * A candidate passes when sum_i Y'_i X'_ij X'_ik >= kappa ||Y'||_1 (double
 * sums over i in order), i.e. gamma^g_jk >= (1 + kappa) / 2.
 */

/* Row scaling of R15: X' (n x p column-major float) and Y' (double). */
void orc_unbiased_scale(const float *X, const double *Y, int64_t n, int64_t p, float *Xs, double *Ys)
{
    for (int64_t i = 0; i < n; i++) {
        float nu = 0.0f;
        for (int64_t j = 0; j < p; j++) {
            float a = fabsf(X[j * n + i]);
            if (a > nu)
                nu = a;
        }
        for (int64_t j = 0; j < p; j++)
            Xs[j * n + i] = nu > 0.0f ? X[j * n + i] / nu : 0.0f;
        Ys[i] = Y[i] * ((double)nu * (double)nu);
    }
}

/* R15: the transformed value (+1 / -1) of entry (i, j) in draw m of run l. */
int orc_unbiased_draw(const float *Xs, int64_t n, int64_t p, uint64_t seed, int64_t run,
                      int32_t M, int32_t m, int64_t i, int64_t j)
{
    uint64_t t = ((uint64_t)run * (uint64_t)M + (uint64_t)m) * (uint64_t)p + (uint64_t)j;
    uint64_t u24 = orc_splitmix64_at(seed + 0x632BE59BD9B4E019ULL, t) >> 40;
    float g = (Xs[j * n + i] + 1.0f) / 2.0f;
    return ((double)u24 < (double)g * 16777216.0) ? 1 : -1;
}

/* sum_i Y'_i X'_ij X'_ik in double, i in order. */
double orc_real_dot(const float *Xs, const double *Ys, int64_t n, int64_t j, int64_t k)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++)
        s += Ys[i] * ((double)Xs[j * n + i] * (double)Xs[k * n + i]);
    return s;
}

/* The search of R15 over runs [l0, l1): writes up to `cap` pairs (j, k) and
 * their dot products, sorted, each pair once; returns the count, -1 when Y'
 * is unusable (R9). */
int64_t orc_xyz_unbiased_range(const float *X, const double *Y, int64_t n, int64_t p, int64_t l0,
                               int64_t l1, int32_t M, double kappa, uint64_t seed, int32_t *out,
                               double *dots, int64_t cap)
{
    float *Xs = (float *)malloc((size_t)(n * p) * sizeof(float));
    double *Ys = (double *)malloc((size_t)n * sizeof(double));
    int64_t *q = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int8_t *sgn = (int8_t *)malloc((size_t)n);
    orc_unbiased_scale(X, Y, n, p, Xs, Ys);
    if (orc_quantize_y(Ys, n, q, sgn) != 0) {
        free(Xs);
        free(Ys);
        free(q);
        free(sgn);
        return -1;
    }
    double norm1 = 0.0;
    for (int64_t i = 0; i < n; i++)
        norm1 += fabs(Ys[i]);
    int64_t *rows = (int64_t *)malloc((size_t)(M > 0 ? M : 1) * sizeof(int64_t));
    orc_vec found = {0, 0, 0};
    orc_vec cand = {0, 0, 0};
    for (int64_t l = l0; l < l1; l++) {
        orc_draw_rows_weighted(q, n, seed, l, M, rows);
        /* the transformed matrix restricted to this run's draws: draw m is
         * stored in "row" m of an M x p matrix */
        int8_t *Xm = (int8_t *)malloc((size_t)((M > 0 ? M : 1) * p));
        int8_t *Sm = (int8_t *)malloc((size_t)(M > 0 ? M : 1));
        int64_t *idx = (int64_t *)malloc((size_t)(M > 0 ? M : 1) * sizeof(int64_t));
        for (int32_t m = 0; m < M; m++) {
            for (int64_t j = 0; j < p; j++)
                Xm[j * M + m] = (int8_t)orc_unbiased_draw(Xs, n, p, seed, l, M, m, rows[m], j);
            Sm[m] = sgn[rows[m]];
            idx[m] = m;
        }
        cand.n = 0;
        int64_t ne = orc_rows_candidates(Xm, Sm, M, p, idx, M, &cand);
        for (int64_t e = 0; e < ne; e++) {
            int32_t j = cand.v[e].j, k = cand.v[e].k;
            if (orc_real_dot(Xs, Ys, n, j, k) >= kappa * norm1)
                orc_vec_push(&found, j, k, 0);
        }
        free(idx);
        free(Sm);
        free(Xm);
    }
    int64_t u = orc_sort_unique(found.v, found.n);
    for (int64_t i = 0; i < u && i < cap; i++) {
        out[2 * i + 0] = found.v[i].j;
        out[2 * i + 1] = found.v[i].k;
        dots[i] = orc_real_dot(Xs, Ys, n, found.v[i].j, found.v[i].k);
    }
    free(found.v);
    free(cand.v);
    free(rows);
    free(sgn);
    free(q);
    free(Ys);
    free(Xs);
    return u;
}
