// C ABI of libxyz: context life cycle, search orchestration, parity hooks.
//
// A search over runs [l0, l1) is split into launch groups of R runs.  For
// each group the device runs: keybuild (K2) -> LSD radix sort of the R*p
// composite keys (K3) -> join (K4) -> exclusive scan of bucket pair counts
// -> verify (K5).  Passing (j, k, a) records of all groups accumulate in one
// device buffer; after the last group they are sorted by (j, k) and made
// unique (K6), which is the union over runs of Algorithm 2, and copied to
// the host.  Host work is validation, sizing, and launching; the only
// synchronisations are the record count read before the final sort and the
// result copy.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/xyz.h"
#include "xyz_internal.cuh"

static_assert(sizeof(xyz_pair) == sizeof(xyz::PairOut), "pair layout");

namespace xyz {

static thread_local std::string g_err;

// entry budget of a launch group (the filter path holds 64 times that in runs' columns)
constexpr int64_t kDefaultChunkEntries = (int64_t)1 << 25;

void set_error(const std::string &msg) { g_err = msg; }

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

int64_t amin_rule(int64_t n, double kappa)
{
    // least a in [0, n] with (double)(2a - n) >= kappa * (double)n; the
    // left side grows with a, so a binary search over a finds it.
    const double rhs = kappa * (double)n;
    if ((double)n < rhs)
        return n + 1;
    int64_t lo = 0, hi = n;   // hi always passes
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if ((double)(2 * mid - n) >= rhs)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

static int ceil_log2(int64_t x)
{
    int b = 0;
    while (((int64_t)1 << b) < x)
        ++b;
    return b;
}

}  // namespace xyz

using namespace xyz;

// ------------------------------------------------------------------ ctx

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct xyz_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool owns_packed = true;     // false for a view sharing another context's packed X
    Packed pk;
    int *d_bad = nullptr;
    int64_t packed_bytes = 0;

    // workspace, grown on demand
    DevBuf keysA, keysB, valsA, valsB, radix_tmp, cnz, buckets, pair_counts, pair_off, scan_tmp;
    DevBuf counters;   // see the ctr_* accessors
    DevBuf ents, seg, members;   // partitioned grouping
    DevBuf kc_scratch;           // filter path: one key row per CTA
    DevBuf lst_keys, lst_cols;   // class-split filter: per-CTA class lists of keys and columns
    DevBuf seg_keys, seg_vals, seg_count;   // filter path: per-CTA survivor segments
    DevBuf buckets2, pair_counts2, pair_off2, scan_tmp2;   // filter path: spilled runs
    int64_t surv_cap = 0;        // filter path: survivor capacity (CTAs x segment)
    int64_t seg_cap = 0;         // filter path: survivors one CTA may write per group
    int64_t mem_cap = 0;         // filter path: members of on-chip groups per launch group
    int64_t spill_flush = 0;     // filter path: launch groups per spill flush (0: one per search)
    int onchip_parts = 32;       // filter path: hash partitions on chip for runs past its capacity
    int fuse_filters = 1;        // xyz_search_many: may join a fused filter launch
    DevBuf resp, ybs;            // batched search: response of each output pair, response bits
    DevBuf y_alt, y_stage;       // response updates: packed copy checked before use, host staging
    // real response (Section 3.1): live weights and a staging set swapped in
    // once a new response has been checked
    DevBuf wq, wcdf, wplanes, wq2, wcdf2, wplanes2, wmeta, wscan, yreal;
    int w_exp = 0;               // max|Y| = f 2^w_exp, f in [0.5, 1)
    // real X through the unbiased transform (Section 3.2)
    DevBuf xrs, xcs, xnu, ypr, ysd, ysd2, rbad;
    DevBuf vstart;               // verification: bucket of each block of 32 candidates
    // host copy of the last search's output pairs (and their responses),
    // taken with its output count when the record count was small;
    // hout_n = -1 when there is none
    std::vector<PairOut> hout;
    std::vector<uint32_t> hresp;
    int64_t hout_n = -1;
    int64_t vstart_cap = (int64_t)1 << 22;   // blocks of 32 candidates that vstart holds
    DevBuf pXc, pXr, pyb, pbad;  // packed X, response bits, input-check flag (owned contexts)
    DevBuf rec_keys, rec_keys_alt, rec_agree, rec_agree_alt, flags, pos, out, dedup_tmp, raw;
    int64_t rec_cap = 1 << 16;
    int64_t chunk_entries = kDefaultChunkEntries;
    xyz_tiles tiles{0, 0, 0};    // launch shapes set by xyz_set_tiles
    bool use_filter = true;
    bool force_big = false;      // class-split filter wherever it applies (xyz_set_filter 2)
    uint32_t big_lcap = 0;       // class-split filter: entries per class list and CTA (grown on overflow)
    bool big_off = false;        // class-split filter given up (its classes were too uneven)

    bool timing = false;
    xyz_stats stats;
};

// Workspace blocks released by a context (grown or destroyed) are kept per
// device and handed to the next request of a similar size, so that creating
// contexts, growing workspaces and serving searches do not pay cudaMalloc /
// cudaFree (which synchronise the device) in steady state.  A block is
// released only when its context's stream has no work in flight (after a
// finished search, or the synchronisation in destroy_ctx).
std::mutex g_pool_mu;
std::multimap<std::pair<int, size_t>, void *> g_pool;   // (device, bytes) -> block
size_t g_pool_bytes = 0;
constexpr size_t POOL_CAP = (size_t)64 << 30;

void pool_put(void *p, size_t bytes)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (g_pool_bytes + bytes > POOL_CAP) {
        cudaFree(p);
        return;
    }
    g_pool.emplace(std::make_pair(dev, bytes), p);
    g_pool_bytes += bytes;
}

// a cached block of want..2*want bytes on the current device, or null
void *pool_get(size_t want, size_t *got)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pool.lower_bound(std::make_pair(dev, want));
    if (it == g_pool.end() || it->first.first != dev || it->first.second > 2 * want)
        return nullptr;
    void *p = it->second;
    *got = it->first.second;
    g_pool_bytes -= *got;
    g_pool.erase(it);
    return p;
}

// While set (by the calling thread), ensure() allocates nothing: it adds to
// *t_size_only the bytes by which the buffer would grow and records the new
// size in the (copied) buffer descriptor, which is never dereferenced.
thread_local int64_t *t_size_only = nullptr;

static int ensure(DevBuf &b, size_t bytes)
{
    if (b.bytes >= bytes && b.ptr)
        return XYZ_OK;
    if (t_size_only) {
        const size_t want = bytes < 256 ? 256 : bytes;
        *t_size_only += (int64_t)want - (int64_t)(b.ptr ? b.bytes : 0);
        b.bytes = want;
        b.ptr = &b;
        return XYZ_OK;
    }
    if (b.ptr)
        pool_put(b.ptr, b.bytes);
    b.ptr = nullptr;
    b.bytes = 0;
    size_t want = bytes < 256 ? 256 : bytes;
    size_t got = 0;
    if ((b.ptr = pool_get(want, &got))) {
        b.bytes = got;
        return XYZ_OK;
    }
    cudaError_t e = cudaMalloc(&b.ptr, want);
    if (e != cudaSuccess) {
        b.ptr = nullptr;
        cudaGetLastError();
        return fail(XYZ_ENOMEM, std::string("cudaMalloc of ") + std::to_string(want) +
                                    " bytes failed: " + cudaGetErrorString(e));
    }
    b.bytes = want;
    return XYZ_OK;
}

static void release(DevBuf &b)
{
    if (b.ptr)
        pool_put(b.ptr, b.bytes);
    b.ptr = nullptr;
    b.bytes = 0;
}

static int64_t ws_bytes(const xyz_ctx *c)
{
    const DevBuf *all[] = {&c->keysA,   &c->keysB,       &c->valsA,     &c->valsB,
                           &c->radix_tmp, &c->cnz,       &c->buckets,   &c->pair_counts,
                           &c->pair_off, &c->scan_tmp,   &c->counters,  &c->rec_keys,
                           &c->rec_keys_alt, &c->rec_agree, &c->rec_agree_alt, &c->flags,
                           &c->pos,     &c->out,         &c->dedup_tmp, &c->raw,
                           &c->ents, &c->seg, &c->members, &c->kc_scratch, &c->lst_keys, &c->lst_cols,
                           &c->seg_keys, &c->seg_vals, &c->seg_count,
                           &c->buckets2, &c->pair_counts2, &c->pair_off2, &c->scan_tmp2,
                           &c->resp, &c->ybs, &c->y_alt, &c->y_stage,
                           &c->wq, &c->wcdf, &c->wplanes, &c->wq2, &c->wcdf2, &c->wplanes2,
                           &c->wmeta, &c->wscan, &c->yreal,
                           &c->xrs, &c->xcs, &c->xnu, &c->ypr, &c->ysd, &c->ysd2, &c->rbad, &c->vstart};
    int64_t s = 0;
    for (const DevBuf *b : all)
        s += (int64_t)b->bytes;
    return s;
}

// --------------------------------------------------------- stage timing

namespace {

enum Stage { ST_KEYS = 0, ST_SORT, ST_JOIN, ST_VERIFY, ST_DEDUP, ST_N };

struct Timer {
    bool on;
    cudaStream_t s;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
    cudaEvent_t cur = nullptr;
    int cur_stage = -1;
    int64_t launches[ST_N] = {0, 0, 0, 0, 0};
    int64_t *counter;
    int64_t at_begin = 0;

    Timer(bool on_, cudaStream_t s_, int64_t *counter_) : on(on_), s(s_), counter(counter_) {}
    void begin(int st)
    {
        cur_stage = st;
        at_begin = *counter;
        if (!on)
            return;
        cudaEventCreate(&cur);
        cudaEventRecord(cur, s);
    }
    void end()
    {
        launches[cur_stage] += *counter - at_begin;
        if (!on)
            return;
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, s);
        marks.push_back({cur_stage, {cur, e}});
        cur = nullptr;
    }
    // after a stream sync
    void collect(xyz_stats &st)
    {
        double ms[ST_N] = {0, 0, 0, 0, 0};
        float first_last = 0.f;
        for (auto &m : marks) {
            float t = 0.f;
            cudaEventElapsedTime(&t, m.second.first, m.second.second);
            ms[m.first] += t;
        }
        if (!marks.empty())
            cudaEventElapsedTime(&first_last, marks.front().second.first, marks.back().second.second);
        st.ms_keys = ms[ST_KEYS];
        st.ms_sort = ms[ST_SORT];
        st.ms_join = ms[ST_JOIN];
        st.ms_verify = ms[ST_VERIFY];
        st.ms_dedup = ms[ST_DEDUP];
        st.ms_total = first_last;
        st.launches_keys = launches[ST_KEYS];
        st.launches_sort = launches[ST_SORT];
        st.launches_join = launches[ST_JOIN];
        st.launches_verify = launches[ST_VERIFY];
        st.launches_dedup = launches[ST_DEDUP];
    }
    ~Timer()
    {
        for (auto &m : marks) {
            cudaEventDestroy(m.second.first);
            cudaEventDestroy(m.second.second);
        }
        if (cur)
            cudaEventDestroy(cur);
    }
};

struct Plan {
    int64_t R;        // runs per launch group
    int NB, BB;       // filter path: response blocks per run, responses per block
    bool filter;      // per-run survivor filter with on-chip grouping (M <= 31, p <= 262144)
    bool big;         // ... in its class-split form (one response, M <= 28, larger p)
    bool part;        // partitioned grouping (M <= 31, large p)
    bool k64;         // 64-bit composite keys (LSD path)
    int kbits;        // bits of a column index (record keys use 2*kbits)
};

Plan make_plan(const xyz_ctx *c, int64_t runs, int M, int B)
{
    Plan pl;
    const int64_t p = c->pk.p;
    int64_t entries = c->chunk_entries < ((int64_t)1 << 31) ? c->chunk_entries : ((int64_t)1 << 31);
    int64_t rmax = entries / p;
    if (rmax < 1)
        rmax = 1;
    if (rmax > 65535)
        rmax = 65535;
    int64_t R = runs < rmax ? runs : rmax;
    pl.filter = (c->use_filter || B > 1) && filter_supported(p, M);
    // one binary response past the shared-memory filter's p (or forced):
    // the class-split filter, on the same buffers and host loop
    pl.big = c->use_filter && !c->big_off && B == 1 && !c->pk.Xrs && filter_big_supported(p, M) &&
             (!pl.filter || c->force_big);
    if (pl.big)
        pl.filter = true;
    pl.part = !pl.filter && part_supported(p, M);
    pl.k64 = false;
    pl.NB = pl.BB = 1;
    pl.kbits = ceil_log2(p);
    if (pl.kbits < 1)
        pl.kbits = 1;
    if (pl.filter) {
        // only a few percent of a run's columns survive, so a launch group may
        // span 64 times the entry budget (up to 16384 runs: the whole of most
        // searches); every launch group ends with a tail of CTAs finishing
        // their last runs, so fewer groups are faster.  Batches keep about
        // 4096 (run, response) items.
        int64_t rf = B > 1 ? (4096 / B > 0 ? 4096 / B : 1) : 64 * entries / p;
        if (rf < 1)
            rf = 1;
        if (rf > 16384)
            rf = 16384;
        pl.R = runs < rf ? runs : rf;
        // enough (run, response block) items for every SM
        const int64_t want = 2 * (int64_t)filter_grid();
        int64_t nb = (want + pl.R - 1) / pl.R;
        if (nb > B)
            nb = B;
        if (nb < 1)
            nb = 1;
        pl.BB = (int)((B + nb - 1) / nb);
        pl.NB = (int)((B + pl.BB - 1) / pl.BB);
        return pl;
    }
    if (pl.part) {
        pl.R = R < 1 ? 1 : R;
        return pl;
    }
    int rb = ceil_log2(R);
    if (M + rb <= 32) {
        pl.k64 = false;
    } else if (M <= 28) {
        pl.k64 = false;
        R = (int64_t)1 << (32 - M);
    } else {
        pl.k64 = true;
        if (M + rb > 64)
            R = (int64_t)1 << (64 - M);   // M = 64 -> one run per group
    }
    pl.R = R < 1 ? 1 : R;
    return pl;
}

int ensure_search_ws(xyz_ctx *c, const Plan &pl, int B, int64_t runs)
{
    const int64_t N = pl.R * c->pk.p;
    const size_t ksz = pl.k64 ? 8 : 4;
    const int64_t bcap = N / 2 + 1;
    int rc;
    if (pl.filter) {
        // spilled runs are rare: each CTA's segment starts with room for
        // about one run and grows when it overflows
        if (c->seg_cap < 1)
            c->seg_cap = c->pk.p + 4096;
        const int64_t grid = filter_grid();
        const int64_t cap = grid * c->seg_cap;
        c->surv_cap = cap;
        const int64_t sb = cap / 2 + 1;
        const int64_t items = pl.R * B;
        if (c->mem_cap < 1) {
            // members grouped on chip per launch group, grown on overflow
            const int64_t per = c->pk.p < 4096 ? c->pk.p : 4096;
            c->mem_cap = items * per > 65536 ? items * per : 65536;
        }
        const int64_t mcap = c->mem_cap;
        const int64_t mb = mcap / 2 + 1;
        const int64_t cnz_bytes = (int64_t)B << ceil_log2(runs);
        if (pl.big) {
            const uint32_t want = filter_big_lcap(c->pk.p);
            if (c->big_lcap < want)
                c->big_lcap = want;
            const size_t words = filter_big_list_words(c->pk.p, c->big_lcap);
            if ((rc = ensure(c->lst_keys, words * 4)) || (rc = ensure(c->lst_cols, words * 4)))
                return rc;
        }
        if ((rc = ensure(c->kc_scratch, pl.big ? 4 : filter_scratch_words(c->pk.p) * 4)) ||
            (rc = ensure(c->seg_keys, (size_t)cap * 8)) || (rc = ensure(c->seg_vals, (size_t)cap * 4)) ||
            (rc = ensure(c->seg_count, (size_t)grid * 4)) ||
            (rc = ensure(c->keysA, cap * 8)) || (rc = ensure(c->keysB, cap * 8)) ||
            (rc = ensure(c->valsA, cap * 4)) || (rc = ensure(c->valsB, cap * 4)) ||
            (rc = ensure(c->radix_tmp, radix_temp_bytes(cap))) || (rc = ensure(c->cnz, cnz_bytes)) ||
            (rc = ensure(c->members, mcap * 4)) || (rc = ensure(c->buckets, mb * sizeof(Bucket))) ||
            (rc = ensure(c->pair_counts, mb * 8)) || (rc = ensure(c->pair_off, mb * 8)) ||
            (rc = ensure(c->scan_tmp, scan_temp_bytes(mb))) ||
            (rc = ensure(c->buckets2, sb * sizeof(Bucket))) || (rc = ensure(c->pair_counts2, sb * 8)) ||
            (rc = ensure(c->pair_off2, sb * 8)) || (rc = ensure(c->scan_tmp2, scan_temp_bytes(sb))) ||
            (rc = ensure(c->counters, 128)))
            return rc;
        return XYZ_OK;
    }
    if (pl.part) {
        if ((rc = ensure(c->ents, N * 8)) || (rc = ensure(c->members, N * 4)) ||
            (rc = ensure(c->seg, part_seg_words(c->pk.p, (int)pl.R) * 4)) ||
            (rc = ensure(c->cnz, pl.R)) || (rc = ensure(c->buckets, bcap * sizeof(Bucket))) ||
            (rc = ensure(c->pair_counts, bcap * 8)) || (rc = ensure(c->pair_off, bcap * 8)) ||
            (rc = ensure(c->scan_tmp, scan_temp_bytes(bcap))) || (rc = ensure(c->counters, 128)))
            return rc;
        return XYZ_OK;
    }
    if ((rc = ensure(c->keysA, N * ksz)) || (rc = ensure(c->keysB, N * ksz)) ||
        (rc = ensure(c->valsA, N * 4)) || (rc = ensure(c->valsB, N * 4)) ||
        (rc = ensure(c->radix_tmp, radix_temp_bytes(N))) || (rc = ensure(c->cnz, pl.R)) ||
        (rc = ensure(c->buckets, bcap * sizeof(Bucket))) ||
        (rc = ensure(c->pair_counts, bcap * 8)) || (rc = ensure(c->pair_off, bcap * 8)) ||
        (rc = ensure(c->scan_tmp, scan_temp_bytes(bcap))) || (rc = ensure(c->counters, 128)))
        return rc;
    return XYZ_OK;
}

// The verification's table of the bucket of each block of 32 candidates
// (4 bytes per block) starts at 2^22 blocks and grows, after a search's
// first launch group, to twice the blocks that group had (at most 2^27);
// candidates past the table find their bucket by a binary search instead.
constexpr int64_t VSTART_MAX = (int64_t)1 << 27;
// a search copies its output to the host with the output count when it has
// at most this many records (the output is at most that long)
constexpr int64_t HOUT_MAX = 65536;

int ensure_records(xyz_ctx *c, int B)
{
    const int64_t cap = c->rec_cap;
    int rc;
    if ((rc = ensure(c->vstart, (size_t)c->vstart_cap * 4)))
        return rc;
    if ((rc = ensure(c->rec_keys, cap * 8)) || (rc = ensure(c->rec_keys_alt, cap * 8)) ||
        (rc = ensure(c->rec_agree, cap * 4)) || (rc = ensure(c->rec_agree_alt, cap * 4)) ||
        (rc = ensure(c->flags, cap * 4)) || (rc = ensure(c->pos, cap * 4)) ||
        (rc = ensure(c->out, cap * sizeof(PairOut))) ||
        (rc = ensure(c->dedup_tmp, radix_temp_bytes(cap) + scan_temp_bytes(cap))) ||
        (B > 1 && (rc = ensure(c->resp, cap * 4))))
        return rc;
    return XYZ_OK;
}

// Device counters: per launch group (cleared before each group) the bucket
// and member counts; per search the spill count and overflow flags, the
// spill-path bucket count, the record and output counts, the error flag,
// the group's candidate total, the candidate sum, the spill total, the
// filter's work-item counter, the columns the filter kept, the bucket
// members the on-chip grouping wrote and the runs grouped on chip from the
// segment.
uint32_t *ctr_u32(xyz_ctx *c) { return reinterpret_cast<uint32_t *>(c->counters.ptr); }
uint32_t *ctr_nbuckets(xyz_ctx *c) { return ctr_u32(c) + 0; }
uint32_t *ctr_members(xyz_ctx *c) { return ctr_u32(c) + 1; }
uint32_t *ctr_nsurv(xyz_ctx *c) { return ctr_u32(c) + 2; }
int *ctr_sovf(xyz_ctx *c) { return reinterpret_cast<int *>(ctr_u32(c) + 3); }
uint32_t *ctr_nbuckets2(xyz_ctx *c) { return ctr_u32(c) + 4; }
uint32_t *ctr_nrec(xyz_ctx *c) { return ctr_u32(c) + 5; }
uint32_t *ctr_nout(xyz_ctx *c) { return ctr_u32(c) + 6; }
int *ctr_err(xyz_ctx *c) { return reinterpret_cast<int *>(ctr_u32(c) + 7); }
uint64_t *ctr_total(xyz_ctx *c) { return reinterpret_cast<uint64_t *>((char *)c->counters.ptr + 32); }
uint64_t *ctr_cand(xyz_ctx *c) { return reinterpret_cast<uint64_t *>((char *)c->counters.ptr + 40); }
uint64_t *ctr_total2(xyz_ctx *c) { return reinterpret_cast<uint64_t *>((char *)c->counters.ptr + 48); }
uint32_t *ctr_work(xyz_ctx *c) { return reinterpret_cast<uint32_t *>((char *)c->counters.ptr + 56); }
unsigned long long *ctr_kept(xyz_ctx *c)
{
    return reinterpret_cast<unsigned long long *>((char *)c->counters.ptr + 64);
}

#define CU(expr)                                                                         \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess)                                                           \
            return fail(XYZ_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));  \
    } while (0)

// Runs [l0, l1) for B responses with threshold amin.  ybs: the responses'
// bit rows on the device (B rows of Wp words; B == 1 and ybs == pk.yb for an
// ordinary search; B > 1 needs the filter path).  Results (sorted by
// (response, j, k), each once) go to the device `out` buffer, and their
// responses to `resp` when B > 1; the count goes to *nout_host.  An
// attempt that overflowed a buffer is redone once the buffer has grown.
// Phases, so that the launch groups of several searches can be captured
// into one CUDA graph: SP_PREPARE sizes the workspace only; SP_ENQUEUE
// enqueues the launch groups (no host synchronisation, no allocation, spills
// left for the end); SP_FINISH does the rest (spills, union) after they ran,
// and returns SP_RERUN when a buffer overflowed so the caller redoes the
// search with SP_ALL.  A search of one launch group whose filter joins a
// fused launch with others (search_fusable) splits SP_ENQUEUE in two:
// SP_ENQUEUE_PRE enqueues what comes before the filter and stores the
// filter's arguments in *defer; SP_ENQUEUE_POST, after the fused launch,
// what comes after it.
enum SearchPhase { SP_ALL = 0, SP_ENQUEUE = 1, SP_FINISH = 2, SP_PREPARE = 3, SP_ENQUEUE_PRE = 4,
                   SP_ENQUEUE_POST = 5 };
constexpr int SP_RERUN = 100;

// Thresholds of a search at kappa: a real response passes when
// 2S - Q >= kappa Q (Q the total weight), a real X when the dot product of
// the transformed columns reaches kappa ||Y'||_1 (the oracle's reading).
void set_kappa(xyz_ctx *c, double kappa)
{
    c->pk.wkq = kappa * (double)c->pk.wtotal;
    c->pk.wscale = 0.0;
    c->pk.rkq = kappa * c->pk.rnorm;
}

// Key class of the fused filter launch that a search of `runs` runs at M
// can join (after SP_PREPARE), 0 when it cannot: one launch group, one
// response, binary X and the single-filter path.
int search_fusable(xyz_ctx *c, int64_t runs, int M)
{
    const Plan pl = make_plan(c, runs, M, 1);
    if (!pl.filter || pl.big || c->pk.Xrs || runs > pl.R)
        return 0;
    return fused_key_class(M);
}

int run_search_multi(xyz_ctx *c, const uint32_t *ybs, int B, int64_t l0, int64_t l1, int M,
                     int64_t amin, uint64_t seed, int64_t *nout_host, int phase = SP_ALL,
                     FilterArgs *defer = nullptr)
{
    const bool enq = phase == SP_ENQUEUE || phase == SP_ENQUEUE_PRE || phase == SP_ENQUEUE_POST;
    const int64_t runs = l1 - l0;
    const int64_t p = c->pk.p;
    Plan pl = make_plan(c, runs, M, B);            // replanned when the class-split filter is given up
    if (B > 1 && !pl.filter)
        return fail(XYZ_EINVAL, "batched search needs M <= 31 and p <= 262144");
    if (c->pk.Xrs && (!pl.filter || B > 1))
        return fail(XYZ_EINVAL, "a real X needs M <= 31, p <= 262144 and one response");
    const int bbits = ceil_log2(B);
    const int rbits = ceil_log2(runs);
    if (pl.filter && bbits + rbits + M > 64)
        return fail(XYZ_EINVAL, "too many runs x responses for one search");
    int rc;
    for (int attempt = 0; attempt < 8; ++attempt) {
        if (phase != SP_FINISH) {
            if ((rc = ensure_search_ws(c, pl, B, runs)) || (rc = ensure_records(c, B)))
                return rc;
            if (phase == SP_PREPARE)
                return XYZ_OK;
        }
        int64_t launches = 0;
        Timer tm(c->timing && phase == SP_ALL, c->stream, &launches);
        xyz_stats st;
        std::memset(&st, 0, sizeof(st));
        if (phase != SP_FINISH && phase != SP_ENQUEUE_POST)
            CU(cudaMemsetAsync(c->counters.ptr, 0, 128, c->stream));
        if ((phase == SP_ENQUEUE_PRE || phase == SP_ENQUEUE_POST) &&
            (!pl.filter || pl.big || B != 1 || c->pk.Xrs || runs > pl.R || (phase == SP_ENQUEUE_PRE && !defer)))
            return fail(XYZ_EINVAL, "search cannot join a fused filter launch");
        int64_t chunks = phase == SP_FINISH ? (runs + pl.R - 1) / pl.R : 0;
        int64_t surv_total = 0;
        // host copy of the device counters (one copy of the block per
        // synchronisation); hc_fresh while no kernel has run since it was taken
        alignas(8) uint32_t hc[32];
        bool hc_fresh = false;
        auto read_counters = [&]() -> int {
            CU(cudaMemcpyAsync(hc, c->counters.ptr, sizeof(hc), cudaMemcpyDeviceToHost, c->stream));
            CU(cudaStreamSynchronize(c->stream));
            hc_fresh = true;
            return XYZ_OK;
        };
        int key_bits_max = 0;
        bool redo = false;
        if (pl.filter) {
            const int grid = filter_grid();
            const int64_t mb = c->mem_cap / 2 + 1;
            const int sbits = bbits + rbits + M;
            key_bits_max = sbits;
            // Runs with too many survivors for the chip spill to per-CTA
            // segments; the spills of `flush` launch groups (all of them when
            // flush == 0) are sorted, joined and verified together.
            auto flush_spills = [&]() -> int {
                tm.begin(ST_KEYS);
                CU(launch_compact((const uint64_t *)c->seg_keys.ptr, (const uint32_t *)c->seg_vals.ptr,
                                  (const uint32_t *)c->seg_count.ptr, (uint32_t)c->seg_cap, grid,
                                  (uint64_t *)c->keysA.ptr, (uint32_t *)c->valsA.ptr, ctr_nsurv(c),
                                  c->stream, &launches));
                tm.end();
                if (int r = read_counters())
                    return r;
                const uint32_t ns = hc[2], mem_tried = hc[1];
                const int sovf = (int)hc[3];
                if (sovf & 1) {
                    // a spill segment overflowed: larger segments up to a
                    // bound, then more frequent flushes
                    const int64_t seg_limit = ((int64_t)1 << 27) / grid;
                    if (c->seg_cap * 2 <= seg_limit || c->spill_flush == 1)
                        c->seg_cap *= 2;
                    else
                        c->spill_flush = c->spill_flush ? (c->spill_flush + 1) / 2
                                                        : ((l1 - l0 + pl.R - 1) / pl.R + 1) / 2;
                    redo = true;
                }
                if (sovf & 4) {
                    // a class list of the class-split filter did: room for
                    // all of a run's keys in one class (it cannot overflow
                    // again), or, when the device has no room for that, the
                    // path without the class-split filter
                    const uint32_t lmax = filter_big_lcap_max(p);
                    bool give_up = c->big_lcap >= lmax;
                    if (!give_up) {
                        const size_t words = filter_big_list_words(p, lmax);
                        if (ensure(c->lst_keys, words * 4) || ensure(c->lst_cols, words * 4)) {
                            g_err.clear();
                            give_up = true;
                        } else {
                            c->big_lcap = lmax;
                        }
                    }
                    if (give_up) {
                        c->big_off = true;
                        pl = make_plan(c, runs, M, B);
                    }
                    redo = true;
                }
                if (sovf & 2) {
                    // the on-chip groups' members did: at least double, and at
                    // least what the last launch group tried to reserve
                    const int64_t want = (int64_t)mem_tried + (int64_t)mem_tried / 4;
                    c->mem_cap = want > 2 * c->mem_cap ? want : 2 * c->mem_cap;
                    redo = true;
                }
                if (redo || ns == 0)
                    return XYZ_OK;               // nothing launched since the counters were read
                hc_fresh = false;
                surv_total += ns;
                const int64_t sb = c->surv_cap / 2 + 1;
                bool alt = false;
                tm.begin(ST_SORT);
                CU(radix_sort64((uint64_t *)c->keysA.ptr, (uint32_t *)c->valsA.ptr,
                                (uint64_t *)c->keysB.ptr, (uint32_t *)c->valsB.ptr, (int64_t)ns, sbits,
                                c->radix_tmp.ptr, &alt, c->stream, &launches));
                tm.end();
                const uint64_t *ks = (const uint64_t *)(alt ? c->keysB.ptr : c->keysA.ptr);
                const uint32_t *vs = (const uint32_t *)(alt ? c->valsB.ptr : c->valsA.ptr);
                tm.begin(ST_JOIN);
                CU(cudaMemsetAsync(ctr_nbuckets2(c), 0, 4, c->stream));
                CU(launch_join64(ks, (int64_t)ns, M, bbits + rbits, (const uint8_t *)c->cnz.ptr,
                                 (Bucket *)c->buckets2.ptr, (uint64_t *)c->pair_counts2.ptr,
                                 ctr_nbuckets2(c), c->stream, &launches, rbits));
                CU(scan_u64_dev((const uint64_t *)c->pair_counts2.ptr, (uint64_t *)c->pair_off2.ptr,
                                ctr_nbuckets2(c), sb, ctr_total2(c), ctr_cand(c), c->scan_tmp2.ptr,
                                c->stream, &launches));
                tm.end();
                tm.begin(ST_VERIFY);
                CU(launch_verify(c->pk, (const Bucket *)c->buckets2.ptr,
                                 (const uint64_t *)c->pair_off2.ptr, ctr_nbuckets2(c), ctr_total2(c), vs,
                                 amin, pl.kbits, (uint64_t *)c->rec_keys.ptr,
                                 (uint32_t *)c->rec_agree.ptr, ctr_nrec(c), (uint32_t)c->rec_cap,
                                 c->stream, &launches, B > 1 ? ybs : nullptr, nullptr,
                                 (uint32_t *)c->vstart.ptr, c->vstart_cap, ctr_err(c)));
                tm.end();
                CU(launch_seg_reset((uint32_t *)c->seg_count.ptr, c->stream, &launches));
                return XYZ_OK;
            };
            if (phase != SP_FINISH && phase != SP_ENQUEUE_POST)
                CU(launch_seg_reset((uint32_t *)c->seg_count.ptr, c->stream, &launches));
            int64_t since_flush = 0;
            for (int64_t g0 = l0; g0 < l1 && !redo && phase != SP_FINISH; g0 += pl.R) {
                const int64_t Rc = (l1 - g0) < pl.R ? (l1 - g0) : pl.R;
                ++chunks;
                if (phase != SP_ENQUEUE_POST) {
                    CU(cudaMemsetAsync(ctr_u32(c), 0, 8, c->stream));   // buckets, members
                    CU(cudaMemsetAsync(ctr_work(c), 0, 4, c->stream));  // the filter's work items
                }
                tm.begin(ST_KEYS);
                if (phase == SP_ENQUEUE_POST)
                    ;                                   // the filter ran in the fused launch
                else if (pl.big)
                    CU(launch_filter_big(c->pk, M, seed, g0, (int)Rc, rbits, g0 - l0, grid,
                                         (uint32_t)(c->mem_cap < 0xFFFFFFFELL ? c->mem_cap : 0xFFFFFFFELL),
                                         (uint32_t)mb, (uint32_t *)c->lst_keys.ptr, (uint32_t *)c->lst_cols.ptr,
                                         c->big_lcap, (uint64_t *)c->seg_keys.ptr, (uint32_t *)c->seg_vals.ptr,
                                         (uint32_t *)c->seg_count.ptr, (uint32_t)c->seg_cap, ctr_sovf(c),
                                         (uint8_t *)c->cnz.ptr, (uint32_t *)c->members.ptr, ctr_members(c),
                                         (Bucket *)c->buckets.ptr, (uint64_t *)c->pair_counts.ptr,
                                         ctr_nbuckets(c), c->stream, &launches, c->onchip_parts, ctr_work(c),
                                         ctr_kept(c)));
                else
                    CU(launch_filter(c->pk, ybs, B, M, seed, g0, (int)Rc, pl.NB, pl.BB, rbits, g0 - l0,
                                     grid, (uint32_t)(c->mem_cap < 0xFFFFFFFELL ? c->mem_cap : 0xFFFFFFFELL),
                                     (uint32_t)mb, (uint32_t *)c->kc_scratch.ptr,
                                     (uint64_t *)c->seg_keys.ptr, (uint32_t *)c->seg_vals.ptr,
                                     (uint32_t *)c->seg_count.ptr, (uint32_t)c->seg_cap, ctr_sovf(c),
                                     (uint8_t *)c->cnz.ptr, (uint32_t *)c->members.ptr, ctr_members(c),
                                     (Bucket *)c->buckets.ptr, (uint64_t *)c->pair_counts.ptr,
                                     ctr_nbuckets(c), c->stream, &launches, c->onchip_parts, ctr_work(c),
                                     ctr_kept(c), phase == SP_ENQUEUE_PRE ? defer : nullptr));
                tm.end();
                if (phase == SP_ENQUEUE_PRE)
                    return XYZ_OK;                      // one launch group: the rest after the fused launch
                tm.begin(ST_JOIN);
                CU(scan_u64_dev((const uint64_t *)c->pair_counts.ptr, (uint64_t *)c->pair_off.ptr,
                                ctr_nbuckets(c), mb, ctr_total(c), ctr_cand(c), c->scan_tmp.ptr,
                                c->stream, &launches));
                tm.end();
                tm.begin(ST_VERIFY);
                CU(launch_verify(c->pk, (const Bucket *)c->buckets.ptr,
                                 (const uint64_t *)c->pair_off.ptr, ctr_nbuckets(c), ctr_total(c),
                                 (const uint32_t *)c->members.ptr, amin, pl.kbits,
                                 (uint64_t *)c->rec_keys.ptr, (uint32_t *)c->rec_agree.ptr,
                                 ctr_nrec(c), (uint32_t)c->rec_cap, c->stream, &launches,
                                 B > 1 ? ybs : nullptr, ctr_sovf(c), (uint32_t *)c->vstart.ptr, c->vstart_cap,
                                 ctr_err(c)));
                tm.end();
                if (phase == SP_ALL && g0 == l0 && g0 + pl.R < l1) {
                    // the first of several launch groups tells whether the
                    // member space and the record space suffice: when not,
                    // they grow now and the search restarts after one group
                    // (a whole search would be lost at the end)
                    int sovf = 0;
                    uint32_t mem_tried = 0, nrec1 = 0;
                    uint64_t cand1 = 0;
                    CU(cudaMemcpyAsync(&sovf, ctr_sovf(c), 4, cudaMemcpyDeviceToHost, c->stream));
                    CU(cudaMemcpyAsync(&mem_tried, ctr_members(c), 4, cudaMemcpyDeviceToHost, c->stream));
                    CU(cudaMemcpyAsync(&nrec1, ctr_nrec(c), 4, cudaMemcpyDeviceToHost, c->stream));
                    CU(cudaMemcpyAsync(&cand1, ctr_total(c), 8, cudaMemcpyDeviceToHost, c->stream));
                    CU(cudaStreamSynchronize(c->stream));
                    // room in the block-start table for the later groups'
                    // candidates (nothing is in flight: the table may move)
                    const int64_t want_blocks = 2 * (int64_t)((cand1 + 31) / 32);
                    if (!(sovf & 2) && want_blocks > c->vstart_cap && c->vstart_cap < VSTART_MAX) {
                        int64_t cap = c->vstart_cap;
                        while (cap < want_blocks && cap < VSTART_MAX)
                            cap *= 2;
                        if (ensure(c->vstart, (size_t)cap * 4) == XYZ_OK) {
                            c->vstart_cap = cap;
                        } else {
                            // no room: a table of the old size again (the
                            // failed attempt released it); the candidates
                            // past it find their bucket by binary search
                            g_err.clear();
                            if ((rc = ensure(c->vstart, (size_t)c->vstart_cap * 4)))
                                return rc;
                        }
                    }
                    if (sovf & 2) {
                        const int64_t want = (int64_t)mem_tried + (int64_t)mem_tried / 4;
                        c->mem_cap = want > 2 * c->mem_cap ? want : 2 * c->mem_cap;
                        redo = true;
                    }
                    if ((sovf & 5) && (rc = flush_spills()))      // segments or class lists: grown there
                        return rc;
                    const int64_t groups = (runs + pl.R - 1) / pl.R;
                    const int64_t want_rec = 2 * (int64_t)nrec1 * groups;
                    if (want_rec > c->rec_cap && !(sovf & 2)) {
                        int64_t cap = c->rec_cap;
                        while (cap < want_rec && cap < (int64_t)0xF0000000LL / 2)
                            cap *= 2;
                        c->rec_cap = cap;
                        redo = true;
                    }
                }
                if (phase == SP_ALL && c->spill_flush && ++since_flush == c->spill_flush && g0 + pl.R < l1) {
                    since_flush = 0;
                    if ((rc = flush_spills()))
                        return rc;
                }
            }
            if (enq)
                return XYZ_OK;
            if (redo)
                continue;
            if ((rc = flush_spills()))
                return rc;
            if (redo) {
                if (phase == SP_FINISH)
                    return SP_RERUN;
                continue;
            }
        } else {
            for (int64_t g0 = l0; g0 < l1 && phase != SP_FINISH; g0 += pl.R) {
                const int64_t Rc = (l1 - g0) < pl.R ? (l1 - g0) : pl.R;
                const int64_t Nc = Rc * p;
                const int rb = ceil_log2(Rc);
                const int bits = M + rb;
                key_bits_max = bits > key_bits_max ? bits : key_bits_max;
                ++chunks;
                CU(cudaMemsetAsync(ctr_u32(c), 0, 8, c->stream));   // buckets, members
                const int64_t bcap = Nc / 2 + 1;
                if (pl.part) {
                    tm.begin(ST_KEYS);
                    CU(launch_keybuild_part(c->pk, M, seed, g0, (int)Rc, (uint64_t *)c->ents.ptr,
                                            (uint32_t *)c->seg.ptr, (uint8_t *)c->cnz.ptr, c->stream,
                                            &launches));
                    tm.end();
                    tm.begin(ST_JOIN);
                    CU(launch_group(c->pk, (int)Rc, (const uint64_t *)c->ents.ptr,
                                    (const uint32_t *)c->seg.ptr, (const uint8_t *)c->cnz.ptr,
                                    (uint32_t *)c->members.ptr, ctr_members(c),
                                    (Bucket *)c->buckets.ptr, (uint64_t *)c->pair_counts.ptr,
                                    ctr_nbuckets(c), ctr_err(c), c->stream, &launches));
                    CU(scan_u64_dev((const uint64_t *)c->pair_counts.ptr, (uint64_t *)c->pair_off.ptr,
                                    ctr_nbuckets(c), bcap, ctr_total(c), ctr_cand(c), c->scan_tmp.ptr,
                                    c->stream, &launches));
                    tm.end();
                    tm.begin(ST_VERIFY);
                    CU(launch_verify(c->pk, (const Bucket *)c->buckets.ptr,
                                     (const uint64_t *)c->pair_off.ptr, ctr_nbuckets(c), ctr_total(c),
                                     (const uint32_t *)c->members.ptr, amin, pl.kbits,
                                     (uint64_t *)c->rec_keys.ptr, (uint32_t *)c->rec_agree.ptr,
                                     ctr_nrec(c), (uint32_t)c->rec_cap, c->stream, &launches, nullptr,
                                     nullptr, (uint32_t *)c->vstart.ptr, c->vstart_cap, ctr_err(c)));
                    tm.end();
                    continue;
                }
                bool alt = false;
                tm.begin(ST_KEYS);
                if (pl.k64)
                    CU(launch_keybuild64(c->pk, M, seed, g0, (int)Rc, rb, (uint64_t *)c->keysA.ptr,
                                         (uint32_t *)c->valsA.ptr, (uint8_t *)c->cnz.ptr, nullptr,
                                         nullptr, c->stream, &launches));
                else
                    CU(launch_keybuild32(c->pk, M, seed, g0, (int)Rc, rb, (uint32_t *)c->keysA.ptr,
                                         (uint32_t *)c->valsA.ptr, (uint8_t *)c->cnz.ptr, nullptr,
                                         nullptr, c->stream, &launches));
                tm.end();
                tm.begin(ST_SORT);
                if (pl.k64)
                    CU(radix_sort64((uint64_t *)c->keysA.ptr, (uint32_t *)c->valsA.ptr,
                                    (uint64_t *)c->keysB.ptr, (uint32_t *)c->valsB.ptr, Nc, bits,
                                    c->radix_tmp.ptr, &alt, c->stream, &launches));
                else
                    CU(radix_sort32((uint32_t *)c->keysA.ptr, (uint32_t *)c->valsA.ptr,
                                    (uint32_t *)c->keysB.ptr, (uint32_t *)c->valsB.ptr, Nc, bits,
                                    c->radix_tmp.ptr, &alt, c->stream, &launches));
                tm.end();
                void *ks = alt ? c->keysB.ptr : c->keysA.ptr;
                uint32_t *vs = (uint32_t *)(alt ? c->valsB.ptr : c->valsA.ptr);
                tm.begin(ST_JOIN);
                if (pl.k64)
                    CU(launch_join64((const uint64_t *)ks, Nc, M, rb, (const uint8_t *)c->cnz.ptr,
                                     (Bucket *)c->buckets.ptr, (uint64_t *)c->pair_counts.ptr,
                                     ctr_nbuckets(c), c->stream, &launches));
                else
                    CU(launch_join32((const uint32_t *)ks, Nc, M, rb, (const uint8_t *)c->cnz.ptr,
                                     (Bucket *)c->buckets.ptr, (uint64_t *)c->pair_counts.ptr,
                                     ctr_nbuckets(c), c->stream, &launches));
                CU(scan_u64_dev((const uint64_t *)c->pair_counts.ptr, (uint64_t *)c->pair_off.ptr,
                                ctr_nbuckets(c), bcap, ctr_total(c), ctr_cand(c), c->scan_tmp.ptr,
                                c->stream, &launches));
                tm.end();
                tm.begin(ST_VERIFY);
                CU(launch_verify(c->pk, (const Bucket *)c->buckets.ptr,
                                 (const uint64_t *)c->pair_off.ptr, ctr_nbuckets(c), ctr_total(c), vs,
                                 amin, pl.kbits, (uint64_t *)c->rec_keys.ptr,
                                 (uint32_t *)c->rec_agree.ptr, ctr_nrec(c), (uint32_t)c->rec_cap,
                                 c->stream, &launches, nullptr, nullptr, (uint32_t *)c->vstart.ptr,
                                 c->vstart_cap, ctr_err(c)));
                tm.end();
            }
        }
        if (enq)
            return XYZ_OK;
        // record count, candidates, errors, kept columns and the last group's
        // buckets -> host (already there when the spill flush read them last)
        if (!hc_fresh && (rc = read_counters()))
            return rc;
        const uint32_t nrec = hc[5];
        const uint64_t cand = (uint64_t)hc[10] | ((uint64_t)hc[11] << 32);
        const int err = (int)hc[7];
        const uint32_t nb_last = hc[0];
        unsigned long long kept[3];
        for (int i = 0; i < 3; ++i)
            kept[i] = (unsigned long long)hc[16 + 2 * i] | ((unsigned long long)hc[17 + 2 * i] << 32);
        if (err & 2)
            return fail(XYZ_ECUDA, "internal error: a candidate's offset lies outside its bucket");
        if (err)
            return fail(XYZ_ECUDA, "grouping table could not separate a partition's keys");
        if ((int64_t)nrec > c->rec_cap) {
            int64_t want = c->rec_cap;
            while (want < (int64_t)nrec)
                want *= 2;
            if (want > (int64_t)0xF0000000LL)
                return fail(XYZ_ENOMEM, "too many passing pairs for one search");
            c->rec_cap = want;
            if (phase == SP_FINISH)
                return SP_RERUN;
            continue;
        }
        tm.begin(ST_DEDUP);
        if (nrec > 0 && (int64_t)nrec <= unique_small_cap()) {
            CU(launch_unique_small((const uint64_t *)c->rec_keys.ptr, (const uint32_t *)c->rec_agree.ptr,
                                   (int64_t)nrec, pl.kbits, c->pk.n, (PairOut *)c->out.ptr, ctr_nout(c),
                                   c->stream, &launches, B > 1 ? (uint32_t *)c->resp.ptr : nullptr));
        } else if (nrec > 0) {
            bool alt = false;
            char *dt = (char *)c->dedup_tmp.ptr;
            size_t rt = radix_temp_bytes(c->rec_cap);
            CU(radix_sort64((uint64_t *)c->rec_keys.ptr, (uint32_t *)c->rec_agree.ptr,
                            (uint64_t *)c->rec_keys_alt.ptr, (uint32_t *)c->rec_agree_alt.ptr,
                            (int64_t)nrec, bbits + 2 * pl.kbits, dt, &alt, c->stream, &launches));
            const uint64_t *rk = (const uint64_t *)(alt ? c->rec_keys_alt.ptr : c->rec_keys.ptr);
            const uint32_t *ra = (const uint32_t *)(alt ? c->rec_agree_alt.ptr : c->rec_agree.ptr);
            CU(launch_unique(rk, ra, ctr_nrec(c), c->rec_cap, pl.kbits, c->pk.n,
                             (uint32_t *)c->flags.ptr, (uint32_t *)c->pos.ptr, dt + rt,
                             (PairOut *)c->out.ptr, ctr_nout(c), c->stream, &launches,
                             B > 1 ? (uint32_t *)c->resp.ptr : nullptr));
        }
        tm.end();
        if (c->pk.Xcs && nrec > 0)
            CU(launch_real_strengths(c->pk, (PairOut *)c->out.ptr, ctr_nout(c), (int64_t)nrec, c->stream,
                                     &launches));
        else if (c->pk.cdf && nrec > 0)
            CU(launch_weighted_strengths(c->pk, (PairOut *)c->out.ptr, ctr_nout(c), (int64_t)nrec, c->stream,
                                         &launches));
        // the output count, and, when the records are few, the output
        // itself (at most nrec pairs), under one synchronisation
        uint32_t nout = 0;
        c->hout_n = -1;
        if (nrec > 0) {
            const bool stage = (int64_t)nrec <= HOUT_MAX;
            CU(cudaMemcpyAsync(&nout, ctr_nout(c), 4, cudaMemcpyDeviceToHost, c->stream));
            if (stage) {
                c->hout.resize(nrec);
                CU(cudaMemcpyAsync(c->hout.data(), c->out.ptr, (size_t)nrec * sizeof(PairOut), cudaMemcpyDeviceToHost,
                                   c->stream));
                if (B > 1) {
                    c->hresp.resize(nrec);
                    CU(cudaMemcpyAsync(c->hresp.data(), c->resp.ptr, (size_t)nrec * 4, cudaMemcpyDeviceToHost,
                                       c->stream));
                }
            }
            CU(cudaStreamSynchronize(c->stream));
            if (stage)
                c->hout_n = nout;
        }
        st.attempts = attempt + 1;
        st.filter_kept = pl.filter ? (int64_t)kept[0] : 0;
        st.bucket_members = pl.filter ? (int64_t)kept[1] : 0;
        st.segment_grouped_runs = pl.filter ? (int64_t)kept[2] : 0;
        st.runs = runs;
        st.chunks = chunks;
        st.runs_per_chunk = pl.R;
        st.candidates = (int64_t)cand;
        st.passing = nrec;
        st.unique_pairs = nout;
        st.key_bits = pl.part ? M : key_bits_max;
        st.sort_passes = pl.part ? 0 : radix_passes(key_bits_max);
        st.survivors = pl.filter ? surv_total : runs * c->pk.p;
        st.gpu_launches = launches;
        tm.collect(st);
        st.buckets = nb_last;
        c->stats = st;
        *nout_host = nout;
        return XYZ_OK;
    }
    return fail(XYZ_ENOMEM, "search buffers kept overflowing");
}

// The last search's n output pairs (and, with resp_dst, their responses)
// into host memory: from the copy the search took, else from the device.
int copy_pairs(xyz_ctx *c, int64_t n, void *dst, uint32_t *resp_dst = nullptr)
{
    if (n <= 0)
        return XYZ_OK;
    if (c->hout_n == n && (!resp_dst || c->hresp.size() >= (size_t)n)) {
        std::memcpy(dst, c->hout.data(), (size_t)n * sizeof(PairOut));
        if (resp_dst)
            std::memcpy(resp_dst, c->hresp.data(), (size_t)n * 4);
        return XYZ_OK;
    }
    CU(cudaMemcpyAsync(dst, c->out.ptr, (size_t)n * sizeof(PairOut), cudaMemcpyDeviceToHost, c->stream));
    if (resp_dst)
        CU(cudaMemcpyAsync(resp_dst, c->resp.ptr, (size_t)n * 4, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return XYZ_OK;
}

int run_search(xyz_ctx *c, int64_t l0, int64_t l1, int M, int64_t amin, uint64_t seed,
               int64_t *nout_host)
{
    return run_search_multi(c, c->pk.yb, 1, l0, l1, M, amin, seed, nout_host);
}

int check_ctx(const xyz_ctx *c)
{
    if (!c)
        return fail(XYZ_EINVAL, "null context");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess)
        return fail(XYZ_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    return XYZ_OK;
}

int check_M(int M)
{
    if (M < 0 || M > XYZ_MAX_M)
        return fail(XYZ_EINVAL, "M must be in [0, 64]");
    return XYZ_OK;
}

int check_kappa(double kappa)
{
    if (!std::isfinite(kappa) || kappa < -1.0 || kappa > 1.0)
        return fail(XYZ_EINVAL, "kappa must be finite and in [-1, 1]");
    return XYZ_OK;
}

int create_common(const int8_t *dX, const int8_t *dY, int64_t n, int64_t p, cudaStream_t stream,
                  bool own_stream, xyz_ctx *c)
{
    c->stream = stream;
    c->own_stream = own_stream;
    Packed &pk = c->pk;
    pk.n = n;
    pk.p = p;
    pk.W = (n + 31) / 32;
    pk.Wp = (pk.W + 3) / 4 * 4;
    pk.P = (p + 31) / 32;
    pk.Pp = (pk.P + 7) / 8 * 8;
    size_t bXc = (size_t)p * pk.Wp * 4, bXr = (size_t)n * pk.Pp * 4, byb = (size_t)pk.Wp * 4;
    int rc;
    if ((rc = ensure(c->pXc, bXc)) || (rc = ensure(c->pXr, bXr)) || (rc = ensure(c->pyb, byb)) ||
        (rc = ensure(c->pbad, 16)))
        return rc;
    pk.Xc = (uint32_t *)c->pXc.ptr;
    pk.Xr = (uint32_t *)c->pXr.ptr;
    pk.yb = (uint32_t *)c->pyb.ptr;
    c->d_bad = (int *)c->pbad.ptr;
    c->packed_bytes = (int64_t)(bXc + bXr + byb);
    CU(cudaMemsetAsync(c->d_bad, 0, 16, stream));
    int64_t launches = 0;
    CU(launch_pack(dX, dY, pk, c->d_bad, stream, &launches));
    int bad = 0;
    CU(cudaMemcpyAsync(&bad, c->d_bad, 4, cudaMemcpyDeviceToHost, stream));
    CU(cudaStreamSynchronize(stream));
    if (bad)
        return fail(XYZ_EINVAL, "entries of X and Y must be -1 or +1");
    return XYZ_OK;
}

void destroy_ctx(xyz_ctx *c)
{
    if (!c)
        return;
    cudaSetDevice(c->device);
    if (c->stream)
        cudaStreamSynchronize(c->stream);
    if (c->owns_packed) {                 // packed X, response bits and flag: cached blocks
        release(c->pXc);
        release(c->pXr);
        release(c->pyb);
        release(c->pbad);
    } else {
        cudaFree(c->d_bad);
    }
    DevBuf *all[] = {&c->keysA,   &c->keysB,       &c->valsA,     &c->valsB,    &c->radix_tmp,
                     &c->cnz,     &c->buckets,     &c->pair_counts, &c->pair_off, &c->scan_tmp,
                     &c->counters, &c->rec_keys,   &c->rec_keys_alt, &c->rec_agree,
                     &c->rec_agree_alt, &c->flags, &c->pos,       &c->out,      &c->dedup_tmp,
                     &c->raw,     &c->ents,        &c->seg,       &c->members,  &c->kc_scratch, &c->lst_keys, &c->lst_cols,
                     &c->seg_keys, &c->seg_vals,   &c->seg_count, &c->buckets2, &c->pair_counts2,
                     &c->pair_off2, &c->scan_tmp2, &c->resp,   &c->ybs, &c->y_alt, &c->y_stage,
                     &c->wq, &c->wcdf, &c->wplanes, &c->wq2, &c->wcdf2, &c->wplanes2,
                     &c->wmeta, &c->wscan, &c->yreal,
                     &c->xrs, &c->xcs, &c->xnu, &c->ypr, &c->ysd, &c->ysd2, &c->rbad, &c->vstart};
    for (DevBuf *b : all)
        release(*b);
    if (c->own_stream && c->stream)
        cudaStreamDestroy(c->stream);
    delete c;
}

// Device address of a host pointer that lies in page-locked memory mapped
// into the device's address space, else null (pageable memory, or any
// error, which is cleared).
const void *mapped_device_ptr(const void *h)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

int check_dims(int64_t n, int64_t p)
{
    if (n < 1 || n >= ((int64_t)1 << 31))
        return fail(XYZ_EINVAL, "n must be in [1, 2^31)");
    if (p < 2 || p >= ((int64_t)1 << 31))
        return fail(XYZ_EINVAL, "p must be in [2, 2^31)");
    return XYZ_OK;
}

}  // namespace

// ================================================================ C ABI

extern "C" {

const char *xyz_last_error(void) { return g_err.c_str(); }

int xyz_create_dev(const int8_t *dX, const int8_t *dY, int64_t n, int64_t p, void *stream,
                   xyz_ctx **out)
{
    if (!dX || !dY || !out)
        return fail(XYZ_EINVAL, "null pointer argument");
    int rc = check_dims(n, p);
    if (rc)
        return rc;
    xyz_ctx *c = new (std::nothrow) xyz_ctx();
    if (!c)
        return fail(XYZ_ENOMEM, "host allocation failed");
    std::memset(&c->stats, 0, sizeof(c->stats));
    cudaGetDevice(&c->device);
    cudaStream_t s = (cudaStream_t)stream;
    bool own = false;
    if (!s) {
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return fail(XYZ_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
        }
        own = true;
    }
    rc = create_common(dX, dY, n, p, s, own, c);
    if (rc) {
        std::string msg = g_err;
        destroy_ctx(c);
        g_err = msg;
        return rc;
    }
    *out = c;
    g_err.clear();
    return XYZ_OK;
}

int xyz_create_sign(const float *X, int64_t n, int64_t p, uint64_t coin_seed, xyz_ctx **out)
{
    if (!X || !out)
        return fail(XYZ_EINVAL, "null pointer argument");
    int rc = check_dims(n, p);
    if (rc)
        return rc;
    const size_t count = (size_t)n * (size_t)p;
    float *dXf = nullptr;
    int8_t *dX8 = nullptr, *dY = nullptr;
    int *dbad = nullptr;
    cudaStream_t s = nullptr;
    auto cleanup = [&]() {
        cudaFree(dXf);
        cudaFree(dX8);
        cudaFree(dY);
        cudaFree(dbad);
        if (s)
            cudaStreamDestroy(s);
    };
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaMalloc(&dXf, count * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&dX8, count);
    if (e == cudaSuccess)
        e = cudaMalloc(&dY, (size_t)n);
    if (e == cudaSuccess)
        e = cudaMalloc(&dbad, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(XYZ_ENOMEM, std::string("staging of a real X: ") + cudaGetErrorString(e));
    }
    int64_t launches = 0;
    int bad = 0;
    e = cudaMemcpyAsync(dXf, X, count * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(dY, 1, (size_t)n, s);          // default response: all +1
    if (e == cudaSuccess)
        e = launch_sign_transform(dXf, (int64_t)count, coin_seed, dX8, dbad, s, &launches);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cleanup();
        return fail(XYZ_ECUDA, std::string("sign transform: ") + cudaGetErrorString(e));
    }
    if (bad) {
        cleanup();
        return fail(XYZ_EINVAL, "entries of X must not be NaN");
    }
    rc = xyz_create_dev(dX8, dY, n, p, nullptr, out);
    cleanup();
    return rc;
}

int xyz_create_unbiased(const float *X, const double *Y, int64_t n, int64_t p, xyz_ctx **out)
{
    if (!X || !Y || !out)
        return fail(XYZ_EINVAL, "null pointer argument");
    int rc = check_dims(n, p);
    if (rc)
        return rc;
    xyz_ctx *c = nullptr;
    if ((rc = xyz_create_sign(X, n, p, 0, &c)))      // packed sign bits: the binary view of X
        return rc;
    const int64_t Pf = (p + 31) / 32 * 32, Wf = (n + 31) / 32 * 32;
    const size_t count = (size_t)n * (size_t)p;
    DevBuf dX, dY;
    auto bail = [&](int code) {
        release(dX);
        release(dY);
        std::string msg = g_err;
        destroy_ctx(c);
        g_err = msg;
        return code;
    };
    if ((rc = ensure(dX, count * sizeof(float))) || (rc = ensure(dY, (size_t)n * 8)) ||
        (rc = ensure(c->xrs, (size_t)n * Pf * sizeof(float))) ||
        (rc = ensure(c->xcs, (size_t)p * Wf * sizeof(float))) || (rc = ensure(c->xnu, (size_t)n * 4)) ||
        (rc = ensure(c->ysd, (size_t)Wf * 12)) || (rc = ensure(c->rbad, 16)))
        return bail(rc);
    int64_t launches = 0;
    unsigned bad = 0;
    cudaError_t e = cudaMemcpyAsync(dX.ptr, X, count * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dY.ptr, Y, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = launch_unbiased_scale((const float *)dX.ptr, n, p, Pf, Wf, (float *)c->xrs.ptr, (float *)c->xcs.ptr,
                                  (float *)c->xnu.ptr, (unsigned *)c->rbad.ptr, c->stream, &launches);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&bad, c->rbad.ptr, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        fail(XYZ_ECUDA, std::string("scaling a real X: ") + cudaGetErrorString(e));
        return bail(XYZ_ECUDA);
    }
    if (bad) {
        fail(XYZ_EINVAL, "entries of X must not be NaN");
        return bail(XYZ_EINVAL);
    }
    c->pk.Xrs = (const float *)c->xrs.ptr;
    c->pk.Pf = Pf;
    c->pk.Xcs = (const float *)c->xcs.ptr;
    c->pk.Wf = Wf;
    c->pk.ysd = (const double *)c->ysd.ptr;
    if ((rc = xyz_set_y_real_dev(c, (const double *)dY.ptr)))
        return bail(rc);
    release(dX);
    release(dY);
    *out = c;
    return XYZ_OK;
}

int xyz_create(const int8_t *X, const int8_t *Y, int64_t n, int64_t p, xyz_ctx **out)
{
    if (!X || !Y || !out)
        return fail(XYZ_EINVAL, "null pointer argument");
    int rc = check_dims(n, p);
    if (rc)
        return rc;
    // Pinned host buffers that the device can address (mapped page-locked
    // memory): the pack kernel reads them directly, so the transfer and the
    // packing are one pass over X and no staging copy is made.
    const int8_t *mX = (const int8_t *)mapped_device_ptr(X), *mY = (const int8_t *)mapped_device_ptr(Y);
    if (mX && mY)
        return xyz_create_dev(mX, mY, n, p, nullptr, out);   // returns after the pack has run
    DevBuf sX, sY;                              // staging, from the block cache
    if ((rc = ensure(sX, (size_t)n * p)) || (rc = ensure(sY, (size_t)n))) {
        release(sX);
        return rc;
    }
    cudaError_t e;
    if ((e = cudaMemcpy(sX.ptr, X, (size_t)n * p, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(sY.ptr, Y, (size_t)n, cudaMemcpyHostToDevice)) != cudaSuccess) {
        release(sX);
        release(sY);
        return fail(XYZ_ECUDA, std::string("cudaMemcpy of X/Y: ") + cudaGetErrorString(e));
    }
    rc = xyz_create_dev((const int8_t *)sX.ptr, (const int8_t *)sY.ptr, n, p, nullptr, out);
    if (!rc)
        cudaStreamSynchronize((*out)->stream);  // packing read the staging buffers
    release(sX);
    release(sY);
    return rc;
}

int xyz_set_y_dev(xyz_ctx *ctx, const int8_t *dY)
{
    int rc = check_ctx(ctx);
    if (rc)
        return rc;
    if (ctx->pk.Xrs)
        return fail(XYZ_EINVAL, "a real X takes a real response (xyz_set_y_real)");
    if (!dY)
        return fail(XYZ_EINVAL, "null pointer argument");
    // pack into a second buffer first so a bad Y leaves the context unchanged
    const size_t bytes = (size_t)ctx->pk.Wp * 4;
    if ((rc = ensure(ctx->y_alt, bytes)))
        return rc;
    Packed tmp = ctx->pk;
    tmp.yb = (uint32_t *)ctx->y_alt.ptr;
    int64_t launches = 0;
    CU(cudaMemsetAsync(ctx->d_bad, 0, 16, ctx->stream));
    CU(launch_pack_y(dY, tmp, ctx->d_bad, ctx->stream, &launches));
    int bad = 0;
    CU(cudaMemcpyAsync(&bad, ctx->d_bad, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (bad)
        return fail(XYZ_EINVAL, "entries of Y must be -1 or +1");
    CU(cudaMemcpyAsync(ctx->pk.yb, ctx->y_alt.ptr, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->pk.cdf = nullptr;               // binary response: uniform rows, plain agreement
    ctx->pk.planes = nullptr;
    ctx->pk.wtotal = 0;
    return XYZ_OK;
}

int xyz_set_y_real_dev(xyz_ctx *ctx, const double *dY)
{
    int rc = check_ctx(ctx);
    if (rc)
        return rc;
    if (!dY)
        return fail(XYZ_EINVAL, "null pointer argument");
    if (!ctx->owns_packed)
        return fail(XYZ_EINVAL, "context does not own its response");
    const int64_t n = ctx->pk.n, Wp = ctx->pk.Wp;
    if (ctx->pk.Xrs) {
        // real X: the response of the scaled rows, Y'_i = Y_i nu_i^2 (its
        // padded copy goes to a second buffer, swapped in once Y' is accepted)
        int64_t launches = 0;
        if ((rc = ensure(ctx->ypr, (size_t)n * 8)) || (rc = ensure(ctx->ysd2, (size_t)ctx->pk.Wf * 12)))
            return rc;
        CU(launch_unbiased_y(dY, (const float *)ctx->xnu.ptr, n, ctx->pk.Wf, (double *)ctx->ypr.ptr,
                             (double *)ctx->ysd2.ptr, ctx->stream, &launches));
        dY = (const double *)ctx->ypr.ptr;
    }
    if ((rc = ensure(ctx->y_alt, (size_t)Wp * 4)) || (rc = ensure(ctx->wq2, (size_t)n * 8)) ||
        (rc = ensure(ctx->wcdf2, (size_t)n * 8)) ||
        (rc = ensure(ctx->wplanes2, (size_t)Wp * XYZ_WPLANES * 4)) || (rc = ensure(ctx->wmeta, 64)) ||
        (rc = ensure(ctx->wscan, weights_scan_bytes(n))))
        return rc;
    char *meta = (char *)ctx->wmeta.ptr;      // [0] max bits, [8] bad flag, [16] total
    int64_t launches = 0;
    CU(launch_prepare_weights(dY, n, Wp, (uint64_t *)ctx->wq2.ptr, (uint32_t *)ctx->y_alt.ptr,
                              (uint32_t *)ctx->wplanes2.ptr, (uint64_t *)ctx->wcdf2.ptr,
                              (uint64_t *)(meta + 16), (unsigned long long *)meta, (int *)(meta + 8),
                              ctx->wscan.ptr, ctx->stream, &launches));
    uint64_t host[3] = {0, 0, 0};
    CU(cudaMemcpyAsync(host, meta, 24, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if ((host[1] & 0xFFFFFFFFu) || host[0] == 0)
        return fail(XYZ_EINVAL, "entries of a real Y must be finite and not all zero");
    CU(cudaMemcpyAsync(ctx->pk.yb, ctx->y_alt.ptr, (size_t)Wp * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    std::swap(ctx->wq, ctx->wq2);
    std::swap(ctx->wcdf, ctx->wcdf2);
    std::swap(ctx->wplanes, ctx->wplanes2);
    if (ctx->pk.Xrs) {
        std::swap(ctx->ysd, ctx->ysd2);
        ctx->pk.ysd = (const double *)ctx->ysd.ptr;
    }
    ctx->pk.cdf = (const uint64_t *)ctx->wcdf.ptr;
    ctx->pk.planes = (const uint32_t *)ctx->wplanes.ptr;
    ctx->pk.wtotal = host[2];
    double maxabs = 0.0;
    std::memcpy(&maxabs, &host[0], 8);
    std::frexp(maxabs, &ctx->w_exp);
    if (ctx->pk.Xrs) {
        // ||Y'||_1 in double, rows in order
        std::vector<double> yp((size_t)n);
        CU(cudaMemcpyAsync(yp.data(), dY, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        double s1 = 0.0;
        for (int64_t i = 0; i < n; ++i)
            s1 += std::fabs(yp[(size_t)i]);
        ctx->pk.rnorm = s1;
    }
    return XYZ_OK;
}

int xyz_set_y_real(xyz_ctx *ctx, const double *Y)
{
    int rc = check_ctx(ctx);
    if (rc)
        return rc;
    if (!Y)
        return fail(XYZ_EINVAL, "null pointer argument");
    if ((rc = ensure(ctx->yreal, (size_t)ctx->pk.n * 8)))
        return rc;
    CU(cudaMemcpyAsync(ctx->yreal.ptr, Y, (size_t)ctx->pk.n * 8, cudaMemcpyHostToDevice, ctx->stream));
    return xyz_set_y_real_dev(ctx, (const double *)ctx->yreal.ptr);
}

int xyz_set_y(xyz_ctx *ctx, const int8_t *Y)
{
    int rc = check_ctx(ctx);
    if (rc)
        return rc;
    if (!Y)
        return fail(XYZ_EINVAL, "null pointer argument");
    if ((rc = ensure(ctx->y_stage, (size_t)ctx->pk.n)))
        return rc;
    CU(cudaMemcpyAsync(ctx->y_stage.ptr, Y, (size_t)ctx->pk.n, cudaMemcpyHostToDevice, ctx->stream));
    return xyz_set_y_dev(ctx, (const int8_t *)ctx->y_stage.ptr);
}

void xyz_destroy(xyz_ctx *ctx) { destroy_ctx(ctx); }

int xyz_info(const xyz_ctx *ctx, int64_t *n, int64_t *p, int64_t *device_bytes)
{
    if (!ctx)
        return fail(XYZ_EINVAL, "null context");
    if (n)
        *n = ctx->pk.n;
    if (p)
        *p = ctx->pk.p;
    if (device_bytes)
        *device_bytes = ctx->packed_bytes + ws_bytes(ctx);
    return XYZ_OK;
}

int xyz_search_range(xyz_ctx *ctx, int64_t l0, int64_t l1, int32_t M, double kappa, uint64_t seed,
                     xyz_pair **pairs, int64_t *npairs)
{
    int rc = check_ctx(ctx);
    if (rc)
        return rc;
    if (!pairs || !npairs)
        return fail(XYZ_EINVAL, "null output pointer");
    if (l0 < 0 || l1 <= l0)
        return fail(XYZ_EINVAL, "need 0 <= l0 < l1");
    if ((rc = check_M(M)) || (rc = check_kappa(kappa)))
        return rc;
    const int64_t amin = amin_rule(ctx->pk.n, kappa);
    int64_t nout = 0;
    set_kappa(ctx, kappa);
    if (amin > ctx->pk.n && !ctx->pk.cdf) {
        std::memset(&ctx->stats, 0, sizeof(ctx->stats));
        *pairs = nullptr;
        *npairs = 0;
        return XYZ_OK;
    }
    rc = run_search(ctx, l0, l1, M, amin, seed, &nout);
    if (rc)
        return rc;
    xyz_pair *host = nullptr;
    if (nout > 0) {
        host = (xyz_pair *)std::malloc((size_t)nout * sizeof(xyz_pair));
        if (!host)
            return fail(XYZ_ENOMEM, "host allocation of results failed");
        if ((rc = copy_pairs(ctx, nout, host))) {
            std::free(host);
            return rc;
        }
    }
    *pairs = host;
    *npairs = nout;
    return XYZ_OK;
}

int xyz_brute_force(xyz_ctx *ctx, double kappa, xyz_pair **pairs, int64_t *npairs)
{
    int rc = check_ctx(ctx);
    if (rc)
        return rc;
    if (!pairs || !npairs)
        return fail(XYZ_EINVAL, "null output pointer");
    if ((rc = check_kappa(kappa)))
        return rc;
    xyz_ctx *c = ctx;
    if (c->pk.cdf)
        return fail(XYZ_EINVAL, "the exhaustive screen takes a binary response");
    const int64_t amin = amin_rule(c->pk.n, kappa);
    std::memset(&c->stats, 0, sizeof(c->stats));
    *pairs = nullptr;
    *npairs = 0;
    if (amin > c->pk.n)
        return XYZ_OK;
    const int kbits = ceil_log2(c->pk.p) < 1 ? 1 : ceil_log2(c->pk.p);
    for (int attempt = 0; attempt < 8; ++attempt) {
        if ((rc = ensure_records(c, 1)) || (rc = ensure(c->counters, 128)))
            return rc;
        int64_t launches = 0;
        CU(cudaMemsetAsync(c->counters.ptr, 0, 128, c->stream));
        CU(launch_brute(c->pk, amin, kbits, (uint64_t *)c->rec_keys.ptr, (uint32_t *)c->rec_agree.ptr,
                        ctr_nrec(c), (uint32_t)c->rec_cap, c->stream, &launches));
        uint32_t nrec = 0;
        CU(cudaMemcpyAsync(&nrec, ctr_nrec(c), 4, cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        if ((int64_t)nrec > c->rec_cap) {
            int64_t want = c->rec_cap;
            while (want < (int64_t)nrec)
                want *= 2;
            if (want > (int64_t)0xF0000000LL)
                return fail(XYZ_ENOMEM, "too many passing pairs");
            c->rec_cap = want;
            continue;
        }
        uint32_t nout = 0;
        if (nrec > 0 && (int64_t)nrec <= unique_small_cap()) {
            CU(launch_unique_small((const uint64_t *)c->rec_keys.ptr, (const uint32_t *)c->rec_agree.ptr,
                                   (int64_t)nrec, kbits, c->pk.n, (PairOut *)c->out.ptr, ctr_nout(c), c->stream,
                                   &launches));
            CU(cudaMemcpyAsync(&nout, ctr_nout(c), 4, cudaMemcpyDeviceToHost, c->stream));
            CU(cudaStreamSynchronize(c->stream));
        } else if (nrec > 0) {
            // order the passing pairs by (j, k)
            bool alt = false;
            char *dt = (char *)c->dedup_tmp.ptr;
            size_t rt = radix_temp_bytes(c->rec_cap);
            CU(radix_sort64((uint64_t *)c->rec_keys.ptr, (uint32_t *)c->rec_agree.ptr,
                            (uint64_t *)c->rec_keys_alt.ptr, (uint32_t *)c->rec_agree_alt.ptr, (int64_t)nrec,
                            2 * kbits, dt, &alt, c->stream, &launches));
            const uint64_t *rk = (const uint64_t *)(alt ? c->rec_keys_alt.ptr : c->rec_keys.ptr);
            const uint32_t *ra = (const uint32_t *)(alt ? c->rec_agree_alt.ptr : c->rec_agree.ptr);
            CU(launch_unique(rk, ra, ctr_nrec(c), c->rec_cap, kbits, c->pk.n, (uint32_t *)c->flags.ptr,
                             (uint32_t *)c->pos.ptr, dt + rt, (PairOut *)c->out.ptr, ctr_nout(c), c->stream,
                             &launches));
            CU(cudaMemcpyAsync(&nout, ctr_nout(c), 4, cudaMemcpyDeviceToHost, c->stream));
            CU(cudaStreamSynchronize(c->stream));
        }
        xyz_pair *host = nullptr;
        if (nout > 0) {
            host = (xyz_pair *)std::malloc((size_t)nout * sizeof(xyz_pair));
            if (!host)
                return fail(XYZ_ENOMEM, "host allocation of results failed");
            cudaError_t e = cudaMemcpyAsync(host, c->out.ptr, (size_t)nout * sizeof(xyz_pair),
                                            cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess)
                e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) {
                std::free(host);
                return fail(XYZ_ECUDA, std::string("copy of results: ") + cudaGetErrorString(e));
            }
        }
        c->stats.candidates = c->pk.p * (c->pk.p - 1) / 2;
        c->stats.passing = nrec;
        c->stats.unique_pairs = nout;
        c->stats.gpu_launches = launches;
        *pairs = host;
        *npairs = nout;
        return XYZ_OK;
    }
    return fail(XYZ_ENOMEM, "result buffers kept overflowing");
}

namespace {

// One search over runs [0, L) whose pass threshold is already on the context
// (amin, or pk.wkq for a real response); results appended to `out`.
int search_collect(xyz_ctx *c, int32_t L, int32_t M, int64_t amin, uint64_t seed, std::vector<xyz_pair> &out)
{
    int64_t nout = 0;
    int rc = run_search(c, 0, L, M, amin, seed, &nout);
    if (rc)
        return rc;
    const size_t at = out.size();
    out.resize(at + (size_t)nout);
    return copy_pairs(c, nout, out.data() + at);
}

// Both signs of the response (Section 4 runs xyz with Y set to +r and -r):
// the second search runs on flipped sign bits; its pairs are reported for
// +Y (agree -> n - agree, strength -> -strength) and united with the first
// search's, each pair once, sorted by (j, k).
int search_both_signs(xyz_ctx *c, int32_t L, int32_t M, int64_t amin_plus, int64_t amin_minus, uint64_t seed,
                      xyz_pair **pairs, int64_t *npairs)
{
    std::vector<xyz_pair> plus, minus;
    int rc = search_collect(c, L, M, amin_plus, seed, plus);
    if (rc)
        return rc;
    int64_t launches = 0;
    CU(launch_flip_signs(c->pk, c->stream, &launches));
    rc = search_collect(c, L, M, amin_minus, seed, minus);
    cudaError_t e = launch_flip_signs(c->pk, c->stream, &launches);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    if (rc)
        return rc;
    if (e != cudaSuccess)
        return fail(XYZ_ECUDA, std::string("restoring the response signs: ") + cudaGetErrorString(e));
    for (xyz_pair &q : minus) {
        q.agree = (int32_t)c->pk.n - q.agree;
        q.strength = -q.strength;
    }
    std::vector<xyz_pair> all;
    all.reserve(plus.size() + minus.size());
    size_t a = 0, b = 0;
    auto less = [](const xyz_pair &x, const xyz_pair &y) { return x.j != y.j ? x.j < y.j : x.k < y.k; };
    while (a < plus.size() || b < minus.size()) {
        if (b == minus.size() || (a < plus.size() && less(plus[a], minus[b])))
            all.push_back(plus[a++]);
        else if (a == plus.size() || less(minus[b], plus[a]))
            all.push_back(minus[b++]);
        else {
            all.push_back(plus[a++]);      // in both (kappa <= 0): the +Y result
            ++b;
        }
    }
    xyz_pair *host = nullptr;
    if (!all.empty()) {
        host = (xyz_pair *)std::malloc(all.size() * sizeof(xyz_pair));
        if (!host)
            return fail(XYZ_ENOMEM, "host allocation of results failed");
        std::memcpy(host, all.data(), all.size() * sizeof(xyz_pair));
    }
    *pairs = host;
    *npairs = (int64_t)all.size();
    return XYZ_OK;
}

}  // namespace

int xyz_search_abs(xyz_ctx *ctx, int32_t L, int32_t M, double kappa, uint64_t seed, xyz_pair **pairs,
                   int64_t *npairs)
{
    int rc = check_ctx(ctx);
    if (rc)
        return rc;
    if (!pairs || !npairs)
        return fail(XYZ_EINVAL, "null output pointer");
    if (L < 1)
        return fail(XYZ_EINVAL, "L must be >= 1");
    if ((rc = check_M(M)) || (rc = check_kappa(kappa)))
        return rc;
    if (!ctx->owns_packed || ctx->pk.Xrs)
        return fail(XYZ_EINVAL, "needs a binary X on a context that owns its response");
    const int64_t amin = amin_rule(ctx->pk.n, kappa);
    set_kappa(ctx, kappa);
    *pairs = nullptr;
    *npairs = 0;
    if (amin > ctx->pk.n && !ctx->pk.cdf)
        return XYZ_OK;
    return search_both_signs(ctx, L, M, amin, amin, seed, pairs, npairs);
}

int xyz_kkt_screen(xyz_ctx *ctx, const double *r, double lambda, int32_t L, int32_t M, uint64_t seed,
                   xyz_pair **pairs, int64_t *npairs)
{
    int rc = check_ctx(ctx);
    if (rc)
        return rc;
    if (!pairs || !npairs || !r)
        return fail(XYZ_EINVAL, "null pointer argument");
    if (L < 1)
        return fail(XYZ_EINVAL, "L must be >= 1");
    if (!(lambda >= 0.0) || !std::isfinite(lambda))
        return fail(XYZ_EINVAL, "lambda must be finite and >= 0");
    if ((rc = check_M(M)))
        return rc;
    if (ctx->pk.Xrs)
        return fail(XYZ_EINVAL, "the KKT check takes a binary X");
    if ((rc = xyz_set_y_real(ctx, r)))
        return rc;
    // |r^T (X_j o X_k)| / n > lambda as the integer rule |2S - Q| >= t
    const double t = std::floor(std::ldexp(lambda * (double)ctx->pk.n, 24 - ctx->w_exp)) + 1.0;
    ctx->pk.wkq = t;
    ctx->pk.wscale = std::ldexp(1.0, ctx->w_exp - 24) / (double)ctx->pk.n;
    *pairs = nullptr;
    *npairs = 0;
    rc = search_both_signs(ctx, L, M, 0, 0, seed, pairs, npairs);
    ctx->pk.wscale = 0.0;
    return rc;
}

int xyz_autotune_M(xyz_ctx *ctx, double kappa, double gamma, double recall, int32_t M_lo, int32_t M_hi,
                   uint64_t seed, int64_t trial_runs, int32_t *M_best, int64_t *L_best, double *ms_best,
                   double *table)
{
    int rc = check_ctx(ctx);
    if (rc)
        return rc;
    if (!M_best || !L_best || !ms_best)
        return fail(XYZ_EINVAL, "null output pointer");
    if ((rc = check_kappa(kappa)))
        return rc;
    if (!(gamma > 0.0 && gamma < 1.0) || !(recall > 0.0 && recall < 1.0))
        return fail(XYZ_EINVAL, "need 0 < gamma < 1 and 0 < recall < 1");
    if (M_lo < 1 || M_hi < M_lo || M_hi > XYZ_MAX_M || trial_runs < 8)
        return fail(XYZ_EINVAL, "need 1 <= M_lo <= M_hi <= 64 and trial_runs >= 8");
    const int64_t amin = amin_rule(ctx->pk.n, kappa);
    set_kappa(ctx, kappa);
    const bool timing = ctx->timing;
    ctx->timing = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = -1.0;
    int32_t bestM = 0;
    int64_t bestL = 0;
    for (int32_t M = M_lo; M <= M_hi; ++M) {
        const int64_t L = xyz_runs_for_recall(std::pow(gamma, (double)M), recall);
        double pred = -1.0;
        if (L > 0 && L < ((int64_t)1 << 40)) {
            // time on the device: a + b * runs from two trial lengths
            const int64_t r2 = L < trial_runs ? L : trial_runs;
            const int64_t r1 = r2 / 4 > 0 ? r2 / 4 : 1;
            int64_t nout = 0;
            double t[2] = {0.0, 0.0};
            const int64_t rr[2] = {r1, r2};
            if ((rc = run_search(ctx, 0, r1, M, amin, seed, &nout)))      // warm-up: workspace growth
                break;
            for (int i = 0; i < 2 && !rc; ++i) {
                cudaEventRecord(e0, ctx->stream);
                rc = run_search(ctx, 0, rr[i], M, amin, seed + 1 + (uint64_t)i, &nout);
                cudaEventRecord(e1, ctx->stream);
                cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                t[i] = ms;
            }
            if (rc)
                break;
            if (L <= trial_runs) {
                pred = t[1];
            } else {
                const double b = r2 > r1 ? (t[1] - t[0]) / (double)(r2 - r1) : t[1] / (double)r2;
                const double a = t[1] - b * (double)r2;
                pred = (a > 0.0 ? a : 0.0) + (b > 0.0 ? b : t[1] / (double)r2) * (double)L;
            }
            if (best < 0.0 || pred < best) {
                best = pred;
                bestM = M;
                bestL = L;
            }
        }
        if (table) {
            table[3 * (M - M_lo) + 0] = (double)M;
            table[3 * (M - M_lo) + 1] = (double)L;
            table[3 * (M - M_lo) + 2] = pred;
        }
    }
    // confirm: the two best predictions, when they are short enough, are
    // timed as full searches (after a warm-up that sizes their buffers)
    if (!rc && best >= 0.0 && table) {
        int32_t cand[2] = {bestM, -1};
        double second = -1.0;
        for (int32_t M = M_lo; M <= M_hi; ++M) {
            const double pr = table[3 * (M - M_lo) + 2];
            if (M != bestM && pr >= 0.0 && (second < 0.0 || pr < second)) {
                second = pr;
                cand[1] = M;
            }
        }
        double bestMeasured = -1.0;
        for (int i = 0; i < 2 && !rc; ++i) {
            const int32_t M = cand[i];
            if (M < 0 || table[3 * (M - M_lo) + 2] > 200.0)
                continue;
            const int64_t L = (int64_t)table[3 * (M - M_lo) + 1];
            int64_t nout = 0;
            if ((rc = run_search(ctx, 0, L, M, amin, seed + 7, &nout)))
                break;
            cudaEventRecord(e0, ctx->stream);
            rc = run_search(ctx, 0, L, M, amin, seed + 8, &nout);
            cudaEventRecord(e1, ctx->stream);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            table[3 * (M - M_lo) + 2] = ms;
            if (bestMeasured < 0.0 || ms < bestMeasured) {
                bestMeasured = ms;
                best = ms;
                bestM = M;
                bestL = L;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->timing = timing;
    if (rc)
        return rc;
    if (best < 0.0)
        return fail(XYZ_EINVAL, "no M in the range reaches the recall with fewer than 2^40 runs");
    *M_best = bestM;
    *L_best = bestL;
    *ms_best = best;
    return XYZ_OK;
}

int xyz_search_many(xyz_ctx **ctxs, int32_t count, const int32_t *L, const int32_t *M, const double *kappa,
                    const uint64_t *seed, xyz_pair **pairs, int64_t *offsets)
{
    if (!ctxs || !L || !M || !kappa || !seed || !pairs || !offsets || count < 1)
        return fail(XYZ_EINVAL, "null pointer argument or count < 1");
    int rc;
    std::vector<int64_t> amin((size_t)count);
    std::vector<char> live((size_t)count, 0);
    for (int32_t i = 0; i < count; ++i) {
        if ((rc = check_ctx(ctxs[i])))
            return rc;
        if (L[i] < 1 || (rc = check_M(M[i])) || (rc = check_kappa(kappa[i])))
            return rc ? rc : fail(XYZ_EINVAL, "L must be >= 1");
        for (int32_t j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i])
                return fail(XYZ_EINVAL, "each search needs its own context");
        if (ctxs[i]->device != ctxs[0]->device || !ctxs[i]->stream)
            return fail(XYZ_EINVAL, "contexts must share a device and own non-default streams");
        amin[(size_t)i] = amin_rule(ctxs[i]->pk.n, kappa[i]);
        set_kappa(ctxs[i], kappa[i]);
        live[(size_t)i] = amin[(size_t)i] <= ctxs[i]->pk.n || ctxs[i]->pk.cdf;
    }
    // 1. workspace of every search, before any capture
    int64_t nout = 0;
    for (int32_t i = 0; i < count; ++i)
        if (live[(size_t)i] &&
            (rc = run_search_multi(ctxs[i], ctxs[i]->pk.yb, 1, 0, L[i], M[i], amin[(size_t)i], seed[i], &nout,
                                   SP_PREPARE)))
            return rc;
    // searches of one launch group on the single-filter path share fused
    // filter launches, one per key class (in search order, at most
    // XYZ_FUSED_MAX each), on the capture stream between their own work
    std::vector<int> fclass((size_t)count, 0);
    int nfused = 0;
    for (int32_t i = 0; i < count; ++i)
        if (live[(size_t)i] && ctxs[i]->fuse_filters) {
            fclass[(size_t)i] = search_fusable(ctxs[i], L[i], M[i]);
            nfused += fclass[(size_t)i] != 0;
        }
    if (nfused < 2)
        std::fill(fclass.begin(), fclass.end(), 0);
    // 2. the launch groups of all searches, one stream each, captured into
    //    one graph that forks from and joins to a capture stream
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> ev((size_t)count + 2, nullptr);     // fork, one per search, fused filters done
    auto cleanup = [&]() {
        if (exec)
            cudaGraphExecDestroy(exec);
        if (graph)
            cudaGraphDestroy(graph);
        for (cudaEvent_t e : ev)
            if (e)
                cudaEventDestroy(e);
        if (cs)
            cudaStreamDestroy(cs);
    };
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (size_t i = 0; i < ev.size() && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess)
        e = cudaEventRecord(ev[0], cs);
    rc = XYZ_OK;
    if (nfused >= 2 && e == cudaSuccess) {
        // what precedes each fused search's filter, on its own stream
        std::vector<FilterArgs> args((size_t)count);
        std::vector<int32_t> order;
        for (int32_t i = 0; i < count && e == cudaSuccess && !rc; ++i) {
            if (!fclass[(size_t)i])
                continue;
            e = cudaStreamWaitEvent(ctxs[i]->stream, ev[0], 0);
            if (e == cudaSuccess)
                rc = run_search_multi(ctxs[i], ctxs[i]->pk.yb, 1, 0, L[i], M[i], amin[(size_t)i], seed[i], &nout,
                                      SP_ENQUEUE_PRE, &args[(size_t)i]);
            if (e == cudaSuccess && !rc)
                e = cudaEventRecord(ev[(size_t)i + 1], ctxs[i]->stream);
            if (e == cudaSuccess && !rc)
                e = cudaStreamWaitEvent(cs, ev[(size_t)i + 1], 0);
        }
        // the fused launches; each takes its work counter from its first search
        int64_t fl = 0;
        const int kcls[3] = {16, 24, 32};
        for (int k = 0; k < 3 && e == cudaSuccess && !rc; ++k) {
            std::vector<FilterArgs> batch;
            uint32_t *work = nullptr;
            for (int32_t i = 0; i <= count && e == cudaSuccess; ++i) {
                if (i < count && fclass[(size_t)i] == kcls[k]) {
                    if (!work)
                        work = ctr_work(ctxs[i]);
                    batch.push_back(args[(size_t)i]);
                }
                if (!batch.empty() && (i == count || (int)batch.size() == XYZ_FUSED_MAX)) {
                    e = cudaMemsetAsync(work, 0, 4, cs);
                    if (e == cudaSuccess)
                        e = launch_filter_fused(batch.data(), (int)batch.size(), kcls[k], filter_grid(),
                                                work, cs, &fl);
                    batch.clear();
                    work = nullptr;
                }
            }
        }
        if (e == cudaSuccess && !rc)
            e = cudaEventRecord(ev[(size_t)count + 1], cs);
        for (int32_t i = 0; i < count && e == cudaSuccess && !rc; ++i) {
            if (!fclass[(size_t)i])
                continue;
            e = cudaStreamWaitEvent(ctxs[i]->stream, ev[(size_t)count + 1], 0);
            if (e == cudaSuccess)
                rc = run_search_multi(ctxs[i], ctxs[i]->pk.yb, 1, 0, L[i], M[i], amin[(size_t)i], seed[i], &nout,
                                      SP_ENQUEUE_POST);
            if (e == cudaSuccess && !rc)
                e = cudaEventRecord(ev[(size_t)i + 1], ctxs[i]->stream);
            if (e == cudaSuccess && !rc)
                e = cudaStreamWaitEvent(cs, ev[(size_t)i + 1], 0);
        }
    }
    for (int32_t i = 0; i < count && e == cudaSuccess && !rc; ++i) {
        if (!live[(size_t)i] || fclass[(size_t)i])
            continue;
        e = cudaStreamWaitEvent(ctxs[i]->stream, ev[0], 0);
        if (e == cudaSuccess)
            rc = run_search_multi(ctxs[i], ctxs[i]->pk.yb, 1, 0, L[i], M[i], amin[(size_t)i], seed[i], &nout,
                                  SP_ENQUEUE);
        if (e == cudaSuccess && !rc)
            e = cudaEventRecord(ev[(size_t)i + 1], ctxs[i]->stream);
        if (e == cudaSuccess && !rc)
            e = cudaStreamWaitEvent(cs, ev[(size_t)i + 1], 0);
    }
    cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess)
        e = ec;
    if (e == cudaSuccess && !rc)
        e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess && !rc)
        e = cudaGraphLaunch(exec, cs);
    if (e == cudaSuccess && !rc)
        e = cudaStreamSynchronize(cs);
    cleanup();
    if (rc)
        return rc;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(XYZ_ECUDA, std::string("graph of launch groups: ") + cudaGetErrorString(e));
    }
    // 3. per search: spills and union (a search whose buffers overflowed is
    //    redone on its own), results in order
    std::vector<xyz_pair> acc;
    offsets[0] = 0;
    for (int32_t i = 0; i < count; ++i) {
        xyz_ctx *c = ctxs[i];
        int64_t no = 0;
        if (live[(size_t)i]) {
            rc = run_search_multi(c, c->pk.yb, 1, 0, L[i], M[i], amin[(size_t)i], seed[i], &no, SP_FINISH);
            if (rc == SP_RERUN)
                rc = run_search_multi(c, c->pk.yb, 1, 0, L[i], M[i], amin[(size_t)i], seed[i], &no, SP_ALL);
            if (rc)
                return rc;
        }
        const size_t at = acc.size();
        acc.resize(at + (size_t)no);
        if ((rc = copy_pairs(c, no, acc.data() + at)))
            return rc;
        offsets[i + 1] = offsets[i] + no;
    }
    xyz_pair *host = nullptr;
    if (!acc.empty()) {
        host = (xyz_pair *)std::malloc(acc.size() * sizeof(xyz_pair));
        if (!host)
            return fail(XYZ_ENOMEM, "host allocation of results failed");
        std::memcpy(host, acc.data(), acc.size() * sizeof(xyz_pair));
    }
    *pairs = host;
    return XYZ_OK;
}

int xyz_search(xyz_ctx *ctx, int32_t L, int32_t M, double kappa, uint64_t seed, xyz_pair **pairs,
               int64_t *npairs)
{
    if (L < 1)
        return fail(XYZ_EINVAL, "L must be >= 1");
    return xyz_search_range(ctx, 0, L, M, kappa, seed, pairs, npairs);
}

void xyz_free_pairs(xyz_pair *pairs) { std::free(pairs); }
void xyz_free(void *ptr) { std::free(ptr); }

int xyz_get_stats(const xyz_ctx *ctx, xyz_stats *out)
{
    if (!ctx || !out)
        return fail(XYZ_EINVAL, "null pointer argument");
    *out = ctx->stats;
    return XYZ_OK;
}

int xyz_set_timing(xyz_ctx *ctx, int enable)
{
    if (!ctx)
        return fail(XYZ_EINVAL, "null context");
    ctx->timing = enable != 0;
    return XYZ_OK;
}

int xyz_set_tiles(xyz_ctx *ctx, const xyz_tiles *tiles)
{
    if (!ctx || !tiles)
        return fail(XYZ_EINVAL, "null argument");
    const int ft = tiles->filter_threads;
    if (ft != 0 && (ft < 512 || ft > 1024 || ft % 32 != 0))
        return fail(XYZ_EINVAL, "filter_threads must be 0 or a multiple of 32 in [512, 1024]");
    if (tiles->verify_blocks_per_sm < 0 || tiles->group_runs < 0)
        return fail(XYZ_EINVAL, "verify_blocks_per_sm and group_runs must be >= 0");
    ctx->pk.filter_threads = ft;
    ctx->pk.verify_bpsm = tiles->verify_blocks_per_sm;
    // the filter path's launch group holds 64 entries' worth of runs per
    // entry budget: group_runs runs of p columns need group_runs * p / 64
    ctx->chunk_entries = tiles->group_runs == 0 ? kDefaultChunkEntries
                                                : (tiles->group_runs * ctx->pk.p + 63) / 64;
    ctx->tiles = *tiles;
    return XYZ_OK;
}

int xyz_autotune_tiles(xyz_ctx *ctx, int32_t M, double kappa, uint64_t seed, int64_t trial_runs, xyz_tiles *best,
                       double *ms_best)
{
    int rc = check_ctx(ctx);
    if (rc)
        return rc;
    if (!best || !ms_best)
        return fail(XYZ_EINVAL, "null output pointer");
    if ((rc = check_kappa(kappa)))
        return rc;
    if (M < 0 || M > 31 || trial_runs < 8)
        return fail(XYZ_EINVAL, "need 0 <= M <= 31 and trial_runs >= 8");
    const int64_t amin = amin_rule(ctx->pk.n, kappa);
    set_kappa(ctx, kappa);
    const bool timing = ctx->timing;
    ctx->timing = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    uint64_t trial = 0;
    // one warm-up search, then the timed one, with the shapes t
    auto measure = [&](const xyz_tiles &t, double *ms) -> int {
        int r = xyz_set_tiles(ctx, &t);
        int64_t nout = 0;
        if (!r)
            r = run_search(ctx, 0, trial_runs, M, amin, seed + 2 * trial, &nout);
        if (r)
            return r;
        cudaEventRecord(e0, ctx->stream);
        r = run_search(ctx, 0, trial_runs, M, amin, seed + 2 * trial + 1, &nout);
        cudaEventRecord(e1, ctx->stream);
        cudaEventSynchronize(e1);
        ++trial;
        float f = 0.0f;
        cudaEventElapsedTime(&f, e0, e1);
        *ms = f;
        return r;
    };
    xyz_tiles cur{0, 0, 0};
    double cur_ms = 0.0;
    rc = measure(cur, &cur_ms);
    // the default launch group of the filter path (make_plan's rule)
    const int64_t rdef = 64 * kDefaultChunkEntries / ctx->pk.p < 16384 ? 64 * kDefaultChunkEntries / ctx->pk.p : 16384;
    const int64_t rmin = 2 * (int64_t)filter_grid();
    const int32_t threads[4] = {640, 768, 896, 1024};
    for (int i = 0; i < 4 && !rc; ++i) {
        xyz_tiles t = cur;
        t.filter_threads = threads[i];
        double ms = 0.0;
        if ((rc = measure(t, &ms)))
            break;
        if (ms < cur_ms) {
            cur = t;
            cur_ms = ms;
        }
    }
    for (int i = 1; i <= 2 && !rc; ++i) {
        xyz_tiles t = cur;
        t.group_runs = rdef >> i;
        if (t.group_runs < rmin)
            break;
        double ms = 0.0;
        if ((rc = measure(t, &ms)))
            break;
        if (ms < cur_ms) {
            cur = t;
            cur_ms = ms;
        }
    }
    for (int b = 2; b >= 1 && !rc; --b) {
        xyz_tiles t = cur;
        t.verify_blocks_per_sm = b;
        double ms = 0.0;
        if ((rc = measure(t, &ms)))
            break;
        if (ms < cur_ms) {
            cur = t;
            cur_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->timing = timing;
    if (rc)
        return rc;
    xyz_set_tiles(ctx, &cur);
    *best = cur;
    *ms_best = cur_ms;
    return XYZ_OK;
}

int xyz_set_chunk_entries(xyz_ctx *ctx, int64_t entries)
{
    if (!ctx)
        return fail(XYZ_EINVAL, "null context");
    if (entries < 1)
        return fail(XYZ_EINVAL, "entries must be >= 1");
    ctx->chunk_entries = entries;
    return XYZ_OK;
}

namespace {

// Pack B responses (device int8, B rows of n) into ctx->ybs; -1/+1 only.
int pack_responses(xyz_ctx *ctx, const int8_t *dYs, int32_t B)
{
    const size_t row = (size_t)ctx->pk.Wp * 4;
    int rc = ensure(ctx->ybs, row * (size_t)B);
    if (rc)
        return rc;
    int64_t launches = 0;
    CU(cudaMemsetAsync(ctx->d_bad, 0, 16, ctx->stream));
    for (int32_t b = 0; b < B; ++b) {
        Packed tmp = ctx->pk;
        tmp.yb = (uint32_t *)((char *)ctx->ybs.ptr + row * b);
        CU(launch_pack_y(dYs + (int64_t)b * ctx->pk.n, tmp, ctx->d_bad, ctx->stream, &launches));
    }
    int bad = 0;
    CU(cudaMemcpyAsync(&bad, ctx->d_bad, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (bad)
        return fail(XYZ_EINVAL, "entries of the responses must be -1 or +1");
    return XYZ_OK;
}

// Copy `nout` device results (and their responses) to host pairs + offsets.
int collect_batch(xyz_ctx *ctx, int32_t B, int64_t nout, bool have_resp, int32_t only,
                  std::vector<xyz_pair> &acc, std::vector<int64_t> &counts)
{
    if (nout == 0)
        return XYZ_OK;
    const size_t at = acc.size();
    acc.resize(at + (size_t)nout);
    std::vector<uint32_t> resp;
    if (have_resp)
        resp.resize((size_t)nout);
    int rc = copy_pairs(ctx, nout, acc.data() + at, have_resp ? resp.data() : nullptr);
    if (rc)
        return rc;
    for (int64_t i = 0; i < nout; ++i) {
        const uint32_t b = have_resp ? resp[(size_t)i] : (uint32_t)only;
        if (b >= (uint32_t)B)
            return fail(XYZ_ECUDA, "response index out of range in batched results");
        counts[b] += 1;
    }
    return XYZ_OK;
}

int search_batch_dev(xyz_ctx *ctx, const int8_t *dYs, int32_t B, int32_t L, int32_t M, double kappa,
                     uint64_t seed, xyz_pair **pairs, int64_t *offsets)
{
    int rc = check_ctx(ctx);
    if (rc)
        return rc;
    if (!dYs || !pairs || !offsets)
        return fail(XYZ_EINVAL, "null pointer argument");
    if (B < 1 || L < 1)
        return fail(XYZ_EINVAL, "need B >= 1 and L >= 1");
    if ((rc = check_M(M)) || (rc = check_kappa(kappa)))
        return rc;
    if (ctx->pk.cdf)
        return fail(XYZ_EINVAL, "batched search takes binary responses");
    if ((rc = pack_responses(ctx, dYs, B)))
        return rc;
    const int64_t amin = amin_rule(ctx->pk.n, kappa);
    std::vector<xyz_pair> acc;
    std::vector<int64_t> counts((size_t)B, 0);
    const size_t row = (size_t)ctx->pk.Wp * 4;
    if (amin <= ctx->pk.n) {
        Plan pl = make_plan(ctx, L, M, B);
        if (B > 1 && pl.filter) {
            int64_t nout = 0;
            if ((rc = run_search_multi(ctx, (const uint32_t *)ctx->ybs.ptr, B, 0, L, M, amin, seed,
                                       &nout)) ||
                (rc = collect_batch(ctx, B, nout, true, 0, acc, counts)))
                return rc;
        } else {
            // one response at a time on the resident X (results are identical)
            uint32_t *own = ctx->pk.yb;
            for (int32_t b = 0; b < B && !rc; ++b) {
                ctx->pk.yb = (uint32_t *)((char *)ctx->ybs.ptr + row * b);
                int64_t nout = 0;
                rc = run_search(ctx, 0, L, M, amin, seed, &nout);
                if (!rc)
                    rc = collect_batch(ctx, B, nout, false, b, acc, counts);
            }
            ctx->pk.yb = own;
            if (rc)
                return rc;
        }
    }
    xyz_pair *host = nullptr;
    if (!acc.empty()) {
        host = (xyz_pair *)std::malloc(acc.size() * sizeof(xyz_pair));
        if (!host)
            return fail(XYZ_ENOMEM, "host allocation of results failed");
        std::memcpy(host, acc.data(), acc.size() * sizeof(xyz_pair));
    }
    offsets[0] = 0;
    for (int32_t b = 0; b < B; ++b)
        offsets[b + 1] = offsets[b] + counts[(size_t)b];
    *pairs = host;
    return XYZ_OK;
}

}  // namespace

int xyz_search_batch_dev(xyz_ctx *ctx, const int8_t *dYs, int32_t B, int32_t L, int32_t M, double kappa,
                         uint64_t seed, xyz_pair **pairs, int64_t *offsets)
{
    return search_batch_dev(ctx, dYs, B, L, M, kappa, seed, pairs, offsets);
}

int xyz_search_batch(xyz_ctx *ctx, const int8_t *Ys, int32_t B, int32_t L, int32_t M, double kappa,
                     uint64_t seed, xyz_pair **pairs, int64_t *offsets)
{
    int rc = check_ctx(ctx);
    if (rc)
        return rc;
    if (!Ys || B < 1)
        return fail(XYZ_EINVAL, "need Ys and B >= 1");
    int8_t *dYs = nullptr;
    const size_t bytes = (size_t)B * (size_t)ctx->pk.n;
    if (cudaMalloc(&dYs, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(XYZ_ENOMEM, "cudaMalloc of response staging failed");
    }
    cudaError_t e = cudaMemcpy(dYs, Ys, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dYs);
        return fail(XYZ_ECUDA, std::string("cudaMemcpy of responses: ") + cudaGetErrorString(e));
    }
    rc = search_batch_dev(ctx, dYs, B, L, M, kappa, seed, pairs, offsets);
    cudaFree(dYs);
    return rc;
}

int xyz_set_filter(xyz_ctx *ctx, int enable)
{
    if (!ctx)
        return fail(XYZ_EINVAL, "null context");
    if (enable < 0 || enable > 2)
        return fail(XYZ_EINVAL, "enable must be 0, 1 or 2");
    ctx->use_filter = enable != 0;
    ctx->force_big = enable == 2;
    return XYZ_OK;
}

int xyz_set_spill_flush(xyz_ctx *ctx, int64_t groups)
{
    if (!ctx || groups < 0)
        return fail(XYZ_EINVAL, "need a context and groups >= 0");
    ctx->spill_flush = groups;
    return XYZ_OK;
}

int xyz_set_onchip_partitions(xyz_ctx *ctx, int32_t max_parts)
{
    if (!ctx || max_parts < 0 || max_parts > 32)
        return fail(XYZ_EINVAL, "need a context and max_parts in [0, 32]");
    ctx->onchip_parts = max_parts;
    return XYZ_OK;
}

int xyz_set_fused_filter(xyz_ctx *ctx, int enable)
{
    if (!ctx || (enable != 0 && enable != 1))
        return fail(XYZ_EINVAL, "need a context and enable in {0, 1}");
    ctx->fuse_filters = enable;
    return XYZ_OK;
}

int xyz_run_keys(xyz_ctx *ctx, int32_t M, uint64_t seed, int64_t run, uint64_t *kx, uint64_t *c)
{
    int rc = check_ctx(ctx);
    if (rc)
        return rc;
    if (!kx || !c)
        return fail(XYZ_EINVAL, "null output pointer");
    if (run < 0)
        return fail(XYZ_EINVAL, "run must be >= 0");
    if ((rc = check_M(M)))
        return rc;
    const int64_t p = ctx->pk.p;
    Plan pl;
    pl.R = 1;
    pl.NB = pl.BB = 1;
    pl.filter = false;
    pl.part = false;
    pl.k64 = true;
    pl.kbits = 1;
    if ((rc = ensure_search_ws(ctx, pl, 1, 1)) || (rc = ensure(ctx->raw, (size_t)(p + 1) * 8)))
        return rc;
    int64_t launches = 0;
    uint64_t *raw = (uint64_t *)ctx->raw.ptr;
    CU(launch_keybuild64(ctx->pk, M, seed, run, 1, 0, (uint64_t *)ctx->keysA.ptr,
                         (uint32_t *)ctx->valsA.ptr, (uint8_t *)ctx->cnz.ptr, raw, raw + p,
                         ctx->stream, &launches));
    CU(cudaMemcpyAsync(kx, raw, (size_t)p * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(c, raw + p, 8, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return XYZ_OK;
}

int xyz_run_candidates(xyz_ctx *ctx, int32_t M, uint64_t seed, int64_t run, int32_t **jk,
                       int64_t *count)
{
    int rc = check_ctx(ctx);
    if (rc)
        return rc;
    if (!jk || !count)
        return fail(XYZ_EINVAL, "null output pointer");
    if (run < 0)
        return fail(XYZ_EINVAL, "run must be >= 0");
    if ((rc = check_M(M)))
        return rc;
    int64_t nout = 0;
    ctx->pk.wkq = -INFINITY;                           // every candidate passes
    ctx->pk.rkq = -INFINITY;
    if ((rc = run_search(ctx, run, run + 1, M, 0, seed, &nout)))
        return rc;
    int32_t *host = nullptr;
    if (nout > 0) {
        std::vector<PairOut> tmp((size_t)nout);
        if ((rc = copy_pairs(ctx, nout, tmp.data())))
            return rc;
        host = (int32_t *)std::malloc((size_t)nout * 2 * sizeof(int32_t));
        if (!host)
            return fail(XYZ_ENOMEM, "host allocation failed");
        for (int64_t i = 0; i < nout; ++i) {
            host[2 * i] = tmp[i].j;
            host[2 * i + 1] = tmp[i].k;
        }
    }
    *jk = host;
    *count = nout;
    return XYZ_OK;
}

int xyz_agree(xyz_ctx *ctx, const int32_t *j, const int32_t *k, int64_t count, int32_t *agree)
{
    int rc = check_ctx(ctx);
    if (rc)
        return rc;
    if (count < 0 || (count > 0 && (!j || !k || !agree)))
        return fail(XYZ_EINVAL, "bad pair arrays");
    for (int64_t t = 0; t < count; ++t)
        if (j[t] < 0 || j[t] >= ctx->pk.p || k[t] < 0 || k[t] >= ctx->pk.p)
            return fail(XYZ_EINVAL, "pair index out of range");
    if (count == 0)
        return XYZ_OK;
    if ((rc = ensure(ctx->raw, (size_t)count * 12)))
        return rc;
    int32_t *dj = (int32_t *)ctx->raw.ptr, *dk = dj + count, *da = dk + count;
    int64_t launches = 0;
    CU(cudaMemcpyAsync(dj, j, (size_t)count * 4, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(dk, k, (size_t)count * 4, cudaMemcpyHostToDevice, ctx->stream));
    CU(launch_agree_pairs(ctx->pk, dj, dk, count, da, ctx->stream, &launches));
    CU(cudaMemcpyAsync(agree, da, (size_t)count * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return XYZ_OK;
}

int xyz_sample_agree(xyz_ctx *ctx, int64_t count, uint64_t seed, int32_t *j_out, int32_t *k_out,
                     int32_t *agree)
{
    int rc = check_ctx(ctx);
    if (rc)
        return rc;
    if (count < 0 || (count > 0 && (!j_out || !k_out || !agree)))
        return fail(XYZ_EINVAL, "bad output arrays");
    if (count == 0)
        return XYZ_OK;
    if ((rc = ensure(ctx->raw, (size_t)count * 12)))
        return rc;
    int32_t *dj = (int32_t *)ctx->raw.ptr, *dk = dj + count, *da = dk + count;
    int64_t launches = 0;
    CU(launch_sample_pairs(ctx->pk, count, seed, dj, dk, da, ctx->stream, &launches));
    CU(cudaMemcpyAsync(j_out, dj, (size_t)count * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(k_out, dk, (size_t)count * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(agree, da, (size_t)count * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return XYZ_OK;
}

int64_t xyz_amin(int64_t n, double kappa) { return amin_rule(n, kappa); }

}  // extern "C"

// Read-only views of a context for other translation units of the library.
namespace xyz {
const Packed *ctx_packed(const xyz_ctx *c) { return &c->pk; }
cudaStream_t ctx_stream(const xyz_ctx *c) { return c->stream; }
int ctx_device(const xyz_ctx *c) { return c->device; }

// A context with its own stream and workspace that searches the packed X of
// other contexts (view_target); it never frees packed arrays.
int view_create(int device, xyz_ctx **out)
{
    xyz_ctx *c = new (std::nothrow) xyz_ctx();
    if (!c)
        return fail(XYZ_ENOMEM, "host allocation failed");
    std::memset(&c->stats, 0, sizeof(c->stats));
    c->device = device;
    c->owns_packed = false;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaMalloc(&c->d_bad, 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        destroy_ctx(c);
        return fail(XYZ_ECUDA, std::string("view set-up: ") + cudaGetErrorString(e));
    }
    c->own_stream = true;
    *out = c;
    return XYZ_OK;
}

void view_target(xyz_ctx *view, const xyz_ctx *base, uint32_t *yb)
{
    view->pk = base->pk;
    if (yb)
        view->pk.yb = yb;
}

int64_t ctx_device_bytes(const xyz_ctx *c) { return (c->owns_packed ? c->packed_bytes : 0) + ws_bytes(c); }

// Sizing snapshots of a context (its buffer sizes and capacities); a copy
// shares the original's buffers and frees none of them.
xyz_ctx *ctx_sizing_copy(const xyz_ctx *c) { return new (std::nothrow) xyz_ctx(*c); }
void ctx_sizing_update(xyz_ctx *dst, const xyz_ctx *src) { *dst = *src; }
void ctx_sizing_free(xyz_ctx *c) { delete c; }

// Bytes by which the workspace of `view` (a sizing snapshot) grows to run
// `runs` runs at M of a search on base's packed X: the same sizing as a
// search, on a copy, with nothing allocated.  Searches grow some buffers on
// overflow as they go (members, records, segments); this counts their sizes
// at the start of a search.
int64_t ctx_slice_growth(const xyz_ctx *view, const xyz_ctx *base, int64_t runs, int M)
{
    xyz_ctx tmp = *view;
    view_target(&tmp, base, nullptr);
    int64_t grow = 0;
    t_size_only = &grow;
    const Plan pl = make_plan(&tmp, runs, M, 1);
    ensure_search_ws(&tmp, pl, 1, runs);
    ensure_records(&tmp, 1);
    t_size_only = nullptr;
    return grow;
}

// Pack a host response into yb_dev (Wp words) on c's stream; -1/+1 only.
// Uses c's staging buffer: calls on one context must not overlap.
int pack_response(xyz_ctx *c, const int8_t *Y, uint32_t *yb_dev)
{
    int rc = ensure(c->y_stage, (size_t)c->pk.n);
    if (rc)
        return rc;
    int64_t launches = 0;
    Packed tmp = c->pk;
    tmp.yb = yb_dev;
    int bad = 0;
    CU(cudaMemcpyAsync(c->y_stage.ptr, Y, (size_t)c->pk.n, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemsetAsync(c->d_bad, 0, 16, c->stream));
    CU(launch_pack_y((const int8_t *)c->y_stage.ptr, tmp, c->d_bad, c->stream, &launches));
    CU(cudaMemcpyAsync(&bad, c->d_bad, 4, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (bad)
        return fail(XYZ_EINVAL, "entries of Y must be -1 or +1");
    return XYZ_OK;
}
}  // namespace xyz
