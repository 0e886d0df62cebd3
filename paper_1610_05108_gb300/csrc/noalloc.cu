// xyz_run_candidates_noalloc: the candidate set of one run, computed with no
// device (or host) memory allocation at call time.
//
// Who needs this: callers that cannot call cudaMalloc when they want a
// result -- for example a process whose device memory has been handed in
// full to another allocator (a framework's caching pool that reserved the
// HBM), or a latency-critical loop that must not pay for cudaMalloc/cudaFree,
// which can synchronise the whole device.  Such callers create their context
// once, up front, and afterwards get E_l of any run through this entry point.
//
// All scratch of the search (composite keys, sort buffers, histograms, bucket
// list, pair offsets, records, deduplication buffers) lives in one
// file-scope __device__ array of fixed size, NOALLOC_SCRATCH_BYTES, which
// every GPU that loads the library holds until the process exits.  Host code
// cannot use the array's name as a device address (on the host it is only a
// stand-in symbol), so the first call on each device, with that device
// current, asks the runtime for the address with cudaGetSymbolAddress and
// caches it.  That first call should therefore happen before any stream
// capture is begun on that device.
//
// Every call shares the array and finds it as the previous call left it;
// the counters that must start at zero are cleared at the start of each
// call, and everything else is fully written before it is read.  Calls that
// overlap on the GPU (from different threads or streams) race on the array
// and must be serialised by the caller.
//
// The cached address belongs to the device's primary context: after a
// cudaDeviceReset on that device the cache is stale, and this entry point
// must not be called there again in the same process (every context of the
// library created before the reset is invalid by then anyway).
//
// The pass threshold of the verification is taken from a private copy of
// the context's packed description with every threshold at -infinity, so a
// weighted context returns its whole candidate set whatever search ran on it
// before, and the context itself is not written.  Contexts built by the
// unbiased transform of real X (whose keys come from a random binarisation
// inside the survivor filter) are refused.
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/xyz.h"
#include "xyz_internal.cuh"

namespace xyz {
namespace {

constexpr int64_t NA_P = XYZ_NOALLOC_MAX_P;        // columns
constexpr int64_t NA_REC = XYZ_NOALLOC_MAX_PAIRS;  // candidates of one run
constexpr int64_t NA_BCAP = NA_P / 2 + 1;          // buckets hold >= 2 entries

constexpr int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }

// byte offsets of the scratch regions
constexpr int64_t OFF_KEYS_A = 0;
constexpr int64_t OFF_KEYS_B = OFF_KEYS_A + align256(NA_P * 8);
constexpr int64_t OFF_VALS_A = OFF_KEYS_B + align256(NA_P * 8);
constexpr int64_t OFF_VALS_B = OFF_VALS_A + align256(NA_P * 4);
constexpr int64_t OFF_RADIX = OFF_VALS_B + align256(NA_P * 4);
constexpr int64_t RADIX_BYTES = 16 * 1024;
constexpr int64_t OFF_CNZ = OFF_RADIX + RADIX_BYTES;
constexpr int64_t OFF_BUCKETS = OFF_CNZ + 256;
constexpr int64_t OFF_PCOUNT = OFF_BUCKETS + align256(NA_BCAP * (int64_t)sizeof(Bucket));
constexpr int64_t OFF_POFF = OFF_PCOUNT + align256(NA_BCAP * 8);
constexpr int64_t OFF_SCAN = OFF_POFF + align256(NA_BCAP * 8);
constexpr int64_t SCAN_BYTES = 4 * 1024;
constexpr int64_t OFF_CTR = OFF_SCAN + SCAN_BYTES;
constexpr int64_t OFF_RKEYS = OFF_CTR + 256;
constexpr int64_t OFF_RKEYS_ALT = OFF_RKEYS + align256(NA_REC * 8);
constexpr int64_t OFF_RAGREE = OFF_RKEYS_ALT + align256(NA_REC * 8);
constexpr int64_t OFF_RAGREE_ALT = OFF_RAGREE + align256(NA_REC * 4);
constexpr int64_t OFF_FLAGS = OFF_RAGREE_ALT + align256(NA_REC * 4);
constexpr int64_t OFF_POS = OFF_FLAGS + align256(NA_REC * 4);
constexpr int64_t OFF_OUT = OFF_POS + align256(NA_REC * 4);
constexpr int64_t OFF_DEDUP = OFF_OUT + align256(NA_REC * (int64_t)sizeof(PairOut));
constexpr int64_t DEDUP_BYTES = 64 * 1024;
constexpr int64_t NOALLOC_SCRATCH_BYTES = OFF_DEDUP + DEDUP_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_scratch_dev[MAX_DEVICES] = {};

// Device address of the scratch array on `device` (which must be current).
int scratch_for(int device, unsigned char **out)
{
    if (device < 0 || device >= MAX_DEVICES)
        return fail(XYZ_EINVAL, "device index out of range for the scratch table");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(XYZ_ECUDA, std::string("cudaGetSymbolAddress of the scratch array: ") +
                                       cudaGetErrorString(e));
        g_scratch_dev[device] = (unsigned char *)ptr;
    }
    *out = g_scratch_dev[device];
    return XYZ_OK;
}

int ceil_log2_na(int64_t x)
{
    int b = 0;
    while (((int64_t)1 << b) < x)
        ++b;
    return b;
}

// Restores the caller's current device when the entry point returns.
struct DeviceRestore {
    int prev = -1;
    DeviceRestore() { cudaGetDevice(&prev); }
    ~DeviceRestore()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

#define NA_CU(expr)                                                                      \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess)                                                           \
            return fail(XYZ_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));  \
    } while (0)

}  // namespace
}  // namespace xyz

using namespace xyz;

extern "C" int xyz_run_candidates_noalloc(xyz_ctx *ctx, int32_t M, uint64_t seed, int64_t run,
                                          int32_t *jk, int64_t cap, int64_t *count)
{
    if (!ctx)
        return fail(XYZ_EINVAL, "null context");
    if (!jk || !count || cap < 0)
        return fail(XYZ_EINVAL, "null output pointer or negative capacity");
    if (M < 0 || M > XYZ_MAX_M)
        return fail(XYZ_EINVAL, "M must be in [0, 64]");
    if (run < 0)
        return fail(XYZ_EINVAL, "run must be >= 0");
    // every candidate passes: thresholds at -infinity in a private copy
    Packed pk = *ctx_packed(ctx);
    pk.wkq = -INFINITY;
    pk.rkq = -INFINITY;
    if (pk.Xrs)
        return fail(XYZ_EINVAL, "the allocation-free entry point does not take contexts of real X "
                                "(xyz_create_unbiased); use xyz_run_candidates");
    if (pk.p > NA_P)
        return fail(XYZ_EINVAL, "p = " + std::to_string(pk.p) +
                                    " exceeds the allocation-free limit XYZ_NOALLOC_MAX_P = " +
                                    std::to_string(NA_P));
    const int64_t p = pk.p;
    if ((int64_t)radix_temp_bytes(p) > RADIX_BYTES || (int64_t)scan_temp_bytes(NA_BCAP) > SCAN_BYTES ||
        (int64_t)(radix_temp_bytes(NA_REC) + scan_temp_bytes(NA_REC)) > DEDUP_BYTES)
        return fail(XYZ_EINVAL, "scratch layout too small for this library");
    const int dev = ctx_device(ctx);
    DeviceRestore restore;
    NA_CU(cudaSetDevice(dev));
    unsigned char *base = nullptr;
    int rc = scratch_for(dev, &base);
    if (rc)
        return rc;
    cudaStream_t s = ctx_stream(ctx);

    uint64_t *keysA = (uint64_t *)(base + OFF_KEYS_A), *keysB = (uint64_t *)(base + OFF_KEYS_B);
    uint32_t *valsA = (uint32_t *)(base + OFF_VALS_A), *valsB = (uint32_t *)(base + OFF_VALS_B);
    uint8_t *cnz = (uint8_t *)(base + OFF_CNZ);
    Bucket *buckets = (Bucket *)(base + OFF_BUCKETS);
    uint64_t *pcount = (uint64_t *)(base + OFF_PCOUNT), *poff = (uint64_t *)(base + OFF_POFF);
    uint32_t *ctr = (uint32_t *)(base + OFF_CTR);           // [0] buckets [1] records [2] unique [3] error
    uint64_t *total = (uint64_t *)(base + OFF_CTR + 16);
    uint64_t *cand = (uint64_t *)(base + OFF_CTR + 24);
    uint64_t *rkeys = (uint64_t *)(base + OFF_RKEYS), *rkeys_alt = (uint64_t *)(base + OFF_RKEYS_ALT);
    uint32_t *ragree = (uint32_t *)(base + OFF_RAGREE), *ragree_alt = (uint32_t *)(base + OFF_RAGREE_ALT);
    uint32_t *flags = (uint32_t *)(base + OFF_FLAGS), *pos = (uint32_t *)(base + OFF_POS);
    PairOut *out = (PairOut *)(base + OFF_OUT);
    unsigned char *dedup = base + OFF_DEDUP;

    int64_t launches = 0;
    const int kbits = ceil_log2_na(p) < 1 ? 1 : ceil_log2_na(p);
    const int64_t bcap = p / 2 + 1;
    // counters start at zero on every call
    NA_CU(cudaMemsetAsync(base + OFF_CTR, 0, 256, s));
    NA_CU(launch_keybuild64(pk, M, seed, run, 1, 0, keysA, valsA, cnz, nullptr, nullptr, s, &launches));
    bool alt = false;
    NA_CU(radix_sort64(keysA, valsA, keysB, valsB, p, M, base + OFF_RADIX, &alt, s, &launches));
    const uint64_t *ks = alt ? keysB : keysA;
    const uint32_t *vs = alt ? valsB : valsA;
    NA_CU(launch_join64(ks, p, M, 0, cnz, buckets, pcount, ctr, s, &launches));
    NA_CU(scan_u64_dev(pcount, poff, ctr, bcap, total, cand, base + OFF_SCAN, s, &launches));
    int *verr = (int *)(ctr + 3);
    NA_CU(launch_verify(pk, buckets, poff, ctr, total, vs, 0, kbits, rkeys, ragree, ctr + 1,
                        (uint32_t)NA_REC, s, &launches, nullptr, nullptr, nullptr, 0, verr));
    uint32_t nrec = 0;
    int err = 0;
    NA_CU(cudaMemcpyAsync(&nrec, ctr + 1, 4, cudaMemcpyDeviceToHost, s));
    NA_CU(cudaMemcpyAsync(&err, verr, 4, cudaMemcpyDeviceToHost, s));
    NA_CU(cudaStreamSynchronize(s));
    if (err)
        return fail(XYZ_ECUDA, "internal error: a candidate's offset lies outside its bucket");
    if ((int64_t)nrec > NA_REC)
        return fail(XYZ_ENOMEM, "run has " + std::to_string(nrec) +
                                    " candidates, above the allocation-free limit XYZ_NOALLOC_MAX_PAIRS = " +
                                    std::to_string(NA_REC));
    if ((int64_t)nrec > cap)
        return fail(XYZ_ENOMEM, "output capacity " + std::to_string(cap) + " < " +
                                    std::to_string(nrec) + " candidates");
    bool alt2 = false;
    const size_t rt = radix_temp_bytes(NA_REC);
    NA_CU(radix_sort64(rkeys, ragree, rkeys_alt, ragree_alt, (int64_t)nrec, 2 * kbits, dedup, &alt2, s,
                       &launches));
    NA_CU(launch_unique(alt2 ? rkeys_alt : rkeys, alt2 ? ragree_alt : ragree, ctr + 1, NA_REC, kbits,
                        pk.n, flags, pos, dedup + rt, out, ctr + 2, s, &launches));
    uint32_t nout = 0;
    NA_CU(cudaMemcpyAsync(&nout, ctr + 2, 4, cudaMemcpyDeviceToHost, s));
    NA_CU(cudaStreamSynchronize(s));
    if (nrec == 0)
        nout = 0;
    if (nout > 0) {
        // (j, k) are the first 8 bytes of each 16-byte record
        NA_CU(cudaMemcpy2DAsync(jk, 2 * sizeof(int32_t), out, sizeof(PairOut), 2 * sizeof(int32_t),
                                nout, cudaMemcpyDeviceToHost, s));
        NA_CU(cudaStreamSynchronize(s));
    }
    *count = nout;
    return XYZ_OK;
}
