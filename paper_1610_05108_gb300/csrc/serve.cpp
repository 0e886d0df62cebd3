// Search server: a request loop in front of the xyz search.
//
// Datasets (packed X and a default response) stay resident on the device.
// A request names a dataset, optionally its own response Y, and (L, M,
// kappa, seed).  Requests are admitted while the device memory in use --
// resident datasets, the workers' workspaces, and the admitted requests'
// reservations -- stays within the budget; the rest wait in arrival order.
// Admitted requests are served by continuous batching at run-range
// granularity: each is cut into slices of `slice_runs` runs, and the worker
// threads take slices round-robin over all admitted requests, so a request
// that arrives while others are running starts at the next slice boundary
// and its kernels overlap with theirs on the device (every worker owns a
// CUDA stream and one workspace that it points at whichever dataset its
// current slice belongs to).  The runs of a search are independent and
// counter-seeded (Algorithm 2's loop), so the union of a request's slice
// results is exactly the result of the whole search, whatever else was
// running: results depend only on (X, Y, L, M, kappa, seed).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/xyz.h"
#include "xyz_internal.cuh"

using namespace xyz;

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

enum ReqState { RQ_QUEUED, RQ_ACTIVE, RQ_DONE, RQ_CANCELED, RQ_FAILED };

struct Request {
    int64_t id = 0;
    int dataset = 0;
    uint32_t *yb = nullptr;       // own packed response (device), or null
    int32_t L = 1, M = 0;
    double kappa = 0;
    uint64_t seed = 0;
    int64_t next_run = 0;         // first run not yet handed out
    int slices_out = 0, slices_done = 0;
    int64_t reserve = 0;          // bytes counted against the budget while admitted
    std::vector<std::vector<xyz_pair>> parts;   // slice results, each sorted by (j, k), each pair once
    std::vector<xyz_pair> acc;    // their union (finish)
    ReqState state = RQ_QUEUED;
    int err_code = 0;
    std::string err;
    bool cancel = false;
    Clock::time_point t_submit, t_admit, t_done;
};

struct Dataset {
    xyz_ctx *base = nullptr;
    int64_t bytes = 0;
};

}  // namespace

struct xyz_server {
    int device = 0;
    int64_t budget = 0;
    int64_t slice_runs = 2048;
    std::mutex mu;
    std::mutex pack_mu;               // serialises packing of submitted responses
    std::condition_variable cv_work, cv_done;
    std::vector<Dataset> datasets;
    std::map<int64_t, Request> reqs;
    std::deque<int64_t> queued;       // waiting for admission, arrival order
    std::vector<int64_t> active;      // admitted, runs left to hand out
    size_t rr = 0;                    // round-robin position in `active`
    int64_t next_id = 1;
    int64_t reserved = 0;
    std::vector<int64_t> worker_bytes;
    std::vector<std::thread> threads;
    std::vector<xyz_ctx *> views;
    std::vector<xyz_ctx *> shadows;   // sizing snapshot of each worker's view, updated under the lock
    // device buffers for requests' packed responses, reused across requests
    std::vector<std::pair<size_t, uint32_t *>> yb_free;
    bool stop = false;
    // statistics
    std::vector<double> latencies;
    int64_t completed = 0, canceled = 0, failed = 0;
    double pairs_screened = 0;
    Clock::time_point t0;
    bool started = false;
    Clock::time_point first_submit, last_done;
};

namespace {

int64_t datasets_bytes(const xyz_server *s)
{
    int64_t b = 0;
    for (const Dataset &d : s->datasets)
        b += d.bytes;
    return b;
}

int64_t in_use(const xyz_server *s)
{
    int64_t b = datasets_bytes(s) + s->reserved;
    for (int64_t w : s->worker_bytes)
        b += w;
    for (const auto &f : s->yb_free)
        b += (int64_t)f.first;
    return b;
}

// Return a request's response buffer to the server's free list (lock held).
void release_yb(xyz_server *s, Request &r)
{
    if (r.yb) {
        const Packed &pk = *ctx_packed(s->datasets[r.dataset].base);
        s->yb_free.emplace_back((size_t)pk.Wp * 4, r.yb);
        r.yb = nullptr;
    }
}

// A free response buffer of at least `bytes`, or a new one (lock held).
uint32_t *take_yb(xyz_server *s, size_t bytes)
{
    size_t best = s->yb_free.size();
    for (size_t i = 0; i < s->yb_free.size(); ++i)
        if (s->yb_free[i].first >= bytes && (best == s->yb_free.size() || s->yb_free[i].first < s->yb_free[best].first))
            best = i;
    if (best < s->yb_free.size()) {
        uint32_t *p = s->yb_free[best].second;
        s->yb_free.erase(s->yb_free.begin() + (ptrdiff_t)best);
        return p;
    }
    uint32_t *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

// Device bytes to reserve for a request while it is admitted: its own
// response bits, and the growth its slices may cause in the workers'
// workspaces -- for every worker, since any may take a slice -- sized by the
// library's own workspace rules from each worker's current sizes (lock
// held).  Growth that has happened shows in the workers' measured bytes
// from then on, so until the request finishes it is counted twice: the
// estimate errs towards waiting.
int64_t reservation(xyz_server *s, const Request &r)
{
    const xyz_ctx *base = s->datasets[r.dataset].base;
    int64_t b = r.yb ? (int64_t)ctx_packed(base)->Wp * 4 : 0;
    const int64_t runs = std::min<int64_t>(r.L, s->slice_runs);
    for (const xyz_ctx *sh : s->shadows)
        b += ctx_slice_growth(sh, base, runs, r.M);
    return b;
}

// Move queued requests to active while the budget allows (lock held).
// The oldest waiting request is always admitted when nothing is active,
// so a request larger than the budget cannot wait forever.
void admit(xyz_server *s)
{
    while (!s->queued.empty()) {
        Request &r = s->reqs[s->queued.front()];
        if (r.cancel) {
            r.state = RQ_CANCELED;
            r.t_done = Clock::now();
            s->canceled++;
            release_yb(s, r);
            s->queued.pop_front();
            s->cv_done.notify_all();
            continue;
        }
        r.reserve = reservation(s, r);
        if (!s->active.empty() && in_use(s) + r.reserve > s->budget)
            break;
        r.state = RQ_ACTIVE;
        r.t_admit = Clock::now();
        s->reserved += r.reserve;
        s->active.push_back(r.id);
        s->queued.pop_front();
    }
}

// Union of sorted, duplicate-free slice results into one sorted list with
// each pair once: a merge over the slices' heads (the union within a slice
// ran on the device, in the search).
std::vector<xyz_pair> merge_parts(std::vector<std::vector<xyz_pair>> &parts)
{
    auto later = [](const std::pair<xyz_pair, size_t> &a, const std::pair<xyz_pair, size_t> &b) {
        return a.first.j != b.first.j ? a.first.j > b.first.j : a.first.k > b.first.k;
    };
    std::vector<std::pair<xyz_pair, size_t>> heap;
    std::vector<size_t> at(parts.size(), 0);
    size_t total = 0;
    for (size_t i = 0; i < parts.size(); ++i) {
        total += parts[i].size();
        if (!parts[i].empty())
            heap.emplace_back(parts[i][0], i);
    }
    std::make_heap(heap.begin(), heap.end(), later);
    std::vector<xyz_pair> out;
    out.reserve(total);
    while (!heap.empty()) {
        std::pop_heap(heap.begin(), heap.end(), later);
        const xyz_pair e = heap.back().first;
        const size_t i = heap.back().second;
        heap.pop_back();
        if (out.empty() || out.back().j != e.j || out.back().k != e.k)
            out.push_back(e);
        if (++at[i] < parts[i].size()) {
            heap.emplace_back(parts[i][at[i]], i);
            std::push_heap(heap.begin(), heap.end(), later);
        }
    }
    parts.clear();
    return out;
}

void finish(xyz_server *s, Request &r)
{
    r.acc = merge_parts(r.parts);
    r.t_done = Clock::now();
    s->reserved -= r.reserve;
    if (r.cancel) {
        r.state = RQ_CANCELED;
        s->canceled++;
        r.acc.clear();
    } else if (r.err_code) {
        r.state = RQ_FAILED;
        s->failed++;
    } else {
        r.state = RQ_DONE;
        s->completed++;
        s->latencies.push_back(ms_since(r.t_submit, r.t_done));
        const double p = (double)ctx_packed(s->datasets[r.dataset].base)->p;
        s->pairs_screened += p * (p - 1) / 2;
        s->last_done = r.t_done;
    }
    release_yb(s, r);
    admit(s);
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

void worker_main(xyz_server *s, int w)
{
    cudaSetDevice(s->device);
    xyz_ctx *view = s->views[w];
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        // next slice, round-robin over the admitted requests
        int64_t rid = -1;
        while (!s->stop) {
            for (size_t k = 0; k < s->active.size(); ++k) {
                const size_t i = (s->rr + k) % s->active.size();
                Request &r = s->reqs[s->active[i]];
                if (!r.cancel && r.next_run < r.L && !r.err_code) {
                    rid = r.id;
                    s->rr = i + 1;
                    break;
                }
            }
            if (rid >= 0)
                break;
            s->cv_work.wait(lk);
        }
        if (s->stop)
            return;
        Request &r = s->reqs[rid];
        const int64_t l0 = r.next_run;
        const int64_t l1 = std::min<int64_t>(r.L, l0 + s->slice_runs);
        r.next_run = l1;
        r.slices_out++;
        if (r.next_run >= r.L)
            s->active.erase(std::find(s->active.begin(), s->active.end(), rid));
        xyz_ctx *base = s->datasets[r.dataset].base;
        uint32_t *yb = r.yb;
        const int32_t M = r.M;
        const double kappa = r.kappa;
        const uint64_t seed = r.seed;
        lk.unlock();

        view_target(view, base, yb);
        xyz_pair *pairs = nullptr;
        int64_t np = 0;
        const int rc = xyz_search_range(view, l0, l1, M, kappa, seed, &pairs, &np);
        std::string msg = rc ? xyz_last_error() : "";
        const int64_t wb = ctx_device_bytes(view);

        lk.lock();
        s->worker_bytes[w] = wb;
        ctx_sizing_update(s->shadows[w], view);
        Request &q = s->reqs[rid];
        if (rc) {
            q.err_code = rc;
            q.err = msg;
        } else if (np > 0) {
            q.parts.emplace_back(pairs, pairs + np);
        }
        xyz_free_pairs(pairs);
        q.slices_done++;
        if ((q.next_run >= q.L || q.cancel || q.err_code) && q.slices_done == q.slices_out) {
            auto it = std::find(s->active.begin(), s->active.end(), rid);
            if (it != s->active.end())
                s->active.erase(it);
            finish(s, q);
        }
    }
}

int take_result(xyz_server *s, Request &r, xyz_pair **pairs, int64_t *npairs, double *latency_ms)
{
    if (r.state == RQ_CANCELED)
        return fail(XYZ_ECANCELED, "request was cancelled");
    if (r.state == RQ_FAILED)
        return fail(r.err_code, r.err);
    xyz_pair *host = nullptr;
    if (!r.acc.empty()) {
        host = (xyz_pair *)std::malloc(r.acc.size() * sizeof(xyz_pair));
        if (!host)
            return fail(XYZ_ENOMEM, "host allocation of results failed");
        std::memcpy(host, r.acc.data(), r.acc.size() * sizeof(xyz_pair));
    }
    if (pairs)
        *pairs = host;
    else
        std::free(host);
    if (npairs)
        *npairs = (int64_t)r.acc.size();
    if (latency_ms)
        *latency_ms = ms_since(r.t_submit, r.t_done);
    s->reqs.erase(r.id);
    return XYZ_OK;
}

}  // namespace

extern "C" {

int xyz_server_create(int32_t workers, int64_t hbm_budget_bytes, int64_t slice_runs, xyz_server **out)
{
    if (!out || workers < 1 || workers > 64 || hbm_budget_bytes < 1 || slice_runs < 1)
        return fail(XYZ_EINVAL, "need 1 <= workers <= 64, a positive budget and slice size");
    xyz_server *s = new (std::nothrow) xyz_server();
    if (!s)
        return fail(XYZ_ENOMEM, "host allocation failed");
    cudaGetDevice(&s->device);
    s->budget = hbm_budget_bytes;
    s->slice_runs = slice_runs;
    s->worker_bytes.assign((size_t)workers, 0);
    for (int w = 0; w < workers; ++w) {
        xyz_ctx *v = nullptr;
        int rc = view_create(s->device, &v);
        if (rc) {
            for (xyz_ctx *x : s->views)
                xyz_destroy(x);
            for (xyz_ctx *x : s->shadows)
                ctx_sizing_free(x);
            delete s;
            return rc;
        }
        s->views.push_back(v);
        s->shadows.push_back(ctx_sizing_copy(v));
        if (!s->shadows.back()) {
            for (xyz_ctx *x : s->views)
                xyz_destroy(x);
            for (xyz_ctx *x : s->shadows)
                ctx_sizing_free(x);
            delete s;
            return fail(XYZ_ENOMEM, "host allocation failed");
        }
    }
    for (int w = 0; w < workers; ++w)
        s->threads.emplace_back(worker_main, s, w);
    *out = s;
    return XYZ_OK;
}

int xyz_server_add_dataset(xyz_server *s, const int8_t *X, const int8_t *Y, int64_t n, int64_t p,
                           int32_t *dataset)
{
    if (!s || !dataset)
        return fail(XYZ_EINVAL, "null pointer argument");
    xyz_ctx *c = nullptr;
    int rc = xyz_create(X, Y, n, p, &c);
    if (rc)
        return rc;
    int64_t bytes = 0;
    xyz_info(c, nullptr, nullptr, &bytes);
    std::lock_guard<std::mutex> lk(s->mu);
    if (datasets_bytes(s) + bytes > s->budget) {
        xyz_destroy(c);
        return fail(XYZ_ENOMEM, "dataset does not fit the server's device memory budget");
    }
    s->datasets.push_back(Dataset{c, bytes});
    *dataset = (int32_t)s->datasets.size() - 1;
    return XYZ_OK;
}

int xyz_server_submit(xyz_server *s, int32_t dataset, const int8_t *Y, int32_t L, int32_t M,
                      double kappa, uint64_t seed, int64_t *request)
{
    if (!s || !request)
        return fail(XYZ_EINVAL, "null pointer argument");
    if (L < 1 || M < 0 || M > XYZ_MAX_M || !(kappa >= -1.0 && kappa <= 1.0))
        return fail(XYZ_EINVAL, "bad L, M or kappa");
    xyz_ctx *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (dataset < 0 || dataset >= (int32_t)s->datasets.size())
            return fail(XYZ_EINVAL, "unknown dataset");
        base = s->datasets[dataset].base;
    }
    const Packed &pk = *ctx_packed(base);
    uint32_t *yb = nullptr;
    if (Y) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            yb = take_yb(s, (size_t)pk.Wp * 4);
        }
        if (!yb)
            return fail(XYZ_ENOMEM, "cudaMalloc of a request's response failed");
        int rc;
        {
            std::lock_guard<std::mutex> plk(s->pack_mu);
            rc = pack_response(base, Y, yb);
        }
        if (rc) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->yb_free.emplace_back((size_t)pk.Wp * 4, yb);
            return rc;
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    Request r;
    r.id = s->next_id++;
    r.dataset = dataset;
    r.yb = yb;
    r.L = L;
    r.M = M;
    r.kappa = kappa;
    r.seed = seed;
    r.t_submit = Clock::now();       // the reservation is sized at admission
    if (!s->started) {
        s->started = true;
        s->first_submit = r.t_submit;
    }
    s->reqs[r.id] = std::move(r);
    s->queued.push_back(*request = s->next_id - 1);
    admit(s);
    s->cv_work.notify_all();
    return XYZ_OK;
}

int xyz_server_wait(xyz_server *s, int64_t request, int64_t timeout_ms, xyz_pair **pairs,
                    int64_t *npairs, double *latency_ms)
{
    if (!s)
        return fail(XYZ_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto done = [&] {
        auto it = s->reqs.find(request);
        return it == s->reqs.end() || it->second.state == RQ_DONE || it->second.state == RQ_CANCELED ||
               it->second.state == RQ_FAILED;
    };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, done);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
        return fail(XYZ_ETIMEDOUT, "request not finished within the timeout");
    auto it = s->reqs.find(request);
    if (it == s->reqs.end())
        return fail(XYZ_EINVAL, "unknown request");
    return take_result(s, it->second, pairs, npairs, latency_ms);
}

int xyz_server_poll(xyz_server *s, int64_t request, xyz_pair **pairs, int64_t *npairs, double *latency_ms)
{
    if (!s)
        return fail(XYZ_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(request);
    if (it == s->reqs.end())
        return fail(XYZ_EINVAL, "unknown request");
    ReqState st = it->second.state;
    if (st == RQ_QUEUED || st == RQ_ACTIVE)
        return fail(XYZ_EAGAIN, "request not finished");
    return take_result(s, it->second, pairs, npairs, latency_ms);
}

int xyz_server_cancel(xyz_server *s, int64_t request)
{
    if (!s)
        return fail(XYZ_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(request);
    if (it == s->reqs.end())
        return fail(XYZ_EINVAL, "unknown request");
    Request &r = it->second;
    if (r.state == RQ_QUEUED || r.state == RQ_ACTIVE) {
        r.cancel = true;
        if (r.state == RQ_QUEUED) {
            s->queued.erase(std::find(s->queued.begin(), s->queued.end(), request));
            r.state = RQ_CANCELED;
            r.t_done = Clock::now();
            s->canceled++;
            release_yb(s, r);
            s->cv_done.notify_all();
        } else if (r.slices_done == r.slices_out) {
            auto a = std::find(s->active.begin(), s->active.end(), request);
            if (a != s->active.end())
                s->active.erase(a);
            finish(s, r);
        }
    }
    return XYZ_OK;
}

int xyz_server_get_stats(xyz_server *s, xyz_server_stats *out)
{
    if (!s || !out)
        return fail(XYZ_EINVAL, "null pointer argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->completed = s->completed;
    out->canceled = s->canceled;
    out->failed = s->failed;
    out->queued = (int64_t)s->queued.size();
    int64_t act = 0;
    for (auto &kv : s->reqs)
        act += kv.second.state == RQ_ACTIVE;
    out->active = act;
    out->device_bytes = in_use(s);
    out->budget_bytes = s->budget;
    std::vector<double> l = s->latencies;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) {
            double x = q * (double)(l.size() - 1);
            size_t i = (size_t)x;
            double f = x - (double)i;
            return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
    }
    out->pairs_screened = s->pairs_screened;
    if (s->started && s->completed)
        out->elapsed_ms = ms_since(s->first_submit, s->last_done);
    return XYZ_OK;
}

void xyz_server_destroy(xyz_server *s)
{
    if (!s)
        return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    for (std::thread &t : s->threads)
        t.join();
    for (xyz_ctx *v : s->views)
        xyz_destroy(v);
    for (xyz_ctx *x : s->shadows)
        ctx_sizing_free(x);
    for (auto &kv : s->reqs)
        if (kv.second.yb)
            cudaFree(kv.second.yb);
    for (auto &f : s->yb_free)
        cudaFree(f.second);
    for (Dataset &d : s->datasets)
        xyz_destroy(d.base);
    delete s;
}

}  // extern "C"
