// Continuous-batching pricing server over the exhaustive path sums.
//
// Requests arrive one option at a time (bt_submit). A scheduler thread
//  - admits waiting requests in arrival order while a slot is free and the
//    device pool has room for the request's tables and per-item partials,
//    and builds their tables on a set-up stream;
//  - keeps up to n_streams path-sum launches in flight, each over work items
//    drawn from every admitted request (smallest remaining work first), so
//    requests that arrive while others run are admitted and share the GPU;
//  - enqueues the fixed-order reduction of a request's partials (the same
//    reduction as bt_price_exact, so a result does not depend on the mix it
//    ran in) and the copy of its result to the host on the stream of the
//    launch that holds its last items, after that stream has waited for the
//    other launches holding its items; one event per launch then completes
//    the request, and its memory and slot are freed.
// Every wait in the server is bounded (BT_ETIMEOUT).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "host_common.h"

// Pool offsets are 256-byte aligned; every element type must divide that.
static_assert(256 % sizeof(bt_pentry) == 0 && 256 % sizeof(bt_pow) == 0 && 256 % sizeof(double2) == 0 &&
                  256 % sizeof(float2) == 0 && 256 % sizeof(double) == 0,
              "pool element sizes");

namespace {

using clk = std::chrono::steady_clock;

// Longest wait for the set-up stream (the tables of one admission) before the
// server fails with BT_ETIMEOUT.
#define BT_SETUP_WAIT_MS 10000
size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }
double ms_between(clk::time_point a, clk::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// First-fit sub-allocator over [0, size) with coalescing, 256-byte granules.
struct pool_alloc {
    std::map<size_t, size_t> free_;  // offset -> size
    void init(size_t size) { free_.clear(); free_[0] = size; }
    bool alloc(size_t bytes, size_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                size_t rest = it->second - bytes;
                size_t noff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[noff] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

enum req_state { RQ_PENDING, RQ_ACTIVE, RQ_FINALIZING, RQ_DONE, RQ_FAILED };

struct request {
    uint64_t ticket;
    bt_option opt;
    bt_job job;  // shape and table offsets (pool-relative)
    int prec = BT_PREC_FP32_COMP;
    int slot = -1;
    size_t mem_off = 0, mem_bytes = 0;
    int64_t next_item = 0, done_items = 0;
    uint32_t inflight = 0;  // launch slots whose launch in flight holds items of this request
    req_state state = RQ_PENDING;
    bt_result result;
    bt_status status = BT_OK;
    clk::time_point t_arrive, t_done;
};

struct launch_slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    bt_job *h_jobs = nullptr;  // pinned
    bt_job *d_jobs = nullptr;
    unsigned long long *d_counter = nullptr;
    std::vector<std::pair<uint64_t, int64_t>> parts;  // (ticket, items in this launch)
    bt_job *h_fin_jobs = nullptr, *d_fin_jobs = nullptr;  // reductions enqueued after the launch
    bt_result *h_out = nullptr, *d_out = nullptr;
    std::vector<uint64_t> fin;                         // requests completed by this launch
};

}  // namespace

struct bt_server {
    bt_ctx *ctx;
    bt_server_cfg cfg;
    char *pool = nullptr;
    size_t pool_bytes = 0, fixed_bytes = 0;
    pool_alloc palloc;
    bt_option *d_opts = nullptr;   // slot-indexed
    bt_jparams *d_prm = nullptr;   // slot-indexed
    std::vector<int> free_slots;
    cudaStream_t setup_stream = nullptr;
    cudaEvent_t setup_done = nullptr;
    bt_job *h_setup_jobs = nullptr, *d_setup_jobs = nullptr;
    bt_option *h_setup_opts = nullptr;
    std::vector<launch_slot> slots;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> pending;
    std::vector<uint64_t> active;
    std::unordered_map<uint64_t, request> reqs;
    uint64_t next_ticket = 1;
    bool stopping = false;
    std::thread th;
    bt_status fatal = BT_OK;
    char fatal_msg[256] = {0};

    // statistics
    std::vector<double> lat_ms;
    std::vector<std::pair<uint64_t, clk::time_point>> done_log;  // (ticket, completion), completion order
    int64_t submitted = 0, completed = 0, launches = 0, items_done = 0;
    int32_t peak_active = 0;
    double paths_done = 0.0;
    clk::time_point t_first, t_last;
    bool any = false;
    double busy_s = 0.0;
};

static void server_loop(bt_server *S);

static bt_status server_fail(bt_server *S, bt_status s, const char *what) {
    S->fatal = s;
    snprintf(S->fatal_msg, sizeof(S->fatal_msg), "%s", what);
    return s;
}

extern "C" bt_status bt_server_start(bt_ctx *ctx, const bt_server_cfg *cfg_in, bt_server **out) {
    if (!ctx || !out) return bt_fail(BT_EINVAL, "bt_server_start: bad arguments");
    *out = nullptr;
    bt_server_cfg cfg;
    if (cfg_in) cfg = *cfg_in;
    else memset(&cfg, 0, sizeof(cfg));
    if (cfg.max_active <= 0) cfg.max_active = 1024;
    if (cfg.n_streams <= 0) cfg.n_streams = 6;
    if (cfg.max_items_per_launch <= 0) cfg.max_items_per_launch = 4864;  // 16 waves of 304 blocks
    if (cfg.device_budget_bytes == 0) cfg.device_budget_bytes = (size_t)8 << 30;
    if (cfg.use_fp64 != 0 && cfg.use_fp64 != 1) return bt_fail(BT_EINVAL, "bt_server_start: use_fp64 must be 0 or 1");
    if (cfg.max_active > 65536 || cfg.n_streams > 16)
        return bt_fail(BT_EINVAL, "bt_server_start: max_active <= 65536, n_streams <= 16");
    bt_server *S = new (std::nothrow) bt_server();
    if (!S) return bt_fail(BT_ENOMEM, "bt_server_start: host allocation");
    S->ctx = ctx;
    S->cfg = cfg;
    cudaSetDevice(ctx->device);
    const int A = cfg.max_active;
    // fixed device arrays (slots) followed by the pool for tables and partials
    S->fixed_bytes = up256(sizeof(bt_option) * A) + up256(sizeof(bt_jparams) * A) + up256(sizeof(bt_job) * A) +
                     (size_t)cfg.n_streams * (2 * up256(sizeof(bt_job) * A) + up256(sizeof(bt_result) * A) + 256);
    if (S->fixed_bytes >= cfg.device_budget_bytes) {
        delete S;
        return bt_fail(BT_EBUDGET, "bt_server_start: budget below the fixed arrays");
    }
    S->pool_bytes = cfg.device_budget_bytes - S->fixed_bytes;
    void *mem = nullptr;
    bt_status s = ctx_alloc(ctx, cfg.device_budget_bytes, &mem);
    if (s != BT_OK) {
        delete S;
        return s;
    }
    char *p = (char *)mem;
    S->d_opts = (bt_option *)p; p += up256(sizeof(bt_option) * A);
    S->d_prm = (bt_jparams *)p; p += up256(sizeof(bt_jparams) * A);
    S->d_setup_jobs = (bt_job *)p; p += up256(sizeof(bt_job) * A);
    S->slots.resize(cfg.n_streams);
    cudaError_t e = cudaSuccess;
    for (auto &L : S->slots) {
        L.d_jobs = (bt_job *)p; p += up256(sizeof(bt_job) * A);
        L.d_fin_jobs = (bt_job *)p; p += up256(sizeof(bt_job) * A);
        L.d_out = (bt_result *)p; p += up256(sizeof(bt_result) * A);
        L.d_counter = (unsigned long long *)p; p += 256;
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&L.h_jobs, sizeof(bt_job) * A);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&L.h_fin_jobs, sizeof(bt_job) * A);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&L.h_out, sizeof(bt_result) * A);
    }
    S->pool = p;
    S->palloc.init(S->pool_bytes & ~(size_t)255);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->setup_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->setup_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&S->h_setup_jobs, sizeof(bt_job) * A);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&S->h_setup_opts, sizeof(bt_option) * A);
    if (e == cudaSuccess) e = cudaEventRecord(S->setup_done, S->setup_stream);
    if (e != cudaSuccess) {
        bt_status r = bt_cuda_fail(e, "bt_server_start");
        S->stopping = true;
        bt_server_stop(S);
        return r;
    }
    for (int i = A - 1; i >= 0; --i) S->free_slots.push_back(i);
    S->th = std::thread(server_loop, S);
    *out = S;
    return BT_OK;
}

// Bytes a request needs in the pool: tables and per-item partials.
static size_t request_bytes(const bt_job &J, int prec, size_t *o_suf, size_t *o_ph, size_t *o_pm, size_t *o_pw,
                            size_t *o_part) {
    size_t off = 0;
    *o_suf = off; off = up256(off + (prec == BT_PREC_FP64 ? sizeof(double) : sizeof(float2)) * J.suf_len);
    *o_ph = off; off = up256(off + sizeof(bt_pentry) * ((size_t)1 << J.H));
    *o_pm = off; off = up256(off + sizeof(bt_pentry) * ((size_t)1 << J.M));
    *o_pw = off; off = up256(off + sizeof(bt_pow) * (size_t)(2 * J.N + 3 + J.geo_len));
    *o_part = off; off = up256(off + sizeof(double2) * (size_t)J.n_items);
    return off;
}

extern "C" bt_status bt_submit(bt_server *S, const bt_option *opt, bt_precision prec, uint64_t *ticket) {
    if (!S || !opt || !ticket) return bt_fail(BT_EINVAL, "bt_submit: bad arguments");
    if (prec != BT_PREC_FP64 && prec != BT_PREC_FP32_COMP) return bt_fail(BT_EINVAL, "bt_submit: bad precision %d", (int)prec);
    bt_status s = validate_option(opt, 0, BT_MAX_N_EXACT);
    if (s != BT_OK) return s;
    if (prec == BT_PREC_FP32_COMP) {
        double u, d, p;
        host_tree(opt, &u, &d, &p);
        if (p < 0.004 || 1.0 - p < 0.004)
            return bt_fail(BT_EUNSUPPORTED, "bt_submit: p = %.6g; FP32_COMP needs min(p,1-p) >= 0.004", p);
    }
    request r;
    memset(&r.job, 0, sizeof(r.job));
    int step = 1;
    plan_one_job(opt, 1, 0, &r.job, &step, prec);
    r.prec = prec;
    size_t a, b, c, d, e;
    r.mem_bytes = request_bytes(r.job, prec, &a, &b, &c, &d, &e);
    if (r.mem_bytes > S->pool_bytes)
        return bt_fail(BT_EBUDGET, "bt_submit: request needs %zu bytes, pool holds %zu", r.mem_bytes, S->pool_bytes);
    r.opt = *opt;
    r.t_arrive = clk::now();
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stopping) return bt_fail(BT_EINVAL, "bt_submit: server is stopping");
    if (S->fatal != BT_OK) return bt_fail(S->fatal, "bt_submit: server failed: %s", S->fatal_msg);
    r.ticket = S->next_ticket++;
    *ticket = r.ticket;
    if (!S->any) {
        S->t_first = r.t_arrive;
        S->any = true;
    }
    S->reqs.emplace(r.ticket, r);
    S->pending.push_back(r.ticket);
    S->submitted++;
    S->cv_work.notify_one();
    return BT_OK;
}

extern "C" bt_status bt_poll(bt_server *S, uint64_t ticket, bt_result *out, int32_t *done) {
    if (!S || !out || !done) return bt_fail(BT_EINVAL, "bt_poll: bad arguments");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return bt_fail(BT_EINVAL, "bt_poll: unknown ticket %llu", (unsigned long long)ticket);
    *done = 0;
    if (it->second.state == RQ_DONE || it->second.state == RQ_FAILED) {
        *done = 1;
        *out = it->second.result;
        bt_status st = it->second.status;
        S->reqs.erase(it);
        return st;
    }
    return BT_OK;
}

extern "C" bt_status bt_wait(bt_server *S, uint64_t ticket, int32_t timeout_ms, bt_result *out) {
    if (!S || !out) return bt_fail(BT_EINVAL, "bt_wait: bad arguments");
    std::unique_lock<std::mutex> lock(S->mu);
    auto deadline = clk::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    for (;;) {
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return bt_fail(BT_EINVAL, "bt_wait: unknown ticket %llu", (unsigned long long)ticket);
        if (it->second.state == RQ_DONE || it->second.state == RQ_FAILED) {
            *out = it->second.result;
            bt_status st = it->second.status;
            S->reqs.erase(it);
            return st == BT_OK ? BT_OK : bt_fail(st, "request %llu failed", (unsigned long long)ticket);
        }
        if (S->fatal != BT_OK) return bt_fail(S->fatal, "bt_wait: server failed: %s", S->fatal_msg);
        if (S->cv_done.wait_until(lock, deadline) == std::cv_status::timeout) {
            auto it2 = S->reqs.find(ticket);
            if (it2 != S->reqs.end() && (it2->second.state == RQ_DONE || it2->second.state == RQ_FAILED)) continue;
            return bt_fail(BT_ETIMEOUT, "bt_wait: ticket %llu not done after %d ms", (unsigned long long)ticket,
                           timeout_ms);
        }
    }
}

extern "C" bt_status bt_server_stats(bt_server *S, bt_server_stats_t *st) {
    if (!S || !st) return bt_fail(BT_EINVAL, "bt_server_stats: bad arguments");
    std::lock_guard<std::mutex> lock(S->mu);
    memset(st, 0, sizeof(*st));
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->launches = S->launches;
    st->items = S->items_done;
    st->active = (int32_t)S->active.size();
    st->pending = (int32_t)S->pending.size();
    if (!S->lat_ms.empty()) {
        std::vector<double> v = S->lat_ms;
        std::sort(v.begin(), v.end());
        auto q = [&](double f) { return v[std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5))]; };
        st->p50_ms = q(0.50);
        st->p99_ms = q(0.99);
        st->max_ms = v.back();
        double sum = 0.0;
        for (double x : v) sum += x;
        st->mean_ms = sum / (double)v.size();
        const double span = ms_between(S->t_first, S->t_last) / 1e3;
        if (span > 0) {
            st->throughput_rps = (double)S->completed / span;
            st->paths_per_s = S->paths_done / span;
        }
    }
    st->busy_s = S->busy_s;
    st->peak_active = S->peak_active;
    st->pool_bytes = (int64_t)S->pool_bytes;
    return BT_OK;
}

extern "C" bt_status bt_server_stop(bt_server *S) {
    if (!S) return BT_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stopping = true;
        S->cv_work.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    cudaSetDevice(S->ctx->device);
    for (auto &L : S->slots) {
        if (L.stream) cudaStreamSynchronize(L.stream);
        if (L.stream) cudaStreamDestroy(L.stream);
        if (L.done) cudaEventDestroy(L.done);
        if (L.h_jobs) cudaFreeHost(L.h_jobs);
        if (L.h_fin_jobs) cudaFreeHost(L.h_fin_jobs);
        if (L.h_out) cudaFreeHost(L.h_out);
    }
    if (S->setup_stream) {
        cudaStreamSynchronize(S->setup_stream);
        cudaStreamDestroy(S->setup_stream);
    }
    if (S->setup_done) cudaEventDestroy(S->setup_done);
    if (S->h_setup_jobs) cudaFreeHost(S->h_setup_jobs);
    if (S->h_setup_opts) cudaFreeHost(S->h_setup_opts);
    if (S->d_opts) ctx_free(S->ctx, S->d_opts, S->cfg.device_budget_bytes);
    delete S;
    return BT_OK;
}

// ---------------------------------------------------------------------------
// Scheduler
// ---------------------------------------------------------------------------

// Admit pending requests (arrival order) into free slots while the pool has room.
static void admit(bt_server *S) {
    std::vector<uint64_t> admitted;
    std::vector<request *> rq;  // node pointers stay valid while the request is active
    {
        std::lock_guard<std::mutex> lock(S->mu);
        while (!S->pending.empty() && !S->free_slots.empty()) {
            request &r = S->reqs[S->pending.front()];
            size_t off;
            if (!S->palloc.alloc(r.mem_bytes, &off)) break;  // admission by memory
            r.mem_off = off;
            r.slot = S->free_slots.back();
            S->free_slots.pop_back();
            r.state = RQ_ACTIVE;
            S->pending.pop_front();
            admitted.push_back(r.ticket);
            rq.push_back(&r);
        }
    }
    if (admitted.empty()) return;
    // grouped by precision (FP64 = 0 first): one table launch per group
    std::stable_sort(rq.begin(), rq.end(), [](const request *x, const request *y) { return x->prec < y->prec; });
    for (size_t i = 0; i < rq.size(); ++i) admitted[i] = rq[i]->ticket;
    // the pinned staging of the previous admission must have been copied:
    // poll its event with a limit (every wait of the server is bounded)
    cudaError_t e = cudaEventQuery(S->setup_done);
    const auto give_up = clk::now() + std::chrono::milliseconds(BT_SETUP_WAIT_MS);
    while (e == cudaErrorNotReady && clk::now() < give_up) {
        std::this_thread::yield();
        e = cudaEventQuery(S->setup_done);
    }
    if (e == cudaErrorNotReady) {
        std::lock_guard<std::mutex> lock(S->mu);
        server_fail(S, BT_ETIMEOUT, "admission: the set-up stream did not finish its tables in time");
        return;
    }
    // tables of the new requests on the set-up stream; launches wait on its event
    int max_len = 0;
    for (size_t i = 0; i < admitted.size(); ++i) {
        request &r = *rq[i];
        size_t o_suf, o_ph, o_pm, o_pw, o_part;
        request_bytes(r.job, r.prec, &o_suf, &o_ph, &o_pm, &o_pw, &o_part);
        bt_job &J = r.job;
        const size_t pool_off = r.mem_off;  // pool-relative; every part is 256-byte aligned
        J.opt = r.slot;
        J.prm_off = r.slot;
        J.off_suf = (int64_t)((pool_off + o_suf) / 8);     // float2 / double elements
        J.off_ph = (int64_t)((pool_off + o_ph) / sizeof(bt_pentry));
        J.off_pm = (int64_t)((pool_off + o_pm) / sizeof(bt_pentry));
        J.off_pow = (int64_t)((pool_off + o_pw) / sizeof(bt_pow));
        J.off_geo = J.off_pow + 2 * J.N + 3;
        J.part_off = (int64_t)((pool_off + o_part) / sizeof(double2));
        J.item_begin = 0;
        J.item_offset = 0;
        J.out_call = J.out_call >= 0 ? 0 : -1;
        J.out_put = J.out_put >= 0 ? 0 : -1;
        S->h_setup_jobs[i] = J;
        S->h_setup_opts[i] = r.opt;
        int64_t len = (1ll << J.L) + J.suf_len + (1ll << J.H) + (1ll << J.M) + 2 * J.N + 3 + J.geo_len;
        if (len > max_len) max_len = (int)len;
    }
    const int na = (int)admitted.size();
    cudaStream_t st = S->setup_stream;
    // options go to their slots; params are written to the slots by k_params (prm_off = slot)
    for (int i = 0; i < na && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(S->d_opts + S->h_setup_jobs[i].opt, &S->h_setup_opts[i], sizeof(bt_option),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->d_setup_jobs, S->h_setup_jobs, sizeof(bt_job) * na, cudaMemcpyHostToDevice, st);
    int le = e == cudaSuccess ? bt_launch_params(S->d_opts, S->d_setup_jobs, S->d_prm, na, st) : (int)e;
    // rq is sorted with FP64 (prec 0) first: tables per precision group
    for (int i0 = 0; i0 < na && !le;) {
        int i1 = i0;
        while (i1 < na && rq[i1]->prec == rq[i0]->prec) ++i1;
        le = bt_launch_tables(S->d_setup_jobs + i0, S->d_prm, i1 - i0, max_len, rq[i0]->prec, (float2 *)S->pool,
                              (double *)S->pool, (bt_pentry *)S->pool, (bt_pentry *)S->pool, (bt_pow *)S->pool, st);
        i0 = i1;
    }
    if (!le) le = (int)cudaEventRecord(S->setup_done, st);
    std::lock_guard<std::mutex> lock(S->mu);
    if (le) {
        server_fail(S, BT_ECUDA, cudaGetErrorString((cudaError_t)le));
        return;
    }
    for (uint64_t t : admitted) S->active.push_back(t);
    S->peak_active = std::max(S->peak_active, (int32_t)S->active.size());
}

// Build and launch one path-sum launch over items of the active requests;
// requests whose last items are in it get their reduction and result copy
// enqueued behind it on the same stream.
static bool launch_work(bt_server *S, launch_slot &L, int li) {
    std::vector<std::pair<request *, int64_t>> pick;
    int prec = BT_PREC_FP32_COMP;
    std::vector<request *> fin;
    uint32_t wait_mask = 0;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        std::vector<request *> cand;
        for (uint64_t t : S->active) {
            request &r = S->reqs[t];
            if (r.state == RQ_ACTIVE && r.next_item < r.job.n_items) cand.push_back(&r);
        }
        if (cand.empty()) return false;
        // smallest remaining work first
        std::sort(cand.begin(), cand.end(), [](request *a, request *b) {
            const int64_t ra = a->job.n_items - a->next_item, rb = b->job.n_items - b->next_item;
            return ra != rb ? ra < rb : a->ticket < b->ticket;
        });
        int64_t budget = S->cfg.max_items_per_launch;
        prec = cand[0]->prec;  // a launch runs one precision's kernel
        for (request *r : cand) {
            if (r->prec != prec) continue;
            if (budget <= 0 || (int)pick.size() >= S->cfg.max_active) break;
            const int64_t take = std::min<int64_t>(budget, r->job.n_items - r->next_item);
            pick.push_back({r, take});
            budget -= take;
        }
        for (auto &pr : pick) {
            request *r = pr.first;
            if (r->next_item + pr.second == r->job.n_items) {
                fin.push_back(r);
                wait_mask |= r->inflight;  // other launches that hold its earlier items
            }
            r->inflight |= 1u << li;
        }
    }
    int64_t cursor = 0;
    L.parts.clear();
    L.fin.clear();
    for (size_t i = 0; i < pick.size(); ++i) {
        request *r = pick[i].first;
        bt_job J = r->job;
        J.item_begin = cursor;
        J.item_offset = r->next_item;
        L.h_jobs[i] = J;
        cursor += pick[i].second;
        L.parts.push_back({r->ticket, pick[i].second});
    }
    for (size_t k = 0; k < fin.size(); ++k) {
        bt_job J = fin[k]->job;
        J.out_call = J.out_call >= 0 ? (int)k : -1;
        J.out_put = J.out_put >= 0 ? (int)k : -1;
        L.h_fin_jobs[k] = J;
        L.fin.push_back(fin[k]->ticket);
    }
    {
        std::lock_guard<std::mutex> lock(S->mu);
        for (auto &pr : pick) pr.first->next_item += pr.second;
    }
    const int nj = (int)pick.size(), nf = (int)fin.size();
    cudaError_t e = cudaStreamWaitEvent(L.stream, S->setup_done, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.d_jobs, L.h_jobs, sizeof(bt_job) * nj, cudaMemcpyHostToDevice, L.stream);
    if (e == cudaSuccess && nf)
        e = cudaMemcpyAsync(L.d_fin_jobs, L.h_fin_jobs, sizeof(bt_job) * nf, cudaMemcpyHostToDevice, L.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.d_counter, 0, sizeof(unsigned long long), L.stream);
    int le = (int)e;
    if (!le) {
        bt_exact_args a;
        memset(&a, 0, sizeof(a));
        a.opts = S->d_opts;
        a.jobs = L.d_jobs;
        a.prm = S->d_prm;
        a.n_jobs = nj;
        a.shard = 0;
        a.n_shards = 1;
        a.n_run_items = cursor;
        a.suf32 = (const float2 *)S->pool;
        a.suf64 = (const double *)S->pool;
        a.ph = (const bt_pentry *)S->pool;
        a.pm = (const bt_pentry *)S->pool;
        a.pw = (const bt_pow *)S->pool;
        a.partials = (double2 *)S->pool;
        a.counter = L.d_counter;
        le = bt_launch_exact(&a, prec, prec == BT_PREC_FP64 ? S->ctx->grid64 : S->ctx->grid32, L.stream);
    }
    if (!le && nf) {
        // the other launches holding items of these requests are in flight on
        // their own streams; their events were recorded when they launched
        for (int o = 0; o < (int)S->slots.size() && !le; ++o)
            if (o != li && (wait_mask >> o & 1u)) le = (int)cudaStreamWaitEvent(L.stream, S->slots[o].done, 0);
        if (!le)
            le = bt_launch_finalize(L.d_fin_jobs, S->d_prm, nf, (const double2 *)S->pool, 0, 1, prec, L.d_out,
                                    L.stream);
        if (!le) le = (int)cudaMemcpyAsync(L.h_out, L.d_out, sizeof(bt_result) * nf, cudaMemcpyDeviceToHost, L.stream);
    }
    if (!le) le = (int)cudaEventRecord(L.done, L.stream);
    std::lock_guard<std::mutex> lock(S->mu);
    if (le) {
        server_fail(S, BT_ECUDA, cudaGetErrorString((cudaError_t)le));
        return false;
    }
    L.busy = true;
    S->launches++;
    return true;
}

// Completed launches: count items, complete the requests they finalised.
static bool reap_work(bt_server *S) {
    bool any = false;
    for (int li = 0; li < (int)S->slots.size(); ++li) {
        launch_slot &L = S->slots[li];
        if (!L.busy) continue;
        cudaError_t q = cudaEventQuery(L.done);
        if (q == cudaErrorNotReady) continue;
        std::lock_guard<std::mutex> lock(S->mu);
        L.busy = false;
        if (q != cudaSuccess) {
            server_fail(S, BT_ECUDA, cudaGetErrorString(q));
            continue;
        }
        for (auto &pt : L.parts) {
            S->items_done += pt.second;
            // a request finalised on another stream may be collected already
            auto it = S->reqs.find(pt.first);
            if (it == S->reqs.end()) continue;
            it->second.done_items += pt.second;
            it->second.inflight &= ~(1u << li);
        }
        const auto now = clk::now();
        for (size_t k = 0; k < L.fin.size(); ++k) {
            request &r = S->reqs[L.fin[k]];
            r.result = L.h_out[k];
            r.state = RQ_DONE;
            r.t_done = now;
            S->palloc.release(r.mem_off, r.mem_bytes);
            S->free_slots.push_back(r.slot);
            S->lat_ms.push_back(ms_between(r.t_arrive, now));
            S->done_log.push_back({r.ticket, now});
            S->completed++;
            S->paths_done += (double)r.result.paths;
            S->t_last = now;
            S->active.erase(std::find(S->active.begin(), S->active.end(), r.ticket));
        }
        if (!L.fin.empty()) S->cv_done.notify_all();
        any = true;
    }
    return any;
}

static void server_loop(bt_server *S) {
    cudaSetDevice(S->ctx->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lock(S->mu);
            if (S->fatal != BT_OK) {
                // fail every outstanding request so waiters return
                for (auto &kv : S->reqs)
                    if (kv.second.state != RQ_DONE) {
                        kv.second.state = RQ_FAILED;
                        kv.second.status = S->fatal;
                    }
                S->cv_done.notify_all();
                if (S->stopping) return;
                S->cv_work.wait_for(lock, std::chrono::milliseconds(50));
                continue;
            }
            const bool idle = S->pending.empty() && S->active.empty();
            if (S->stopping && idle) return;
            if (idle) {
                S->cv_work.wait_for(lock, std::chrono::milliseconds(20));
                continue;
            }
        }
        const auto t0 = clk::now();
        bool progress = reap_work(S);
        admit(S);
        for (int li = 0; li < (int)S->slots.size(); ++li)
            if (!S->slots[li].busy && launch_work(S, S->slots[li], li)) progress = true;
        bool busy = false;
        for (auto &L : S->slots) busy |= L.busy;
        if (busy) {
            std::lock_guard<std::mutex> lock(S->mu);
            S->busy_s += std::chrono::duration<double>(clk::now() - t0).count();
        }
        // poll the launch events while work is in flight; otherwise back off
        if (!progress) {
            if (busy) std::this_thread::yield();
            else std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
}

// ---------------------------------------------------------------------------
// Replay of an arrival schedule: batched (through the server) or plain (one
// bt_price_exact per request, first come first served). Latency = completion
// minus scheduled arrival, on the same clock for both.
// ---------------------------------------------------------------------------
extern "C" bt_status bt_serve_replay(bt_ctx *ctx, const bt_server_cfg *cfg, const bt_option *opts,
                                     const double *arrival_s, int32_t n, int32_t mode, bt_result *results,
                                     double *latency_ms, double *wall_s) {
    if (!ctx || !opts || !arrival_s || n < 1 || !results || !latency_ms)
        return bt_fail(BT_EINVAL, "bt_serve_replay: bad arguments");
    const auto t0 = clk::now();
    auto at = [&](int i) { return t0 + std::chrono::duration_cast<clk::duration>(std::chrono::duration<double>(arrival_s[i])); };
    if (mode == 0) {  // plain: one synchronous launch per request, FIFO
        bt_precision prec = cfg && cfg->use_fp64 ? BT_PREC_FP64 : BT_PREC_FP32_COMP;
        for (int i = 0; i < n; ++i) {
            std::this_thread::sleep_until(at(i));
            bt_status s = bt_price_exact(ctx, &opts[i], 1, prec, &results[i], nullptr);
            if (s != BT_OK) return s;
            latency_ms[i] = ms_between(at(i), clk::now());
        }
    } else {
        bt_server *S = nullptr;
        bt_status s = bt_server_start(ctx, cfg, &S);
        if (s != BT_OK) return s;
        std::vector<uint64_t> tickets(n);
        bt_status rs = BT_OK;  // the first failure, submission or result, and its message
        int r_idx = -1;
        std::string r_msg;
        std::thread submitter([&]() {
            for (int i = 0; i < n; ++i) {
                std::this_thread::sleep_until(at(i));
                const bt_status ss =
                    bt_submit(S, &opts[i], cfg && cfg->use_fp64 ? BT_PREC_FP64 : BT_PREC_FP32_COMP, &tickets[i]);
                if (ss != BT_OK) {
                    tickets[i] = 0;
                    if (rs == BT_OK) {
                        rs = ss;
                        r_idx = i;
                        r_msg = bt_last_error(ctx);  // the submitting thread's message
                    }
                }
            }
        });
        submitter.join();
        for (int i = 0; i < n; ++i) {
            if (!tickets[i]) continue;
            s = bt_wait(S, tickets[i], 600000, &results[i]);
            if (s != BT_OK && rs == BT_OK) {
                rs = s;
                r_idx = i;
                r_msg = bt_last_error(ctx);
            }
        }
        std::unordered_map<uint64_t, clk::time_point> done;
        {
            std::lock_guard<std::mutex> lock(S->mu);
            for (auto &d : S->done_log) done[d.first] = d.second;
        }
        bt_server_stop(S);
        if (rs != BT_OK) return bt_fail(rs, "bt_serve_replay: request %d: %s", r_idx, r_msg.c_str());
        for (int i = 0; i < n; ++i) {
            auto it = done.find(tickets[i]);
            latency_ms[i] = it == done.end() ? -1.0 : ms_between(at(i), it->second);
        }
    }
    if (wall_s) *wall_s = std::chrono::duration<double>(clk::now() - t0).count();
    return BT_OK;
}
