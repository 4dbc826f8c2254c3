// Host runtime of libbtree: validation, planning of the prefix/suffix split,
// device memory (within the context's budget) and kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "bt_internal.h"
#include "host_common.h"

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512];

bt_status bt_fail(bt_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}
bt_status bt_cuda_fail(int err, const char *what) {
    return bt_fail(BT_ECUDA, "%s: %s", what, cudaGetErrorString((cudaError_t)err));
}

extern "C" const char *bt_last_error(const bt_ctx *) { return g_err; }
extern "C" const char *bt_version(void) { return "libbtree 0.1 (sm_103a)"; }
extern "C" const char *bt_status_str(bt_status s) {
    switch (s) {
    case BT_OK: return "BT_OK";
    case BT_EINVAL: return "BT_EINVAL";
    case BT_ENOMEM: return "BT_ENOMEM";
    case BT_EBUDGET: return "BT_EBUDGET";
    case BT_ECUDA: return "BT_ECUDA";
    case BT_ETIMEOUT: return "BT_ETIMEOUT";
    case BT_EUNSUPPORTED: return "BT_EUNSUPPORTED";
    }
    return "BT_UNKNOWN";
}

// ---------------------------------------------------------------------------
// Context and budgeted device memory
// ---------------------------------------------------------------------------
extern "C" bt_status bt_create(int device, size_t budget, bt_ctx **out) {
    if (!out) return bt_fail(BT_EINVAL, "bt_create: out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) return bt_fail(BT_ECUDA, "bt_create: no CUDA device (%s)", cudaGetErrorString(e));
    if (device < 0 || device >= n) return bt_fail(BT_EINVAL, "bt_create: device %d out of range [0,%d)", device, n);
    if ((e = cudaSetDevice(device)) != cudaSuccess) return bt_cuda_fail(e, "cudaSetDevice");
    bt_ctx *c = new (std::nothrow) bt_ctx();
    if (!c) return bt_fail(BT_ENOMEM, "bt_create: host allocation");
    c->device = device;
    c->budget = budget ? budget : ((size_t)8 << 30);
    c->used.store(0);
    if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess) {
        delete c;
        return bt_cuda_fail(e, "cudaStreamCreate");
    }
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device);
    c->grid32 = bt_exact_grid_size(BT_PREC_FP32_COMP, device);
    c->grid64 = bt_exact_grid_size(BT_PREC_FP64, device);
    if (c->grid32 < 0 || c->grid64 < 0) {
        const int err = c->grid32 < 0 ? -c->grid32 : -c->grid64;
        cudaStreamDestroy(c->stream);
        delete c;
        return bt_cuda_fail(err, "bt_create: kernel attributes");
    }
    *out = c;
    return BT_OK;
}

extern "C" void bt_destroy(bt_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->cache) ctx_free(c, c->cache, c->cache_bytes);
    cudaStreamDestroy(c->stream);
    delete c;
}

extern "C" size_t bt_device_bytes(const bt_ctx *c) { return c ? c->used.load() : 0; }

bt_status ctx_alloc(bt_ctx *c, size_t bytes, void **p) {
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    size_t cur = c->used.load();
    do {
        if (cur + bytes > c->budget)
            return bt_fail(BT_EBUDGET, "device budget exceeded: %zu + %zu > %zu bytes", cur, bytes, c->budget);
    } while (!c->used.compare_exchange_weak(cur, cur + bytes));
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        c->used.fetch_sub(bytes);
        *p = nullptr;
        return bt_fail(BT_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    return BT_OK;
}

void ctx_free(bt_ctx *c, void *p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 256;
    cudaFree(p);
    c->used.fetch_sub(bytes);
}

cudaStream_t ctx_stream(bt_ctx *c, void *s) { return s ? (cudaStream_t)s : c->stream; }

// The context's reusable scratch of at least `bytes` (the caller holds
// cache_mu): grown on demand, after the context's stream has drained the work
// that used the old one; freed with the context.
bt_status ctx_scratch(bt_ctx *c, size_t bytes, void **p) {
    if (c->cache_bytes < bytes) {
        if (c->cache) {
            cudaStreamSynchronize(c->stream);
            ctx_free(c, c->cache, c->cache_bytes);
            c->cache = nullptr;
            c->cache_bytes = 0;
        }
        bt_status s = ctx_alloc(c, bytes, &c->cache);
        if (s != BT_OK) return s;
        c->cache_bytes = bytes;
    }
    *p = c->cache;
    return BT_OK;
}

// ---------------------------------------------------------------------------
// Tree parameters on the host (validation) -- Section 2, A1-A3
// ---------------------------------------------------------------------------
static bool finite_all(const bt_option &o) {
    return std::isfinite(o.S0) && std::isfinite(o.K) && std::isfinite(o.rate) && std::isfinite(o.sigma) &&
           std::isfinite(o.T) && std::isfinite(o.u) && std::isfinite(o.d) && std::isfinite(o.p);
}

bt_status host_tree(const bt_option *o, double *u, double *d, double *p) {
    const double dt = o->T / (double)o->N;
    double uu;
    if (o->tree_kind == BT_TREE_CRR) {
        uu = std::exp(o->sigma * std::sqrt(dt));
    } else if (o->tree_kind == BT_TREE_SEYDEL) {
        double beta = 0.5 * (std::exp(-o->rate * dt) + std::exp((o->rate + o->sigma * o->sigma) * dt));
        uu = beta + std::sqrt(beta * beta - 1.0);
    } else {
        *u = o->u;
        *d = o->d;
        *p = o->p;
        return BT_OK;
    }
    double dd = 1.0 / uu;
    double pp = (std::exp(o->rate * dt) - dd) / (uu - dd);
    if (!(pp > 0.0 && pp < 1.0))
        return bt_fail(BT_EINVAL, "risk-neutral p = %.17g is not in (0,1) (sigma too small for the rate?)", pp);
    *u = uu;
    *d = dd;
    *p = pp;
    return BT_OK;
}

bt_status validate_option(const bt_option *o, int idx, int max_n) {
    if (o->N < 1 || o->N > max_n) return bt_fail(BT_EINVAL, "option %d: N=%d outside 1..%d", idx, o->N, max_n);
    if (o->tree_kind < 0 || o->tree_kind > 2) return bt_fail(BT_EINVAL, "option %d: bad tree_kind %d", idx, o->tree_kind);
    if (o->payoff < 0 || o->payoff > 7) return bt_fail(BT_EINVAL, "option %d: bad payoff %d", idx, o->payoff);
    if (!finite_all(*o)) return bt_fail(BT_EINVAL, "option %d: non-finite input", idx);
    if (!(o->S0 > 0.0)) return bt_fail(BT_EINVAL, "option %d: S0 must be > 0", idx);
    if (!(o->K >= 0.0)) return bt_fail(BT_EINVAL, "option %d: K must be >= 0", idx);
    if (!(o->T > 0.0)) return bt_fail(BT_EINVAL, "option %d: T must be > 0", idx);
    if (o->tree_kind == BT_TREE_EXPLICIT) {
        if (!(o->u > 1.0 && o->d > 0.0 && o->p > 0.0 && o->p < 1.0))
            return bt_fail(BT_EINVAL, "option %d: explicit tree needs u > 1, d > 0, 0 < p < 1", idx);
        if (std::fabs(o->u * o->d - 1.0) > 1e-12)
            return bt_fail(BT_EINVAL, "option %d: explicit tree needs u*d = 1 (assumption A1)", idx);
    } else if (!(o->sigma > 0.0)) {
        return bt_fail(BT_EINVAL, "option %d: sigma must be > 0", idx);
    }
    double u, d, p;
    bt_status s = host_tree(o, &u, &d, &p);
    if (s != BT_OK) {
        char why[sizeof(g_err)];
        memcpy(why, g_err, sizeof(why));
        return bt_fail(s, "option %d: %s", idx, why);
    }
    return BT_OK;
}

extern "C" bt_status bt_tree_params(const bt_option *o, double *u, double *d, double *p) {
    if (!o || !u || !d || !p) return bt_fail(BT_EINVAL, "bt_tree_params: NULL argument");
    bt_status s = validate_option(o, 0, 1 << 20);
    if (s != BT_OK) return s;
    return host_tree(o, u, d, p);
}

// ---------------------------------------------------------------------------
// Planning of the exhaustive pass
// ---------------------------------------------------------------------------
static int binom_host(int n, int k) {
    if (k < 0 || k > n) return 0;
    long long r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return (int)r;
}

static bool same_params(const bt_option &a, const bt_option &b) {
    return a.N == b.N && a.tree_kind == b.tree_kind && a.S0 == b.S0 && a.K == b.K && a.rate == b.rate &&
           a.sigma == b.sigma && a.T == b.T && a.u == b.u && a.d == b.d && a.p == b.p;
}

// Payoff -> (suffix field, sign mode) of the affine form in exact.cu.
void payoff_field(int payoff, int *field, int *mode) {
    switch (payoff) {
    case BT_EURO_CALL: *field = BT_F_EURO; *mode = BT_MODE_CALL; break;
    case BT_EURO_PUT: *field = BT_F_EURO; *mode = BT_MODE_PUT; break;
    case BT_ASIAN_ARITH_CALL: *field = BT_F_ARITH; *mode = BT_MODE_CALL; break;
    case BT_ASIAN_ARITH_PUT: *field = BT_F_ARITH; *mode = BT_MODE_PUT; break;
    case BT_ASIAN_GEO_CALL: *field = BT_F_GEO; *mode = BT_MODE_CALL; break;
    case BT_ASIAN_GEO_PUT: *field = BT_F_GEO; *mode = BT_MODE_PUT; break;
    case BT_LOOKBACK_FIXED_CALL: *field = BT_F_LOOKMAX; *mode = BT_MODE_CALL; break;
    default: *field = BT_F_LOOKMIN; *mode = BT_MODE_PUT; break;
    }
}

// L = clamp(N - 15, 1, 13): as many suffix steps as shared memory holds,
// leaving at least 2^15 prefixes (32 work items) where the tree has them, so
// that even one small option spreads over the SMs.
int exact_split_L(int N) { return std::max(1, std::min(BT_MAX_L, N - BT_LOW_BITS - BT_MIN_ITEM_BITS)); }
int exact_split_L_fp64(int N) {
    return std::max(1, std::min(BT_MAX_L, N - BT_LOW_BITS - BT_MIN_ITEM_BITS_FP64));
}

// Recombined suffix classes. For the geometric, European and lookback
// payoffs the suffix factor f_s depends on the suffix only through one
// integer key (level sum, end level, max or min level), so within an up-count
// group (same weight) the suffixes fall into a few classes of equal f_s: at
// L = 13, 14 (European), 62 (lookback) or 378 (geometric) classes instead
// of 8192 suffixes. The FP32 pass then sums multiplicity x payoff over the
// classes in pair arithmetic. The key, its definition and the ordering
// (groups by up-count, keys ascending) are shared with k_class_tables.
static int suffix_key(int field, unsigned s, int L) {
    int lvl = 0, mx = -BT_LVL_NONE, mn = BT_LVL_NONE, D = 0;
    for (int t = 1; t <= L; ++t) {
        lvl += ((s >> (L - t)) & 1u) ? 1 : -1;
        mx = std::max(mx, lvl);
        mn = std::min(mn, lvl);
        D += lvl;
    }
    switch (field) {
    case BT_F_GEO: return D;
    case BT_F_EURO: return lvl;
    case BT_F_LOOKMAX: return mx;
    default: return mn;
    }
}

static bool field_has_classes(int field) { return field != BT_F_ARITH; }

// Number of distinct keys per up-count group, for every field and L (cached).
static const int *class_counts(int field, int L) {
    static int table[5][BT_MAX_L + 1][BT_MAX_L + 1];
    static std::once_flag once;
    std::call_once(once, [] {
        for (int f = 0; f < 5; ++f) {
            if (!field_has_classes(f)) continue;
            for (int l = 1; l <= BT_MAX_L; ++l) {
                std::vector<std::vector<char>> seen(l + 1, std::vector<char>(2 * BT_KEY_SPAN + 1, 0));
                for (unsigned s = 0; s < (1u << l); ++s)
                    seen[__builtin_popcount(s)][suffix_key(f, s, l) + BT_KEY_SPAN] = 1;
                for (int k = 0; k <= l; ++k) {
                    int c = 0;
                    for (char x : seen[k]) c += x;
                    table[f][l][k] = c;
                }
            }
        }
    });
    return table[field][L];
}

bool tree_skewed(const bt_option &o) {
    double u, d, p;
    if (host_tree(&o, &u, &d, &p) != BT_OK) return false;
    const double neff_log2 = -(double)o.N * std::log2(p * p + (1.0 - p) * (1.0 - p));
    return neff_log2 < BT_PER_PATH_MIN_NEFF_LOG2;
}

void fill_job_shape(bt_job &J, int N, int field, int mode, int prec, bool skewed) {
    // Below 2^28 paths the per-path FP32 rounding of the arithmetic Asian
    // averages over too few paths for 1e-9, and so it does on a skewed tree
    // (fewer than 2^BT_PER_PATH_MIN_NEFF_LOG2 effective paths): those jobs
    // take the pair-sum class pass with every suffix its own class
    // (multiplicity 1), which rounds no single path.
    const bool arith_cls =
        prec == BT_PREC_FP32_COMP && field == BT_F_ARITH && (N <= BT_ARITH_CLS_MAX_N || skewed);
    J.N = N;
    J.L = prec == BT_PREC_FP64 ? exact_split_L_fp64(N) : exact_split_L(N);
    if (arith_cls) J.L = std::min(J.L, BT_ARITH_CLS_MAX_L);
    J.P = N - J.L;
    J.M = (J.P + 1) / 2;
    J.H = J.P - J.M;
    J.field = field;
    J.mode = mode;
    int off = 0;
    for (int k = 0; k <= J.L; ++k) {
        J.goff[k] = off;
        int c = binom_host(J.L, k);
        off += (c + BT_UNROLL - 1) / BT_UNROLL * BT_UNROLL;
    }
    for (int k = J.L + 1; k < BT_MAX_L + 2; ++k) J.goff[k] = off;
    J.suf_len = off;
    J.cls = 0;
    if (prec == BT_PREC_FP32_COMP && (field_has_classes(field) || arith_cls)) {
        // class table: goff in class units, two float2 slots per class
        const int *cnt = arith_cls ? nullptr : class_counts(field, J.L);
        off = 0;
        for (int k = 0; k <= J.L; ++k) {
            J.goff[k] = off;
            const int c = arith_cls ? binom_host(J.L, k) : cnt[k];
            off += (c + BT_CLS_UNROLL - 1) / BT_CLS_UNROLL * BT_CLS_UNROLL;
        }
        for (int k = J.L + 1; k < BT_MAX_L + 2; ++k) J.goff[k] = off;
        J.suf_len = 2 * off;
        J.cls = 1;
    }
    if (field == BT_F_GEO) {
        int span = J.P * (J.P + 1) / 2 + J.L * J.P + 1;
        J.geo_imin = -span;
        J.geo_len = 2 * span + 1;
    } else {
        J.geo_imin = 0;
        J.geo_len = 0;
    }
    int64_t nP = 1ll << J.P;
    J.n_items = (int32_t)std::max<int64_t>(1, (nP + (1 << BT_LOW_BITS) - 1) >> BT_LOW_BITS);
}

// Plans the pass that starts at option i (used by the allocation-free entry
// point, which keeps its job list on the stack): the same pairing and split
// rules as plan_jobs. Sets *step to the number of options the pass covers.
void plan_one_job(const bt_option *opts, int n, int i, bt_job *J, int *step, int prec) {
    int field, mode;
    payoff_field(opts[i].payoff, &field, &mode);
    J->opt = i;
    J->out_call = mode == BT_MODE_CALL ? i : -1;
    J->out_put = mode == BT_MODE_PUT ? i : -1;
    *step = 1;
    if (i + 1 < n && field != BT_F_LOOKMAX && field != BT_F_LOOKMIN && same_params(opts[i], opts[i + 1])) {
        int f2, m2;
        payoff_field(opts[i + 1].payoff, &f2, &m2);
        if (f2 == field && m2 != mode) {
            mode = BT_MODE_BOTH;
            if (J->out_call < 0) J->out_call = i + 1;
            else J->out_put = i + 1;
            *step = 2;
        }
    }
    fill_job_shape(*J, opts[i].N, field, mode, prec, tree_skewed(opts[i]));
}

struct bt_exact_plan {
    bt_ctx *ctx;
    int prec;
    int n_opts;
    std::vector<bt_job> jobs;
    int64_t n_items;
    int64_t payoff_paths, path_evals;
    int max_table_len;
    // device arena
    char *arena;
    size_t arena_bytes;
    bt_option *d_opts;
    bt_job *d_jobs;
    bt_jparams *d_prm;
    float2 *d_suf32;
    double *d_suf64;
    bt_pentry *d_ph, *d_pm;
    bt_pow *d_pw;
    double2 *d_partials;
    bt_result *d_out;
    unsigned long long *d_counter;
    cudaEvent_t ev0, ev1;
    bool timed;
    bool cached;  // arena borrowed from the context's scratch (not freed by destroy)
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bt_status plan_jobs(const bt_option *opts, int n, int prec, std::vector<bt_job> &jobs, int64_t *n_items,
                    int64_t *payoff_paths, int64_t *path_evals, int max_n) {
    jobs.clear();
    *payoff_paths = 0;
    *path_evals = 0;
    for (int i = 0; i < n; ++i) {
        bt_status s = validate_option(&opts[i], i, max_n);
        if (s != BT_OK) return s;
        if (prec == BT_PREC_FP32_COMP) {
            double u, d, p;
            host_tree(&opts[i], &u, &d, &p);
            if (std::min(p, 1.0 - p) < 0.004)
                return bt_fail(BT_EUNSUPPORTED,
                               "option %d: p = %.6g; FP32_COMP needs min(p,1-p) >= 0.004 (use BT_PREC_FP64)", i, p);
        }
        *payoff_paths += 1ll << opts[i].N;
    }
    int64_t items = 0;
    int64_t suf = 0, ph = 0, pm = 0, pw = 0;
    for (int i = 0; i < n;) {
        bt_job J;
        memset(&J, 0, sizeof(J));
        int field, mode;
        payoff_field(opts[i].payoff, &field, &mode);
        J.opt = i;
        J.out_call = mode == BT_MODE_CALL ? i : -1;
        J.out_put = mode == BT_MODE_PUT ? i : -1;
        int step = 1;
        if (i + 1 < n && field != BT_F_LOOKMAX && field != BT_F_LOOKMIN && same_params(opts[i], opts[i + 1])) {
            int f2, m2;
            payoff_field(opts[i + 1].payoff, &f2, &m2);
            if (f2 == field && m2 != mode) {
                mode = BT_MODE_BOTH;
                if (J.out_call < 0) J.out_call = i + 1;
                else J.out_put = i + 1;
                step = 2;
            }
        }
        fill_job_shape(J, opts[i].N, field, mode, prec, tree_skewed(opts[i]));
        J.item_begin = items;
        J.item_offset = 0;
        J.part_off = items;
        J.prm_off = (int64_t)jobs.size();
        J.off_suf = suf;
        J.off_ph = ph;
        J.off_pm = pm;
        J.off_pow = pw;
        J.off_geo = pw + 2 * J.N + 3;
        items += J.n_items;
        suf += J.suf_len;
        ph += 1ll << J.H;
        pm += 1ll << J.M;
        pw += 2 * J.N + 3 + J.geo_len;
        *path_evals += 1ll << J.N;
        jobs.push_back(J);
        i += step;
    }
    *n_items = items;
    return BT_OK;
}

static bt_status plan_create(bt_ctx *ctx, const bt_option *opts, int32_t n, bt_precision prec, bool cached,
                             bt_exact_plan **out);

extern "C" bt_status bt_exact_plan_create(bt_ctx *ctx, const bt_option *opts, int32_t n, bt_precision prec,
                                          bt_exact_plan **out) {
    return plan_create(ctx, opts, n, prec, false, out);
}

// cached = true borrows the context's scratch (the caller holds cache_mu).
static bt_status plan_create(bt_ctx *ctx, const bt_option *opts, int32_t n, bt_precision prec, bool cached,
                             bt_exact_plan **out) {
    if (!ctx || !opts || !out || n < 1) return bt_fail(BT_EINVAL, "bt_exact_plan_create: bad arguments");
    if (prec != BT_PREC_FP64 && prec != BT_PREC_FP32_COMP) return bt_fail(BT_EINVAL, "bad precision %d", (int)prec);
    *out = nullptr;
    bt_exact_plan *pl = new (std::nothrow) bt_exact_plan();
    if (!pl) return bt_fail(BT_ENOMEM, "host allocation");
    pl->ctx = ctx;
    pl->prec = prec;
    pl->n_opts = n;
    bt_status s = plan_jobs(opts, n, prec, pl->jobs, &pl->n_items, &pl->payoff_paths, &pl->path_evals, BT_MAX_N_EXACT);
    if (s != BT_OK) {
        delete pl;
        return s;
    }
    const int nj = (int)pl->jobs.size();
    int64_t suf = 0, ph = 0, pm = 0, pw = 0;
    int max_len = 0;
    for (const bt_job &J : pl->jobs) {
        suf += J.suf_len;
        ph += 1ll << J.H;
        pm += 1ll << J.M;
        pw += 2 * J.N + 3 + J.geo_len;
        int64_t len = (1ll << J.L) + J.suf_len + (1ll << J.H) + (1ll << J.M) + 2 * J.N + 3 + J.geo_len;
        max_len = (int)std::max<int64_t>(max_len, len);
    }
    pl->max_table_len = max_len;
    size_t off = 0;
    size_t o_opts = off; off = align256(off + sizeof(bt_option) * n);
    size_t o_jobs = off; off = align256(off + sizeof(bt_job) * nj);
    size_t o_prm = off; off = align256(off + sizeof(bt_jparams) * nj);
    size_t o_suf = off; off = align256(off + (prec == BT_PREC_FP64 ? sizeof(double) : sizeof(float2)) * suf);
    size_t o_ph = off; off = align256(off + sizeof(bt_pentry) * ph);
    size_t o_pm = off; off = align256(off + sizeof(bt_pentry) * pm);
    size_t o_pw = off; off = align256(off + sizeof(bt_pow) * pw);
    size_t o_part = off; off = align256(off + sizeof(double2) * pl->n_items);
    size_t o_out = off; off = align256(off + sizeof(bt_result) * n);
    size_t o_cnt = off; off = align256(off + sizeof(unsigned long long));
    cudaSetDevice(ctx->device);
    void *arena = nullptr;
    if (cached) {
        s = ctx_scratch(ctx, off, &arena);
        if (s != BT_OK) {
            delete pl;
            return s;
        }
        pl->cached = true;
    } else {
        s = ctx_alloc(ctx, off, &arena);
        if (s != BT_OK) {
            delete pl;
            return s;
        }
    }
    pl->arena = (char *)arena;
    pl->arena_bytes = off;
    pl->d_opts = (bt_option *)(pl->arena + o_opts);
    pl->d_jobs = (bt_job *)(pl->arena + o_jobs);
    pl->d_prm = (bt_jparams *)(pl->arena + o_prm);
    pl->d_suf32 = prec == BT_PREC_FP64 ? nullptr : (float2 *)(pl->arena + o_suf);
    pl->d_suf64 = prec == BT_PREC_FP64 ? (double *)(pl->arena + o_suf) : nullptr;
    pl->d_ph = (bt_pentry *)(pl->arena + o_ph);
    pl->d_pm = (bt_pentry *)(pl->arena + o_pm);
    pl->d_pw = (bt_pow *)(pl->arena + o_pw);
    pl->d_partials = (double2 *)(pl->arena + o_part);
    pl->d_out = (bt_result *)(pl->arena + o_out);
    pl->d_counter = (unsigned long long *)(pl->arena + o_cnt);
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaMemcpyAsync(pl->d_opts, opts, sizeof(bt_option) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pl->d_jobs, pl->jobs.data(), sizeof(bt_job) * nj, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        bt_exact_plan_destroy(pl);
        return bt_cuda_fail(e, "bt_exact_plan_create: upload");
    }
    *out = pl;
    return BT_OK;
}

static bt_status plan_enqueue(bt_exact_plan *pl, int shard, int n_shards, void *stream) {
    bt_ctx *c = pl->ctx;
    cudaSetDevice(c->device);
    cudaStream_t st = ctx_stream(c, stream);
    const int nj = (int)pl->jobs.size();
    int e = bt_launch_params(pl->d_opts, pl->d_jobs, pl->d_prm, nj, st);
    if (e) return bt_cuda_fail(e, "params kernel");
    e = bt_launch_tables(pl->d_jobs, pl->d_prm, nj, pl->max_table_len, pl->prec, pl->d_suf32, pl->d_suf64, pl->d_ph,
                         pl->d_pm, pl->d_pw, st);
    if (e) return bt_cuda_fail(e, "tables kernel");
    e = (int)cudaMemsetAsync(pl->d_partials, 0, sizeof(double2) * pl->n_items, st);
    if (!e) e = (int)cudaMemsetAsync(pl->d_counter, 0, sizeof(unsigned long long), st);
    if (e) return bt_cuda_fail(e, "memset");
    bt_exact_args a;
    memset(&a, 0, sizeof(a));
    a.opts = pl->d_opts;
    a.jobs = pl->d_jobs;
    a.prm = pl->d_prm;
    a.n_jobs = nj;
    a.shard = shard;
    a.n_shards = n_shards;
    a.n_run_items = pl->n_items > shard ? (pl->n_items - shard + n_shards - 1) / n_shards : 0;
    a.suf32 = pl->d_suf32;
    a.suf64 = pl->d_suf64;
    a.ph = pl->d_ph;
    a.pm = pl->d_pm;
    a.pw = pl->d_pw;
    a.partials = pl->d_partials;
    a.counter = pl->d_counter;
    if (!pl->ev0) {
        if (cudaEventCreate(&pl->ev0) != cudaSuccess || cudaEventCreate(&pl->ev1) != cudaSuccess)
            return bt_cuda_fail((int)cudaGetLastError(), "cudaEventCreate");
    }
    cudaEventRecord(pl->ev0, st);
    e = bt_launch_exact(&a, pl->prec, pl->prec == BT_PREC_FP64 ? c->grid64 : c->grid32, st);
    if (e) return bt_cuda_fail(e, "path-sum kernel");
    cudaEventRecord(pl->ev1, st);
    pl->timed = true;
    e = bt_launch_finalize(pl->d_jobs, pl->d_prm, nj, pl->d_partials, shard, n_shards, pl->prec, pl->d_out, st);
    if (e) return bt_cuda_fail(e, "finalize kernel");
    return BT_OK;
}

extern "C" bt_status bt_exact_plan_run(bt_exact_plan *pl, void *stream) {
    if (!pl) return bt_fail(BT_EINVAL, "bt_exact_plan_run: NULL plan");
    return plan_enqueue(pl, 0, 1, stream);
}

extern "C" bt_status bt_exact_plan_run_shard(bt_exact_plan *pl, int32_t shard, int32_t n_shards, void *stream) {
    if (!pl || n_shards < 1 || shard < 0 || shard >= n_shards)
        return bt_fail(BT_EINVAL, "bt_exact_plan_run_shard: bad shard %d of %d", shard, n_shards);
    return plan_enqueue(pl, shard, n_shards, stream);
}

extern "C" bt_status bt_exact_plan_read(bt_exact_plan *pl, bt_result *out, void *stream) {
    if (!pl || !out) return bt_fail(BT_EINVAL, "bt_exact_plan_read: NULL argument");
    cudaSetDevice(pl->ctx->device);
    cudaStream_t st = ctx_stream(pl->ctx, stream);
    cudaError_t e = cudaMemcpyAsync(out, pl->d_out, sizeof(bt_result) * pl->n_opts, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bt_cuda_fail(e, "bt_exact_plan_read");
    return BT_OK;
}

extern "C" bt_status bt_exact_plan_partials(bt_exact_plan *pl, double *partials, int32_t *item_job,
                                            int64_t *item_first_prefix, void *stream) {
    if (!pl || !partials) return bt_fail(BT_EINVAL, "bt_exact_plan_partials: NULL argument");
    cudaSetDevice(pl->ctx->device);
    cudaStream_t st = ctx_stream(pl->ctx, stream);
    cudaError_t e = cudaMemcpyAsync(partials, pl->d_partials, sizeof(double2) * pl->n_items, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bt_cuda_fail(e, "bt_exact_plan_partials");
    for (size_t j = 0; j < pl->jobs.size(); ++j) {
        const bt_job &J = pl->jobs[j];
        for (int i = 0; i < J.n_items; ++i) {
            if (item_job) item_job[J.item_begin + i] = (int32_t)j;
            if (item_first_prefix) item_first_prefix[J.item_begin + i] = (int64_t)i << BT_LOW_BITS;
        }
    }
    return BT_OK;
}

extern "C" bt_status bt_exact_plan_job(const bt_exact_plan *pl, int32_t j, int32_t *opt_call, int32_t *opt_put,
                                       int32_t *P, int32_t *L, int32_t *ppi) {
    if (!pl || j < 0 || j >= (int)pl->jobs.size()) return bt_fail(BT_EINVAL, "bt_exact_plan_job: bad job %d", j);
    const bt_job &J = pl->jobs[j];
    if (opt_call) *opt_call = J.out_call;
    if (opt_put) *opt_put = J.out_put;
    if (P) *P = J.P;
    if (L) *L = J.L;
    if (ppi) *ppi = 1 << BT_LOW_BITS;
    return BT_OK;
}

extern "C" bt_status bt_exact_split(const bt_option *opt, bt_precision prec, int32_t *P, int32_t *L, int32_t *ppi,
                                    int64_t *n_items) {
    if (!opt) return bt_fail(BT_EINVAL, "bt_exact_split: NULL option");
    if (prec != BT_PREC_FP64 && prec != BT_PREC_FP32_COMP) return bt_fail(BT_EINVAL, "bad precision %d", (int)prec);
    bt_status s = validate_option(opt, 0, BT_MAX_N_EXACT);
    if (s != BT_OK) return s;
    int field, mode;
    payoff_field(opt->payoff, &field, &mode);
    bt_job J;
    memset(&J, 0, sizeof(J));
    fill_job_shape(J, opt->N, field, mode, prec, tree_skewed(*opt));
    if (P) *P = J.P;
    if (L) *L = J.L;
    if (ppi) *ppi = 1 << BT_LOW_BITS;
    if (n_items) *n_items = J.n_items;
    return BT_OK;
}

extern "C" bt_status bt_exact_plan_info_get(const bt_exact_plan *pl, bt_exact_plan_info *info) {
    if (!pl || !info) return bt_fail(BT_EINVAL, "bt_exact_plan_info_get: NULL argument");
    info->n_options = pl->n_opts;
    info->n_jobs = (int32_t)pl->jobs.size();
    info->n_items = pl->n_items;
    info->payoff_paths = pl->payoff_paths;
    info->path_evaluations = pl->path_evals;
    info->device_bytes = pl->arena_bytes;
    info->h2d_bytes = sizeof(bt_option) * (size_t)pl->n_opts + sizeof(bt_job) * pl->jobs.size();
    info->d2h_bytes = sizeof(bt_result) * (size_t)pl->n_opts;
    return BT_OK;
}

extern "C" bt_status bt_exact_plan_kernel_ms(bt_exact_plan *pl, float *ms) {
    if (!pl || !ms || !pl->timed) return bt_fail(BT_EINVAL, "bt_exact_plan_kernel_ms: no timed run");
    cudaSetDevice(pl->ctx->device);
    cudaError_t e = cudaEventSynchronize(pl->ev1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, pl->ev0, pl->ev1);
    if (e != cudaSuccess) return bt_cuda_fail(e, "bt_exact_plan_kernel_ms");
    return BT_OK;
}

extern "C" void bt_exact_plan_destroy(bt_exact_plan *pl) {
    if (!pl) return;
    cudaSetDevice(pl->ctx->device);
    if (pl->arena && !pl->cached) {
        cudaStreamSynchronize(pl->ctx->stream);
        ctx_free(pl->ctx, pl->arena, pl->arena_bytes);
    }
    if (pl->ev0) cudaEventDestroy(pl->ev0);
    if (pl->ev1) cudaEventDestroy(pl->ev1);
    delete pl;
}

extern "C" bt_status bt_price_exact(bt_ctx *ctx, const bt_option *opts, int32_t n, bt_precision prec,
                                    bt_result *out, void *stream) {
    if (!ctx || !opts || !out || n < 1) return bt_fail(BT_EINVAL, "bt_price_exact: bad arguments");
    std::lock_guard<std::mutex> lock(ctx->cache_mu);
    bt_exact_plan *pl = nullptr;
    bt_status s = plan_create(ctx, opts, n, prec, true, &pl);
    if (s != BT_OK) return s;
    s = bt_exact_plan_run(pl, stream);
    if (s == BT_OK) s = bt_exact_plan_read(pl, out, stream);
    bt_exact_plan_destroy(pl);
    return s;
}
