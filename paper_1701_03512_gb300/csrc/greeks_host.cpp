// Host runtime of the Greeks pass: plan, launches, and the chain rule from the
// kernel's sums (value, sum w pay k, dV/du at fixed p, in-the-money weight) to
// dV/dS0, dV/dsigma, dV/drate, dV/dK.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "host_common.h"

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// du/dsigma, du/drate, dp/du (through d = 1/u) and dp/drate of the tree (Section 2).
static void tree_partials(const bt_option &o, double u, double p, double *u_s, double *u_r, double *p_u,
                          double *p_r) {
    const double dt = o.T / (double)o.N;
    if (o.tree_kind == BT_TREE_EXPLICIT) {
        *u_s = *u_r = *p_u = *p_r = 0.0;
        return;
    }
    const double E = std::exp(o.rate * dt);
    if (o.tree_kind == BT_TREE_CRR) {
        *u_s = std::sqrt(dt) * u;
        *u_r = 0.0;
    } else {
        const double e1 = std::exp(-o.rate * dt), e2 = std::exp((o.rate + o.sigma * o.sigma) * dt);
        const double beta = 0.5 * (e1 + e2), sq = std::sqrt(beta * beta - 1.0);
        const double u_b = 1.0 + beta / sq;
        *u_s = u_b * o.sigma * dt * e2;
        *u_r = u_b * 0.5 * dt * (e2 - e1);
    }
    const double D = u - 1.0 / u, num = E - 1.0 / u;
    *p_u = ((1.0 / (u * u)) * D - num * (1.0 + 1.0 / (u * u))) / (D * D);
    *p_r = dt * E / D;
    (void)p;
}

extern "C" bt_status bt_greeks_exact(bt_ctx *ctx, const bt_option *opts, int32_t n, bt_precision prec,
                                     double *value, double *grad, void *stream) {
    if (!ctx || !opts || !value || !grad || n < 1) return bt_fail(BT_EINVAL, "bt_greeks_exact: bad arguments");
    if (prec != BT_PREC_FP32_COMP)
        return bt_fail(BT_EUNSUPPORTED, "bt_greeks_exact: only BT_PREC_FP32_COMP has a derivative pass");
    std::vector<bt_job> jobs((size_t)n);
    int64_t items = 0, suf = 0, ph = 0, pm = 0, pw = 0;
    int max_len = 0;
    for (int i = 0; i < n; ++i) {
        bt_status s = validate_option(&opts[i], i, BT_MAX_N_EXACT);
        if (s != BT_OK) return s;
        double u, d, p;
        host_tree(&opts[i], &u, &d, &p);
        if (p < 0.004 || 1.0 - p < 0.004)
            return bt_fail(BT_EUNSUPPORTED, "option %d: p = %.6g; FP32_COMP needs min(p,1-p) >= 0.004", i, p);
        bt_job &J = jobs[i];
        memset(&J, 0, sizeof(J));
        int step = 1;
        plan_one_job(opts + i, 1, 0, &J, &step, BT_PREC_FP32_COMP);  // one option per pass
        J.opt = i;
        J.out_call = J.out_call >= 0 ? i : -1;
        J.out_put = J.out_put >= 0 ? i : -1;
        J.item_begin = items;
        J.item_offset = 0;
        J.part_off = items;
        J.prm_off = i;
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
        int64_t len = (1ll << J.L) + J.suf_len + (1ll << J.H) + (1ll << J.M) + 2 * J.N + 3 + J.geo_len;
        if (len > max_len) max_len = (int)len;
    }
    size_t off = 0;
    const size_t o_opts = off; off = up256(off + sizeof(bt_option) * n);
    const size_t o_jobs = off; off = up256(off + sizeof(bt_job) * n);
    const size_t o_prm = off; off = up256(off + sizeof(bt_jparams) * n);
    const size_t o_suf = off; off = up256(off + sizeof(float2) * suf);
    const size_t o_sufd = off; off = up256(off + sizeof(float) * suf);
    const size_t o_ph = off; off = up256(off + sizeof(bt_pentry) * ph);
    const size_t o_pm = off; off = up256(off + sizeof(bt_pentry) * pm);
    const size_t o_pw = off; off = up256(off + sizeof(bt_pow) * pw);
    const size_t o_part = off; off = up256(off + sizeof(double4) * items);
    const size_t o_sum = off; off = up256(off + sizeof(double4) * n);
    const size_t o_cnt = off; off = up256(off + sizeof(unsigned long long));
    cudaSetDevice(ctx->device);
    // the context's reusable scratch (no allocation per call once it is large enough)
    std::lock_guard<std::mutex> lock(ctx->cache_mu);
    void *arena = nullptr;
    bt_status s = ctx_scratch(ctx, off, &arena);
    if (s != BT_OK) return s;
    char *b = (char *)arena;
    bt_option *d_opts = (bt_option *)(b + o_opts);
    bt_job *d_jobs = (bt_job *)(b + o_jobs);
    bt_jparams *d_prm = (bt_jparams *)(b + o_prm);
    float2 *d_suf = (float2 *)(b + o_suf);
    float *d_sufd = (float *)(b + o_sufd);
    bt_pentry *d_ph = (bt_pentry *)(b + o_ph);
    bt_pentry *d_pm = (bt_pentry *)(b + o_pm);
    bt_pow *d_pw = (bt_pow *)(b + o_pw);
    double4 *d_part = (double4 *)(b + o_part);
    double4 *d_sum = (double4 *)(b + o_sum);
    unsigned long long *d_cnt = (unsigned long long *)(b + o_cnt);
    cudaStream_t st = ctx_stream(ctx, stream);
    std::vector<double4> sums((size_t)n);
    bt_status rs = BT_OK;
    cudaError_t e = cudaMemcpyAsync(d_opts, opts, sizeof(bt_option) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(bt_job) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_part, 0, sizeof(double4) * items, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) rs = bt_cuda_fail(e, "bt_greeks_exact: upload");
    int le = 0;
    if (rs == BT_OK && (le = bt_launch_params(d_opts, d_jobs, d_prm, n, st))) rs = bt_cuda_fail(le, "params kernel");
    if (rs == BT_OK && (le = bt_launch_tables_d(d_jobs, d_prm, n, max_len, d_suf, d_sufd, d_ph, d_pm, d_pw, st)))
        rs = bt_cuda_fail(le, "tables kernel");
    if (rs == BT_OK) {
        bt_exact_args a;
        memset(&a, 0, sizeof(a));
        a.opts = d_opts;
        a.jobs = d_jobs;
        a.prm = d_prm;
        a.n_jobs = n;
        a.shard = 0;
        a.n_shards = 1;
        a.n_run_items = items;
        a.suf32 = d_suf;
        a.sufd = d_sufd;
        a.ph = d_ph;
        a.pm = d_pm;
        a.pw = d_pw;
        a.partials4 = d_part;
        a.counter = d_cnt;
        if ((le = bt_launch_greeks(&a, ctx->grid32, st))) rs = bt_cuda_fail(le, "derivative kernel");
    }
    if (rs == BT_OK && (le = bt_launch_greeks_finalize(d_jobs, n, d_part, d_sum, st)))
        rs = bt_cuda_fail(le, "derivative finalize kernel");
    if (rs == BT_OK) {
        e = cudaMemcpyAsync(sums.data(), d_sum, sizeof(double4) * n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rs = bt_cuda_fail(e, "bt_greeks_exact: results");
    }
    cudaStreamSynchronize(st);   // the scratch is free for the next call only after this one's work
    if (rs != BT_OK) return rs;
    for (int i = 0; i < n; ++i) {
        const bt_option &o = opts[i];
        double u, d, p;
        host_tree(&o, &u, &d, &p);
        const double sgn = jobs[i].mode == BT_MODE_CALL ? 1.0 : -1.0;
        const double disc = std::exp(-o.rate * o.T);
        const double Vs = sums[i].x, Ks = sums[i].y, Ds = sums[i].z, Ps = sums[i].w;
        const double V = disc * Vs;
        const double dK = -sgn * disc * Ps;
        const double dVdu = disc * Ds;
        const double dVdp = disc / (p * (1.0 - p)) * (Ks - (double)o.N * p * Vs);
        double u_s, u_r, p_u, p_r;
        tree_partials(o, u, p, &u_s, &u_r, &p_u, &p_r);
        value[i] = V;
        grad[4 * i + 0] = (V - o.K * dK) / o.S0;                         // Euler: S0 dV/dS0 + K dV/dK = V
        grad[4 * i + 1] = (dVdu + dVdp * p_u) * u_s;                     // dV/dsigma
        grad[4 * i + 2] = (dVdu + dVdp * p_u) * u_r + dVdp * p_r - o.T * V;  // dV/drate
        grad[4 * i + 3] = dK;                                             // dV/dK
    }
    return BT_OK;
}
