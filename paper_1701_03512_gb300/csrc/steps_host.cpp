// Host runtime of the move-by-move passes: time-varying binomial trees
// (eq. f13 with per-step u_t, d_t, p_t) and trees with b branches per node
// (the end of Section 3). Validation, plan, one allocation, launches, results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "host_common.h"

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

static bt_status validate_scalars(const bt_option &o, int idx) {
    if (o.N < 1 || o.N > BT_MAX_N_EXACT) return bt_fail(BT_EINVAL, "option %d: N=%d outside 1..%d", idx, o.N, BT_MAX_N_EXACT);
    if (o.payoff < 0 || o.payoff > 7) return bt_fail(BT_EINVAL, "option %d: bad payoff %d", idx, o.payoff);
    if (!(std::isfinite(o.S0) && std::isfinite(o.K) && std::isfinite(o.rate) && std::isfinite(o.T)))
        return bt_fail(BT_EINVAL, "option %d: non-finite input", idx);
    if (!(o.S0 > 0.0)) return bt_fail(BT_EINVAL, "option %d: S0 must be > 0", idx);
    if (!(o.K >= 0.0)) return bt_fail(BT_EINVAL, "option %d: K must be >= 0", idx);
    if (!(o.T > 0.0)) return bt_fail(BT_EINVAL, "option %d: T must be > 0", idx);
    return BT_OK;
}

// One option's moves (2b doubles per step): factors > 0, probabilities in
// [0,1] summing to 1; FP32_COMP keeps every positive probability >= 0.004.
static bt_status validate_moves(const double *mv, int N, int b, int idx, int prec) {
    for (int t = 0; t < N; ++t) {
        const double *m = mv + 2 * b * t;
        double psum = 0.0;
        for (int k = 0; k < b; ++k) {
            if (!(std::isfinite(m[k]) && m[k] > 0.0 && m[b + k] >= 0.0 && m[b + k] <= 1.0))
                return bt_fail(BT_EINVAL, "option %d step %d: factors must be > 0, probabilities in [0,1]", idx, t + 1);
            if (prec == BT_PREC_FP32_COMP && m[b + k] > 0.0 && m[b + k] < 0.004)
                return bt_fail(BT_EUNSUPPORTED, "option %d step %d: probability %.6g; FP32_COMP needs >= 0.004", idx,
                               t + 1, m[b + k]);
            psum += m[b + k];
        }
        if (std::fabs(psum - 1.0) > 1e-12)
            return bt_fail(BT_EINVAL, "option %d step %d: probabilities sum to %.17g", idx, t + 1, psum);
    }
    return BT_OK;
}

// Suffix steps of a move-by-move job: b^L <= 2^13 entries in shared memory for the FP32 pass
// (2^12 for FP64), leaving at least 2^15 prefixes where the tree has them (binomial: the lattice
// split).
static int moves_split_L(int N, int b, bt_precision prec) {
    const int max_l = prec == BT_PREC_FP64 ? BT_STEPS_MAX_L : BT_STEPS32_MAX_L;
    int L = 0;
    int64_t nsuf = 1;
    while (L < N && nsuf * b <= (1 << max_l) &&
           (L == 0 || (b == 2 ? L < exact_split_L(N)
                              : std::pow((double)b, (double)(N - L - 1)) >=
                                    (double)(1 << (BT_LOW_BITS + BT_MIN_ITEM_BITS))))) {
        nsuf *= b;
        ++L;
    }
    return L;
}

// Two options form one pass when they price the same tree with the same
// strike (their payoffs are then checked to be a call/put pair of one field).
static bool same_moves_job(const bt_option &a, const bt_option &c, const double *ma, const double *mc, int b) {
    if (!(a.N == c.N && a.S0 == c.S0 && a.K == c.K && a.rate == c.rate && a.T == c.T)) return false;
    return memcmp(ma, mc, sizeof(double) * 2 * (size_t)b * (size_t)a.N) == 0;
}

static bt_status price_moves(bt_ctx *ctx, const bt_option *opts, int32_t n, int b, const double *moves,
                             bt_precision prec, bt_result *out, void *stream) {
    if (prec != BT_PREC_FP64 && prec != BT_PREC_FP32_COMP) return bt_fail(BT_EINVAL, "bad precision %d", (int)prec);
    std::vector<int64_t> first((size_t)n + 1, 0);   // first step of each option in the move array
    for (int i = 0; i < n; ++i) {
        bt_status s = validate_scalars(opts[i], i);
        if (s != BT_OK) return s;
        if ((double)opts[i].N * std::log2((double)b) > 42.0 + 1e-9)
            return bt_fail(BT_EUNSUPPORTED, "option %d: %d^%d paths exceed 2^42", i, b, opts[i].N);
        if ((s = validate_moves(moves + 2 * b * first[i], opts[i].N, b, i, prec)) != BT_OK) return s;
        first[i + 1] = first[i] + opts[i].N;
    }
    std::vector<bt_job> jobs;
    jobs.reserve((size_t)n);
    int64_t items = 0, suf = 0, tab = 0;
    int max_len = 0;
    for (int i = 0; i < n;) {
        jobs.emplace_back();
        bt_job &J = jobs.back();
        memset(&J, 0, sizeof(J));
        int field, mode;
        payoff_field(opts[i].payoff, &field, &mode);
        J.opt = i;
        J.out_call = mode == BT_MODE_CALL ? i : -1;
        J.out_put = mode == BT_MODE_PUT ? i : -1;
        int step = 1;
        // a call immediately followed by the put of the same tree and strike
        // (or the reverse) is one pass: the affine form is shared
        if (i + 1 < n && same_moves_job(opts[i], opts[i + 1], moves + 2 * b * first[i], moves + 2 * b * first[i + 1],
                                        b)) {
            int f2, m2;
            payoff_field(opts[i + 1].payoff, &f2, &m2);
            if (f2 == field && m2 != mode) {
                mode = BT_MODE_BOTH;
                if (J.out_call < 0) J.out_call = i + 1;
                else J.out_put = i + 1;
                step = 2;
            }
        }
        J.N = opts[i].N;
        J.branches = b;
        const int L = moves_split_L(J.N, b, prec);
        int64_t nsuf = 1;
        for (int t = 0; t < L; ++t) nsuf *= b;
        J.L = L;
        J.P = J.N - L;
        J.M = (J.P + 1) / 2;
        J.H = J.P - J.M;
        int64_t nmid = 1, npre = 1;
        for (int t = 0; t < J.M; ++t) nmid *= b;
        for (int t = 0; t < J.P; ++t) npre *= b;
        J.n_suffix = nsuf;
        J.n_mid = nmid;
        J.n_prefix = npre;
        J.field = field;
        J.mode = mode;
        J.suf_len = (int32_t)((nsuf + BT_UNROLL - 1) / BT_UNROLL * BT_UNROLL);   // entries; padding has weight 0
        for (int k = 0; k < BT_MAX_L + 2; ++k) J.goff[k] = k == 0 ? 0 : J.suf_len;
        J.n_items = (int32_t)std::max<int64_t>(1, (npre + (1 << BT_LOW_BITS) - 1) >> BT_LOW_BITS);
        J.item_begin = items;
        J.item_offset = 0;
        J.part_off = items;
        J.prm_off = (int64_t)jobs.size() - 1;
        J.off_suf = suf;
        J.off_ph = tab;
        J.off_pm = tab + npre / nmid;
        J.off_pow = first[i];   // first step of this job in the move array
        items += J.n_items;
        suf += J.suf_len;
        tab += npre / nmid + nmid;
        max_len = std::max(max_len, (int)(J.suf_len + npre / nmid + nmid));
        i += step;
    }
    const int nj = (int)jobs.size();
    const int64_t nsteps = first[n];
    if (items > ((int64_t)1 << 31)) return bt_fail(BT_EUNSUPPORTED, "%lld work items", (long long)items);
    size_t off = 0;
    const size_t o_opts = off; off = up256(off + sizeof(bt_option) * n);
    const size_t o_jobs = off; off = up256(off + sizeof(bt_job) * nj);
    const size_t o_prm = off; off = up256(off + sizeof(bt_jparams) * nj);
    const size_t o_steps = off; off = up256(off + sizeof(double) * 2 * b * nsteps);
    const size_t o_suf = off; off = up256(off + 16 * (size_t)suf);   // float4 or double2 entries
    const size_t o_tab = off; off = up256(off + sizeof(bt_spentry) * tab);
    const size_t o_part = off; off = up256(off + sizeof(double2) * items);
    const size_t o_out = off; off = up256(off + sizeof(bt_result) * n);
    const size_t o_cnt = off; off = up256(off + sizeof(unsigned long long));
    cudaSetDevice(ctx->device);
    // the context's reusable scratch (no allocation per call once it is large enough)
    std::lock_guard<std::mutex> lock(ctx->cache_mu);
    void *arena = nullptr;
    bt_status rs = ctx_scratch(ctx, off, &arena);
    if (rs != BT_OK) return rs;
    char *base = (char *)arena;
    bt_option *d_opts = (bt_option *)(base + o_opts);
    bt_job *d_jobs = (bt_job *)(base + o_jobs);
    bt_jparams *d_prm = (bt_jparams *)(base + o_prm);
    double *d_steps = (double *)(base + o_steps);
    bt_spentry *d_tab = (bt_spentry *)(base + o_tab);
    double2 *d_part = (double2 *)(base + o_part);
    bt_result *d_out = (bt_result *)(base + o_out);
    unsigned long long *d_cnt = (unsigned long long *)(base + o_cnt);
    cudaStream_t st = ctx_stream(ctx, stream);
    cudaError_t e = cudaMemcpyAsync(d_opts, opts, sizeof(bt_option) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(bt_job) * nj, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_steps, moves, sizeof(double) * 2 * b * nsteps, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_part, 0, sizeof(double2) * items, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) rs = bt_cuda_fail(e, "move-by-move pass: upload");
    int le = 0;
    if (rs == BT_OK && (le = bt_launch_steps_params(d_opts, d_jobs, d_steps, d_prm, nj, st)))
        rs = bt_cuda_fail(le, "params kernel");
    if (rs == BT_OK && (le = bt_launch_steps_tables(d_jobs, d_prm, d_steps, nj, max_len, prec, (float4 *)(base + o_suf),
                                                    (double2 *)(base + o_suf), d_tab, st)))
        rs = bt_cuda_fail(le, "tables kernel");
    if (rs == BT_OK) {
        bt_exact_args a;
        memset(&a, 0, sizeof(a));
        a.opts = d_opts;
        a.jobs = d_jobs;
        a.prm = d_prm;
        a.n_jobs = nj;
        a.shard = 0;
        a.n_shards = 1;
        a.n_run_items = items;
        a.suf32 = (const float2 *)(base + o_suf);
        a.suf64 = (const double *)(base + o_suf);
        a.partials = d_part;
        a.counter = d_cnt;
        if ((le = bt_launch_steps(&a, d_tab, prec, ctx->device, st))) rs = bt_cuda_fail(le, "path-sum kernel");
    }
    if (rs == BT_OK && (le = bt_launch_finalize(d_jobs, d_prm, nj, d_part, 0, 1, prec, d_out, st)))
        rs = bt_cuda_fail(le, "finalize kernel");
    if (rs == BT_OK) {
        e = cudaMemcpyAsync(out, d_out, sizeof(bt_result) * n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rs = bt_cuda_fail(e, "move-by-move pass: results");
    }
    cudaStreamSynchronize(st);   // the scratch is free for the next call only after this one's work
    if (rs == BT_OK)
        for (int i = 0; i < n; ++i) {  // b^N paths (finalize wrote 2^N)
            long long paths = 1;
            for (int t = 0; t < opts[i].N; ++t) paths *= b;
            out[i].paths = paths;
        }
    return rs;
}

// Whether the suffix values f_s of a European, geometric or lookback job
// repeat: under one prefix, equal f_s give equal FP32 payoffs, so their
// roundings add up instead of averaging out. The b^L values (the job's own
// split) are computed in FP64, sorted, and counted as distinct where
// neighbours differ by more than 1e-12 relative; more than eight suffixes
// per distinct value on average counts as repeating. A recombining tree (the
// same moves at every step) repeats end prices, level sums and extremes
// hundreds of times (14 end prices for 8192 binomial suffixes); a lookback on
// a tree that does not recombine repeats its running extreme a few times
// (over the continuations that stay inside it: 2 to 4 suffixes per value on
// the trees tested), which the FP32 pass keeps.
static bool suffix_values_repeat(const bt_option &o, int b, const double *mv) {
    int field, mode;
    payoff_field(o.payoff, &field, &mode);
    if (field == BT_F_ARITH) return false;
    const int N = o.N, L = moves_split_L(N, b, BT_PREC_FP32_COMP), P = N - L;   // the FP32 pass's split
    int64_t nsuf = 1;
    for (int t = 0; t < L; ++t) nsuf *= b;
    std::vector<double> f((size_t)nsuf);
    std::vector<int> x((size_t)L);
    for (int64_t s = 0; s < nsuf; ++s) {
        int64_t v = s;
        for (int t = L - 1; t >= 0; --t, v /= b) x[t] = (int)(v % b);   // first suffix step most significant
        double rel = 1.0, mx = 0.0, mn = 1e300, lg = 0.0;
        for (int t = 0; t < L; ++t) {
            rel *= mv[2 * b * (P + t) + x[t]];
            mx = std::max(mx, rel);
            mn = std::min(mn, rel);
            lg += std::log(rel);
        }
        f[s] = field == BT_F_EURO ? rel : field == BT_F_LOOKMAX ? mx : field == BT_F_LOOKMIN ? mn
                                                                                          : std::exp(lg / N);
    }
    std::sort(f.begin(), f.end());
    int64_t distinct = 1;
    for (int64_t i = 1; i < nsuf; ++i)
        if (f[i] - f[i - 1] > 1e-12 * std::max(std::fabs(f[i]), std::fabs(f[i - 1]))) ++distinct;
    return nsuf > 8 * distinct;
}

// FP32_COMP rounds every path once in its FP32 pass (a tree given move by
// move has no classes). Those roundings average under 1e-9 only over 2^28
// paths or more, over at least 2^BT_PER_PATH_MIN_NEFF_LOG2 effective paths
// (1 / sum_x p(x)^2 = prod_t 1 / sum_k q_tk^2: the independent steps' own
// collision probabilities multiply), and when the suffix values do not
// repeat; other options are priced by the FP64 pass (cheap for the small
// trees).
static bool fp32_pass_suffices(const bt_option &o, int b, const double *mv) {
    if ((double)o.N * std::log2((double)b) < 28.0 - 1e-9) return false;
    double neff_log2 = 0.0;
    for (int t = 0; t < o.N; ++t) {
        double c = 0.0;
        for (int k = 0; k < b; ++k) c += mv[2 * b * t + b + k] * mv[2 * b * t + b + k];
        neff_log2 -= std::log2(c);
    }
    if (neff_log2 < BT_PER_PATH_MIN_NEFF_LOG2) return false;
    return !suffix_values_repeat(o, b, mv);
}

static bt_status price_moves_routed(bt_ctx *ctx, const bt_option *opts, int32_t n, int b, const double *moves,
                                    bt_precision prec, bt_result *out, void *stream) {
    if (prec != BT_PREC_FP32_COMP) return price_moves(ctx, opts, n, b, moves, prec, out, stream);
    std::vector<int> grp[2];  // [0] FP64 (small trees), [1] FP32_COMP
    std::vector<int64_t> first(n);
    int64_t t = 0;
    for (int i = 0; i < n; ++i) {
        if (opts[i].N < 1 || opts[i].N > BT_MAX_N_EXACT)
            return bt_fail(BT_EINVAL, "option %d: N=%d outside 1..%d", i, opts[i].N, BT_MAX_N_EXACT);
        first[i] = t;
        t += opts[i].N;
    }
    std::vector<char> fp32(n, 0);
    for (int i = 0; i < n; ++i) {  // validation with the batch's own option indices
        bt_status s = validate_scalars(opts[i], i);
        if (s == BT_OK && (double)opts[i].N * std::log2((double)b) > 42.0 + 1e-9)
            s = bt_fail(BT_EUNSUPPORTED, "option %d: %d^%d paths exceed 2^42", i, b, opts[i].N);
        if (s == BT_OK) s = validate_moves(moves + 2 * b * first[i], opts[i].N, b, i, BT_PREC_FP64);
        if (s != BT_OK) return s;
        fp32[i] = fp32_pass_suffices(opts[i], b, moves + 2 * b * first[i]);
        // the FP32 pass's probability floor (its weights stay in the FP32 pair range)
        if (fp32[i] && (s = validate_moves(moves + 2 * b * first[i], opts[i].N, b, i, prec)) != BT_OK) return s;
        grp[fp32[i] ? 1 : 0].push_back(i);
    }
    if (grp[0].empty()) return price_moves(ctx, opts, n, b, moves, prec, out, stream);
    if (grp[1].empty()) return price_moves(ctx, opts, n, b, moves, BT_PREC_FP64, out, stream);
    for (int g = 0; g < 2; ++g) {
        std::vector<bt_option> o;
        std::vector<double> mv;
        for (int i : grp[g]) {
            o.push_back(opts[i]);
            mv.insert(mv.end(), moves + 2 * b * first[i], moves + 2 * b * (first[i] + opts[i].N));
        }
        std::vector<bt_result> r(o.size());
        bt_status s = price_moves(ctx, o.data(), (int32_t)o.size(), b, mv.data(), g ? prec : BT_PREC_FP64, r.data(),
                                  stream);
        if (s != BT_OK) return s;
        for (size_t k = 0; k < r.size(); ++k) out[grp[g][k]] = r[k];
    }
    return BT_OK;
}

extern "C" bt_status bt_price_exact_moves(bt_ctx *ctx, const bt_option *opts, int32_t n, int32_t branches,
                                          const double *moves, bt_precision prec, bt_result *out, void *stream) {
    if (!ctx || !opts || !moves || !out || n < 1) return bt_fail(BT_EINVAL, "bt_price_exact_moves: bad arguments");
    if (branches < 2 || branches > 8) return bt_fail(BT_EINVAL, "branches = %d outside 2..8", branches);
    return price_moves_routed(ctx, opts, n, branches, moves, prec, out, stream);
}

extern "C" bt_status bt_price_exact_steps(bt_ctx *ctx, const bt_option *opts, int32_t n, const double *steps,
                                          bt_precision prec, bt_result *out, void *stream) {
    if (!ctx || !opts || !steps || !out || n < 1) return bt_fail(BT_EINVAL, "bt_price_exact_steps: bad arguments");
    // (u_t, d_t, p_t) -> binomial moves in digit order: factors (d, u), probabilities (1 - p, p)
    std::vector<double> mv;
    int64_t o = 0;
    for (int i = 0; i < n; ++i) {
        if (opts[i].N < 1 || opts[i].N > BT_MAX_N_EXACT)
            return bt_fail(BT_EINVAL, "option %d: N=%d outside 1..%d", i, opts[i].N, BT_MAX_N_EXACT);
        for (int t = 0; t < opts[i].N; ++t) {
            const double u = steps[3 * (o + t)], d = steps[3 * (o + t) + 1], p = steps[3 * (o + t) + 2];
            if (!(std::isfinite(u) && std::isfinite(d) && std::isfinite(p) && d > 0.0 && u > d && p > 0.0 && p < 1.0))
                return bt_fail(BT_EINVAL, "option %d step %d: needs 0 < d < u and 0 < p < 1", i, t + 1);
            mv.insert(mv.end(), {d, u, 1.0 - p, p});
        }
        o += opts[i].N;
    }
    return price_moves_routed(ctx, opts, n, 2, mv.data(), prec, out, stream);
}
