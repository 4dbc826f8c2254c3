// Host runtime of the Monte Carlo entry points (Section 4).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "host_common.h"
#include "mc_internal.h"

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Payoff -> (suffix quantity, sign) of the affine form shared with the exhaustive kernels.
static void mc_payoff(int payoff, int *field, int *sign) {
    switch (payoff) {
    case BT_EURO_CALL: *field = BT_F_EURO; *sign = 1; break;
    case BT_EURO_PUT: *field = BT_F_EURO; *sign = -1; break;
    case BT_ASIAN_ARITH_CALL: *field = BT_F_ARITH; *sign = 1; break;
    case BT_ASIAN_ARITH_PUT: *field = BT_F_ARITH; *sign = -1; break;
    case BT_ASIAN_GEO_CALL: *field = BT_F_GEO; *sign = 1; break;
    case BT_ASIAN_GEO_PUT: *field = BT_F_GEO; *sign = -1; break;
    case BT_LOOKBACK_FIXED_CALL: *field = BT_F_LOOKMAX; *sign = 1; break;
    default: *field = BT_F_LOOKMIN; *sign = -1; break;
    }
}

// The largest suffix quantity f a call can draw over L steps (the path that only goes up):
// arithmetic sum_j u^j, geometric u^(L(L+1)/(2N)), European and lookback u^L; 0 for a put,
// whose clamp only needs -f <= 0.
static double suffix_f_bound(int field, int sign, int L, int N, double u) {
    if (sign < 0 || L == 0) return 0.0;
    switch (field) {
    case BT_F_ARITH: {
        double f = 0.0, r = 1.0;
        for (int j = 1; j <= L; ++j) f += (r *= u);
        return f;
    }
    case BT_F_GEO: return std::pow(u, (double)L * (double)(L + 1) / (2.0 * (double)N));
    default: return std::pow(u, (double)L);
    }
}

// round(p 2^32) clamped to [1, 2^32 - 1]: the word comparison draws x_t = 1
// with probability thr / 2^32.
static uint32_t bernoulli_threshold(double p) {
    double x = std::floor(p * 4294967296.0 + 0.5);
    if (x < 1.0) x = 1.0;
    if (x > 4294967295.0) x = 4294967295.0;
    return (uint32_t)x;
}

static bt_status mc_run(bt_ctx *ctx, const bt_option *opts, int32_t n, int32_t strata_bits,
                        int64_t samples_per_stratum, uint64_t seed, int32_t kind, int32_t shard, int32_t n_shards,
                        bt_result *out, double *strata_stats, void *stream) {
    if (!ctx || !opts || !out || n < 1) return bt_fail(BT_EINVAL, "bt_price_mc: bad arguments");
    if (kind != BT_MC_PARTITIONED && kind != BT_MC_SHARED) return bt_fail(BT_EINVAL, "bt_price_mc: bad kind %d", kind);
    if (samples_per_stratum < 1 || samples_per_stratum > ((int64_t)1 << 32))
        return bt_fail(BT_EINVAL, "bt_price_mc: samples_per_stratum %lld outside 1..2^32", (long long)samples_per_stratum);
    const int maxbits = kind == BT_MC_SHARED ? BT_MC_SHARED_MAX_BITS : BT_MC_MAX_BITS;
    std::vector<bt_mc_job> jobs((size_t)n);
    int64_t items = 0, strata_total = 0;
    for (int i = 0; i < n; ++i) {
        bt_status s = validate_option(&opts[i], i, BT_MC_MAX_N);
        if (s != BT_OK) return s;
        if (strata_bits < 0 || strata_bits > opts[i].N || strata_bits > maxbits)
            return bt_fail(strata_bits > maxbits ? BT_EUNSUPPORTED : BT_EINVAL,
                           "option %d: strata_bits %d outside 0..min(N=%d, %d)", i, strata_bits, opts[i].N, maxbits);
        if (n_shards > (1 << strata_bits))
            return bt_fail(BT_EINVAL, "%d shards of %d strata", n_shards, 1 << strata_bits);
        bt_mc_job &J = jobs[i];
        memset(&J, 0, sizeof(J));
        host_tree(&opts[i], &J.u, &J.d, &J.p);
        J.N = opts[i].N;
        J.mb = strata_bits;
        J.R = samples_per_stratum;
        mc_payoff(opts[i].payoff, &J.field, &J.sign);
        J.shared = kind == BT_MC_SHARED;
        J.stream = (uint32_t)i;
        J.key_lo = (uint32_t)(seed & 0xffffffffu);
        J.key_hi = (uint32_t)(seed >> 32);
        J.thr = bernoulli_threshold(J.p);
        J.out = i;
        J.S0 = opts[i].S0;
        J.K = opts[i].K;
        J.disc = std::exp(-opts[i].rate * opts[i].T);
        J.uf = (float)J.u;
        J.df = (float)J.d;
        J.lnu_f = (float)std::log(J.u);
        for (int k = 0; k <= J.mb; ++k) J.prob_k[k] = std::pow(J.p, (double)k) * std::pow(1.0 - J.p, (double)(J.mb - k));
        J.fbound = suffix_f_bound(J.field, J.sign, J.N - J.mb, J.N, J.u);
        const int64_t chunks = (J.R + BT_MC_ITEM - 1) / BT_MC_ITEM;
        J.shard = shard;
        J.n_shards = n_shards;
        const int64_t M = J.shared ? 1 : (((int64_t)1 << J.mb) - shard + n_shards - 1) / n_shards;
        J.M = M;
        J.item_begin = items;
        J.n_items = M * chunks;
        J.strata_off = strata_total;
        items += J.n_items;
        strata_total += M;
    }
    if (items > ((int64_t)1 << 31)) return bt_fail(BT_EUNSUPPORTED, "bt_price_mc: %lld work items", (long long)items);
    size_t off = 0;
    const size_t o_jobs = off; off = up256(off + sizeof(bt_mc_job) * n);
    const size_t o_stats = off; off = up256(off + sizeof(double4) * items);
    const size_t o_out = off; off = up256(off + sizeof(bt_result) * n);
    const size_t o_str = off; off = up256(off + (strata_stats ? sizeof(double) * 3 * strata_total : 0));
    const size_t o_nmq = off; off = up256(off + sizeof(double4) * strata_total);
    const size_t o_part = off; off = up256(off + sizeof(double) * 8 * BT_MC_FIN_BLOCKS * n);
    const size_t o_cnt = off; off = up256(off + sizeof(unsigned long long));
    const bool sh = kind == BT_MC_SHARED;
    const size_t o_tab = off; off = up256(off + (sh ? sizeof(float4) * BT_MC_TAB_ENTRIES * n : 0));
    const size_t o_pc = off; off = up256(off + (sh ? sizeof(double) * BT_MC_TAB_BLOCKS * n : 0));
    cudaSetDevice(ctx->device);
    // the context's reusable scratch (no allocation per call once it is large enough)
    std::lock_guard<std::mutex> lock(ctx->cache_mu);
    void *arena = nullptr;
    bt_status s = ctx_scratch(ctx, off, &arena);
    if (s != BT_OK) return s;
    char *b = (char *)arena;
    bt_mc_job *d_jobs = (bt_mc_job *)(b + o_jobs);
    double4 *d_stats = (double4 *)(b + o_stats);
    bt_result *d_out = (bt_result *)(b + o_out);
    double *d_str = strata_stats ? (double *)(b + o_str) : nullptr;
    double4 *d_nmq = (double4 *)(b + o_nmq);
    double *d_part = (double *)(b + o_part);
    unsigned long long *d_cnt = (unsigned long long *)(b + o_cnt);
    cudaStream_t st = ctx_stream(ctx, stream);
    bt_status rs = BT_OK;
    cudaError_t e = cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(bt_mc_job) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) rs = bt_cuda_fail(e, "bt_price_mc: upload");
    if (rs == BT_OK) {
        bt_mc_args a;
        memset(&a, 0, sizeof(a));
        a.jobs = d_jobs;
        a.n_jobs = n;
        a.n_items = items;
        a.item_stats = d_stats;
        a.counter = d_cnt;
        a.key_lo = (uint32_t)(seed & 0xffffffffu);
        a.key_hi = (uint32_t)(seed >> 32);
        a.shared_tab = sh ? (float4 *)(b + o_tab) : nullptr;
        a.shared_pc = sh ? (double *)(b + o_pc) : nullptr;
        int le = bt_launch_mc(&a, kind == BT_MC_SHARED, bt_mc_grid_size(ctx->device, kind == BT_MC_SHARED), st);
        if (le) rs = bt_cuda_fail(le, "MC kernel");
    }
    if (rs == BT_OK) {
        const int64_t chunks = (samples_per_stratum + BT_MC_ITEM - 1) / BT_MC_ITEM;
        int le = bt_launch_mc_finalize(d_jobs, n, chunks, d_stats, strata_total, d_nmq, d_part, d_out, d_str, st);
        if (le) rs = bt_cuda_fail(le, "MC finalize kernel");
    }
    if (rs == BT_OK) {
        e = cudaMemcpyAsync(out, d_out, sizeof(bt_result) * n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && strata_stats)
            e = cudaMemcpyAsync(strata_stats, d_str, sizeof(double) * 3 * strata_total, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rs = bt_cuda_fail(e, "bt_price_mc: results");
    }
    cudaStreamSynchronize(st);   // the scratch is free for the next call only after this one's work
    return rs;
}

extern "C" bt_status bt_price_mc_ex(bt_ctx *ctx, const bt_option *opts, int32_t n, int32_t strata_bits,
                                    int64_t samples_per_stratum, uint64_t seed, int32_t kind, bt_result *out,
                                    double *strata_stats, void *stream) {
    return mc_run(ctx, opts, n, strata_bits, samples_per_stratum, seed, kind, 0, 1, out, strata_stats, stream);
}

extern "C" bt_status bt_price_mc_shard(bt_ctx *ctx, const bt_option *opts, int32_t n, int32_t strata_bits,
                                       int64_t samples_per_stratum, uint64_t seed, int32_t shard, int32_t n_shards,
                                       bt_result *out, double *strata_stats, void *stream) {
    if (n_shards < 1 || shard < 0 || shard >= n_shards)
        return bt_fail(BT_EINVAL, "bt_price_mc_shard: shard %d of %d", shard, n_shards);
    return mc_run(ctx, opts, n, strata_bits, samples_per_stratum, seed, BT_MC_PARTITIONED, shard, n_shards, out,
                  strata_stats, stream);
}

extern "C" bt_status bt_price_mc(bt_ctx *ctx, const bt_option *opts, int32_t n, int32_t strata_bits,
                                 int64_t samples_per_stratum, uint64_t seed, bt_result *out, void *stream) {
    return bt_price_mc_ex(ctx, opts, n, strata_bits, samples_per_stratum, seed, BT_MC_PARTITIONED, out, nullptr,
                          stream);
}

extern "C" bt_status bt_philox4x32_10(bt_ctx *ctx, const uint32_t *ctr, const uint32_t *key, uint32_t *out,
                                      int32_t n) {
    if (!ctx || !ctr || !key || !out || n < 1) return bt_fail(BT_EINVAL, "bt_philox4x32_10: bad arguments");
    cudaSetDevice(ctx->device);
    size_t off = 0;
    const size_t o_c = off; off = up256(off + 16 * (size_t)n);
    const size_t o_k = off; off = up256(off + 8 * (size_t)n);
    const size_t o_o = off; off = up256(off + 16 * (size_t)n);
    void *arena = nullptr;
    bt_status s = ctx_alloc(ctx, off, &arena);
    if (s != BT_OK) return s;
    char *b = (char *)arena;
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaMemcpyAsync(b + o_c, ctr, 16 * (size_t)n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_k, key, 8 * (size_t)n, cudaMemcpyHostToDevice, st);
    int le = e == cudaSuccess ? bt_launch_philox_selftest((const uint4 *)(b + o_c), (const uint2 *)(b + o_k),
                                                          (uint4 *)(b + o_o), n, st)
                              : (int)e;
    if (le == 0) e = cudaMemcpyAsync(out, b + o_o, 16 * (size_t)n, cudaMemcpyDeviceToHost, st);
    if (le == 0 && e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaStreamSynchronize(st);
    ctx_free(ctx, arena, off);
    if (le) return bt_cuda_fail(le, "philox kernel");
    if (e != cudaSuccess) return bt_cuda_fail(e, "bt_philox4x32_10");
    return BT_OK;
}
