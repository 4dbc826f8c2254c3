/*
 * btree.h -- C ABI of libbtree, a GB300 (sm_103a) library for expected values
 * of path-dependent payoffs over the 2^N Bernoulli paths of a recombinant
 * binomial tree (Popuri, Raim, Neerchal, Gobbert, arXiv 1701.03512).
 *
 * General conventions
 *   - Every call returns a bt_status and never aborts or throws across the ABI.
 *     On failure, bt_last_error(ctx) returns a thread-local message.
 *   - Host arrays belong to the caller and are read or written only during
 *     the call (inputs are copied before the call returns).
 *   - Device memory is owned by the library (a context allocates it within the
 *     byte budget given to bt_create; BT_EBUDGET when a call would exceed it).
 *   - `stream` is a cudaStream_t passed as void*; NULL means the context's own
 *     stream. Calls that return host results synchronise that stream first.
 *   - There is no CPU fallback: without a usable GPU, bt_create returns
 *     BT_ECUDA.
 *   - The synchronous pricing calls of one context (exact, move-by-move,
 *     plug-in, Greeks and Monte Carlo) share the context's reusable device
 *     scratch and run one at a time when called from several threads; a
 *     context per thread runs them concurrently.
 *
 * Notation (the paper's): a path x = (x_1..x_N), 1 = up (Section 1); path
 * index b in [0,2^N) holds x_t in bit N-t, so x_1 is the most significant bit,
 * as the rank bits come first in Section 3. S_t = S0 u^{U_t} d^{t-U_t} with
 * U_t = x_1 + ... + x_t (Algorithm 1), p(x) = p^{U_N}(1-p)^{N-U_N} (Section 2),
 * V = e^{-qT} sum_x V_N(x) p(x) (eq. f13); the rate q is called `rate`.
 */
#ifndef BTREE_H
#define BTREE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BT_OK = 0,
    BT_EINVAL = 1,        /* invalid argument (message says which)             */
    BT_ENOMEM = 2,        /* host or device allocation failed                   */
    BT_EBUDGET = 3,       /* the context's device byte budget would be exceeded */
    BT_ECUDA = 4,         /* a CUDA call failed (message carries its error)     */
    BT_ETIMEOUT = 5,      /* a bounded wait expired                             */
    BT_EUNSUPPORTED = 6   /* valid input outside what the library supports    */
} bt_status;

/* Tree parametrisations (Section 2, assumptions A1-A3). */
typedef enum {
    BT_TREE_CRR = 0,      /* u = e^{sigma sqrt(dt)}, d = 1/u                     */
    BT_TREE_SEYDEL = 1,   /* beta = (e^{-q dt} + e^{(q+sigma^2) dt})/2,
                             u = beta + sqrt(beta^2 - 1), d = 1/u. The paper
                             prints "+1" under the root; "-1" is the reading that
                             satisfies A1-A3 with the lognormal second moment and
                             reproduces the exact values printed in Section 5.  */
    BT_TREE_EXPLICIT = 2  /* the caller gives u, d = 1/u, p                     */
} bt_tree_kind;           /* all kinds: p = (e^{q dt} - d)/(u - d) unless EXPLICIT */

/* Payoffs V_N(x). Averages and extremes run over S_1..S_N (Section 5). */
typedef enum {
    BT_EURO_CALL = 0,            /* max(S_N - K, 0)              (eq. call)          */
    BT_EURO_PUT = 1,             /* max(K - S_N, 0)              (eq. put)           */
    BT_ASIAN_ARITH_CALL = 2,     /* max(A - K, 0), A = (1/N) sum_t S_t              */
    BT_ASIAN_ARITH_PUT = 3,      /* max(K - A, 0)                (Section 5)         */
    BT_ASIAN_GEO_CALL = 4,       /* max(G - K, 0), G = exp((1/N) sum_t ln S_t)      */
    BT_ASIAN_GEO_PUT = 5,        /* max(K - G, 0)                                    */
    BT_LOOKBACK_FIXED_CALL = 6,  /* max(max_t S_t - K, 0)                            */
    BT_LOOKBACK_FIXED_PUT = 7    /* max(K - min_t S_t, 0)        (Section 5)         */
} bt_payoff;

typedef enum {
    BT_PREC_FP64 = 0,       /* every path in FP64                                    */
    BT_PREC_FP32_COMP = 1   /* path arithmetic in FP32 on coefficients carried as
                               FP32 pairs, group sums folded with error-free
                               transformations, FP64 across blocks; 1e-9
                               relative for the exhaustive lattice sums          */
} bt_precision;

/* One pricing problem. 80 bytes, naturally aligned. */
typedef struct {
    int32_t N;          /* tree depth, 1..40 for exact sums, 1..4096 for MC      */
    int32_t tree_kind;  /* bt_tree_kind                                          */
    int32_t payoff;     /* bt_payoff                                             */
    int32_t pad;        /* must be 0                                             */
    double S0, K, rate, sigma, T;  /* S0 > 0, K >= 0, T > 0, sigma > 0 (unless
                                      EXPLICIT), all finite                   */
    double u, d, p;     /* read only for BT_TREE_EXPLICIT: u > 1, d = 1/u, 0<p<1 */
} bt_option;

typedef struct {
    double value;       /* discounted value V                                    */
    double err_est;     /* exact sums: the stated error of V from rounding,
                           rel |V|: rel = 1e-12 in FP64 (and for the
                           move-by-move trees FP32_COMP prices in FP64);
                           1e-9 in FP32_COMP. Values below 1e-3 S0 carry
                           1e-12 S0 absolute as well. For the FP32 passes
                           that round each path once this is the measured
                           envelope of averaged roundings, not a bound;
                           MC: 0                                              */
    double stderr_mc;   /* MC: standard error of `value`; exact sums: 0          */
    double var_plain;   /* MC: estimated variance of one undiscounted draw
                           V(X) (for plain-MC comparisons); exact sums: 0        */
    int64_t paths;      /* exact: 2^N paths summed; MC: samples drawn            */
} bt_result;

typedef struct bt_ctx bt_ctx;

/* Library and context ------------------------------------------------------ */
const char *bt_version(void);
const char *bt_status_str(bt_status s);
/* Message of the last failed call on the calling thread ("" if none). The
 * message is thread-local, not per context: ctx is accepted for symmetry with
 * the other calls and may be NULL. */
const char *bt_last_error(const bt_ctx *ctx);

/* Create a context on CUDA device `device` that may hold up to
 * `device_budget_bytes` of library-owned device memory (0 = 8 GiB).
 * BT_ECUDA when no usable device exists. */
bt_status bt_create(int device, size_t device_budget_bytes, bt_ctx **out);
void bt_destroy(bt_ctx *ctx);
/* Device bytes currently held by the context. */
size_t bt_device_bytes(const bt_ctx *ctx);

/* Section 2, A1-A3: (u, d, p) of one option, computed in FP64 on the host.
 * BT_EINVAL if p is not in (0,1) or an input is out of range. */
bt_status bt_tree_params(const bt_option *opt, double *u, double *d, double *p);

/* Exhaustive sums (eq. f13) ------------------------------------------------ */
/* Prices opts[0..n) exactly: every one of the 2^N paths of each option is
 * evaluated. Prefix/suffix decomposition: the first P = N - L steps of a path
 * form its prefix (Section 3's rank bits, eq. f14) and the last L its suffix;
 * each block of threads sums the paths of a range of prefixes against a
 * shared-memory suffix table, and block partials are reduced in FP64 in a
 * fixed order (eq. f15). An arithmetic or geometric Asian or a European call
 * immediately followed by the put of identical parameters (or the reverse) is
 * evaluated in one pass over the paths; each still counts its own 2^N paths.
 * FP32_COMP rounds each path once in FP32 only for the arithmetic Asian on
 * trees of 2^28 paths or more with at least 2^27 effective paths,
 * 1 / sum_x p(x)^2 = (p^2 + (1-p)^2)^-N; every other option (and the other
 * payoffs always) is summed over suffix classes in FP32 pairs with no
 * per-path rounding. out[0..n) receives the results in input order.
 * Synchronous on `stream`.
 * Errors: BT_EINVAL (bad option, message names the index: N < 1 or N > 40,
 * S0 <= 0, K < 0, T <= 0, sigma <= 0, p outside (0,1), u <= d, a non-finite
 * value), BT_EUNSUPPORTED (FP32_COMP with min(p,1-p) < 0.004, whose weights
 * leave the FP32 range), BT_EBUDGET, BT_ECUDA. */
bt_status bt_price_exact(bt_ctx *ctx, const bt_option *opts, int32_t n, bt_precision prec,
                         bt_result *out, void *stream);

/* A prepared exhaustive pass for repeated runs with the inputs resident on the
 * device. plan_create validates and copies opts to device memory owned by the
 * plan and sizes all buffers; plan_run then performs every step on the device
 * (tree parameters, suffix and prefix tables, the path sums, the reduction);
 * plan_read copies the results to the host. */
typedef struct bt_exact_plan bt_exact_plan;
typedef struct {
    int32_t n_options;
    int32_t n_jobs;           /* passes over paths (call/put pairs share one)   */
    int64_t n_items;          /* work items (block-sized prefix ranges)          */
    int64_t payoff_paths;     /* sum over options of 2^N                         */
    int64_t path_evaluations; /* sum over jobs of 2^N                            */
    size_t device_bytes;      /* device memory held by the plan                  */
    size_t h2d_bytes;         /* host-to-device bytes bt_price_exact copies per call */
    size_t d2h_bytes;         /* device-to-host bytes of the results             */
} bt_exact_plan_info;

bt_status bt_exact_plan_create(bt_ctx *ctx, const bt_option *opts, int32_t n, bt_precision prec,
                               bt_exact_plan **out);
/* Enqueue one full pass on `stream` (asynchronous; results stay on device). */
bt_status bt_exact_plan_run(bt_exact_plan *plan, void *stream);
/* Enqueue the pass restricted to shard `shard` of `n_shards` (work items
 * i with i % n_shards == shard, the round-robin partition suggested at the
 * end of Section 3); results then hold this shard's partial values. */
bt_status bt_exact_plan_run_shard(bt_exact_plan *plan, int32_t shard, int32_t n_shards, void *stream);
/* Synchronise `stream` and copy results (input order) to out[0..n). */
bt_status bt_exact_plan_read(bt_exact_plan *plan, bt_result *out, void *stream);
/* Synchronise and copy per-work-item undiscounted partial sums: partials has
 * room for 2*n_items doubles (call slot, put slot per item); item_job and
 * item_first_prefix (may be NULL) receive each item's job index and first
 * prefix index. Work items of job j cover prefixes [first, first + count) of
 * that job's 2^P prefixes, all 2^L suffixes each. */
bt_status bt_exact_plan_partials(bt_exact_plan *plan, double *partials, int32_t *item_job,
                                 int64_t *item_first_prefix, void *stream);
/* Job layout: for job j, option indices (call slot, put slot; -1 if unused),
 * split (P, L) and its number of prefixes per work item. */
bt_status bt_exact_plan_job(const bt_exact_plan *plan, int32_t j, int32_t *opt_call, int32_t *opt_put,
                            int32_t *P, int32_t *L, int32_t *prefixes_per_item);
bt_status bt_exact_plan_info_get(const bt_exact_plan *plan, bt_exact_plan_info *info);
/* The split the exhaustive pass uses for one option priced alone at `prec`,
 * computed on the host (no device, no context): P prefix steps and L suffix
 * steps (P + L = N; Section 3's rank bits are the prefix), work items of
 * prefixes_per_item consecutive prefixes, n_items = ceil(2^P /
 * prefixes_per_item). Work item i covers the path indices [i ppi 2^L,
 * (i + 1) ppi 2^L) (first step most significant). For ranks that compute
 * their share of the items some other way than through a plan. Errors: as
 * bt_price_exact's validation. Any pointer may be NULL. */
bt_status bt_exact_split(const bt_option *opt, bt_precision prec, int32_t *P, int32_t *L, int32_t *prefixes_per_item,
                         int64_t *n_items);
/* Duration in milliseconds of the path-sum kernel of the most recent run,
 * measured with CUDA events recorded on that run's stream just before and
 * after the kernel launch. Synchronises on the end event. BT_EINVAL before
 * the first run. */
bt_status bt_exact_plan_kernel_ms(bt_exact_plan *plan, float *ms);
void bt_exact_plan_destroy(bt_exact_plan *plan);

/* Time-varying trees ------------------------------------------------------- */
/* eq. f13 with per-step moves and probabilities -- the case Section 2 names
 * where eq. f8 no longer applies. Step t of option i multiplies the price by
 * u_t (up, with probability p_t) or by d_t, read from the host array steps:
 * (u_t, d_t, p_t) = steps[3 (o_i + t - 1) + 0, 1, 2] with o_i = N_0 + ... +
 * N_{i-1} (options' steps concatenated, step 1 first). Of opts[i] the fields
 * N (<= 40), payoff, S0, K, rate and T (discount e^{-rate T}) are used;
 * tree_kind, sigma, u, d, p are ignored. The tree need not recombine: every
 * path is evaluated, with weight prod_t p_t^{x_t} (1 - p_t)^{1 - x_t}.
 * Requires 0 < d_t < u_t and 0 < p_t < 1 (BT_EINVAL), and for the FP32
 * pass (see bt_price_exact_moves) min(p_t, 1 - p_t) >= 0.004
 * (BT_EUNSUPPORTED). A call immediately followed by the put of the same
 * field, tree (identical steps) and strike, or the reverse, is one pass.
 * Accuracy, results and errors as bt_price_exact_moves with b = 2;
 * synchronous on `stream`. */
bt_status bt_price_exact_steps(bt_ctx *ctx, const bt_option *opts, int32_t n, const double *steps,
                               bt_precision prec, bt_result *out, void *stream);
/* The same affine passes (FP32_COMP or FP64) for trees with b = branches
 * (2..8) branches per node (the end of Section 3: trinomial and wider trees),
 * moves given as for bt_price_exact_branching: for each option's steps in
 * turn, b factors then b probabilities indexed by the digit (factors > 0,
 * probabilities in [0,1] summing to 1 within 1e-12: BT_EINVAL). b^N <= 2^42.
 * A path is N base-b digits, the first step most significant; paths = b^N.
 * The built-in payoffs only (for a plug-in, bt_price_exact_branching).
 * A call immediately followed by the put of the same field, moves and
 * strike (or the reverse) is one pass. FP32_COMP: the FP32 pass, which
 * rounds every path once, runs a tree of 2^28 paths or more with at least
 * 2^27 effective paths (1 / sum_x p(x)^2 = prod_t 1 / sum_k q_tk^2) whose
 * suffix values do not repeat (on average at most eight suffixes per
 * distinct value: a recombining tree repeats end prices, level sums and
 * extremes); it needs every positive probability >= 0.004 (BT_EUNSUPPORTED)
 * and meets 1e-9 relative (plus 1e-12 S0). Every other option runs the FP64
 * pass (err_est then states 1e-12). */
bt_status bt_price_exact_moves(bt_ctx *ctx, const bt_option *opts, int32_t n, int32_t branches,
                               const double *moves, bt_precision prec, bt_result *out, void *stream);

/* Payoff plug-ins ------------------------------------------------------------ */
/* Any V(x) of the whole path (the general expected value of eq. expval, and
 * eq. f13 for payoffs beyond the eight built in): `source` is CUDA C++
 * defining struct Payoff with the state-machine interface documented in
 * btree_payoff.cuh. bt_plugin_compile appends it to that header and builds
 * the generic pass for the context's GPU with the run-time compiler
 * (libnvrtc, loaded on first use: BT_EUNSUPPORTED without it). A compile
 * error returns BT_EINVAL; the compiler's log (also on success) goes to
 * log[0..log_size) if log is not NULL. The plug-in belongs to the caller
 * until bt_plugin_destroy. */
typedef struct bt_payoff_plugin bt_payoff_plugin;
bt_status bt_plugin_compile(bt_ctx *ctx, const char *source, char *log, size_t log_size, bt_payoff_plugin **out);
void bt_plugin_destroy(bt_payoff_plugin *plugin);
/* V = e^{-rate T} sum_x p(x) V(x) for opts[0..n), every path evaluated
 * (N <= 40; FP64 weights and sums, two state steps per path on average).
 * steps: as for bt_price_exact_steps, or NULL for each option's own tree
 * (tree_kind, sigma, ...). params: host array [n][8] handed to the plug-in,
 * or NULL for param[0] = K and zeros. out[i].value, paths = 2^N, err_est =
 * 1e-13 |value|. Synchronous on `stream`. */
bt_status bt_price_exact_plugin(bt_ctx *ctx, const bt_payoff_plugin *plugin, const bt_option *opts, int32_t n,
                                const double *steps, const double *params, bt_result *out, void *stream);

/* Trees with b branches per node (the end of Section 3: the partition of the
 * paths applies to trinomial and wider trees). A path is N digits in
 * 0..b-1, the first step the most significant digit of its index in base b.
 * moves: host array, for each option's steps in turn (step 1 first, options
 * concatenated), b factors then b probabilities indexed by the digit: digit
 * k of step t multiplies the price by factor k with probability k (factors
 * > 0, probabilities in [0,1] summing to 1 within 1e-12, else BT_EINVAL).
 * With plugin NULL each option's own payoff (opts[i].payoff, K) is priced;
 * else the plug-in with params as for bt_price_exact_plugin. 2 <= branches
 * <= 8, b^N <= 2^40 (BT_EUNSUPPORTED above). Of opts[i]: N, payoff, S0, K,
 * rate, T. Every path is evaluated by the generic pass of btree_payoff.cuh
 * (FP64). paths = b^N. Synchronous on `stream`. */
bt_status bt_price_exact_branching(bt_ctx *ctx, const bt_payoff_plugin *plugin, const bt_option *opts, int32_t n,
                                   int32_t branches, const double *moves, const double *params, bt_result *out,
                                   void *stream);

/* Greeks of the exhaustive value ------------------------------------------- */
/* Not in the paper: derivatives of eq. f13 for opts[0..n): value[i] = V and
 * grad[4 i + 0..3] = dV/dS0, dV/dsigma, dV/drate, dV/dK. One derivative pass
 * over every path accumulates, next to the value, the in-the-money weight,
 * the path-weight derivative sum_x w(x) payoff(x) k(x) (k = up-count, for
 * dV/dp) and the pathwise dV/du at fixed p; the host applies the chain rule
 * through u(sigma, rate) and p(u, rate) of the option's tree (CRR, Seydel; an
 * explicit tree has dV/dsigma = 0 and dV/drate = -T V) and Euler's identity
 * S0 dV/dS0 + K dV/dK = V (the payoffs are homogeneous of degree one in
 * (S0, K)). Only BT_PREC_FP32_COMP (BT_EUNSUPPORTED otherwise). Synchronous. */
bt_status bt_greeks_exact(bt_ctx *ctx, const bt_option *opts, int32_t n, bt_precision prec, double *value,
                          double *grad, void *stream);

/* Monte Carlo (Section 4) -------------------------------------------------- */
typedef enum {
    BT_MC_PARTITIONED = 0,  /* eq. mc12: R suffix draws inside each stratum          */
    BT_MC_SHARED = 1        /* eq. mc16 (Remark of Section 4): the same R suffix
                               draws reused under every stratum's prefix            */
} bt_mc_kind;

/* Partitioned Monte Carlo with equal allocation. Stratum m in [0, 2^strata_bits)
 * fixes the first strata_bits steps to m's bits, most significant first (the
 * rank bits of Section 3); each stratum draws samples_per_stratum suffixes of
 * N - strata_bits steps. Step t of sample i in stratum m goes up iff word
 * (t - strata_bits - 1) % 4 of Philox-4x32-10 with counter
 * ((t - strata_bits - 1) / 4, i, m, option index) and key (seed low 32 bits,
 * seed high 32 bits) is below round(p 2^32) (clamped to [1, 2^32 - 1]).
 * value = e^{-qT} sum_m P(D_m) mean_m (eq. mc12); stderr_mc =
 * e^{-qT} sqrt(sum_m P(D_m)^2 s_m^2 / R) with the unbiased s_m^2; var_plain
 * = the implied variance of one undiscounted draw, sum_m P(D_m) Var_m +
 * Var_D E[V|D] (eq. mc14), for comparison with plain MC; paths = samples.
 * strata_bits = 0 is plain MC. Limits: N <= 4096, strata_bits <= min(N, 24),
 * 1 <= samples_per_stratum <= 2^32. Synchronous on `stream`. */
bt_status bt_price_mc(bt_ctx *ctx, const bt_option *opts, int32_t n, int32_t strata_bits,
                      int64_t samples_per_stratum, uint64_t seed, bt_result *out, void *stream);
/* As bt_price_mc, with the estimator kind (BT_MC_SHARED: counter word 2 is 0
 * for every stratum, strata_bits <= 10, stderr from the sample variance of
 * h_i = sum_m P(D_m) V(z_m, y_i), var_plain = 0) and, if strata_stats is not
 * NULL, per-stratum (mean, unbiased variance, P(D_m)) triples for every
 * option, options concatenated (2^strata_bits triples per option; one triple
 * for BT_MC_SHARED). */
bt_status bt_price_mc_ex(bt_ctx *ctx, const bt_option *opts, int32_t n, int32_t strata_bits,
                         int64_t samples_per_stratum, uint64_t seed, int32_t kind, bt_result *out,
                         double *strata_stats, void *stream);
/* One shard of the Partitioned estimator for splitting strata across GPUs
 * or processes (the strata of Section 4 are the rank blocks of Section 3):
 * this call covers strata m = shard + j * n_shards only (1 <= n_shards <=
 * 2^strata_bits, 0 <= shard < n_shards), with the same Philox streams as the
 * unsharded call, so the shards' strata are exactly its strata. out[i].value
 * and out[i].stderr_mc^2 are this shard's terms of eq. mc12 and of its
 * variance: over all shards, value sums to the unsharded value and
 * stderr_mc^2 to its square (up to FP64 rounding). var_plain = 0 (it needs
 * every stratum's mean); paths = samples drawn by this shard. strata_stats
 * (optional) receives (mean, unbiased variance, P(D_m)) for this shard's
 * strata in ascending m, options concatenated. */
bt_status bt_price_mc_shard(bt_ctx *ctx, const bt_option *opts, int32_t n, int32_t strata_bits,
                            int64_t samples_per_stratum, uint64_t seed, int32_t shard, int32_t n_shards,
                            bt_result *out, double *strata_stats, void *stream);
/* The device Philox-4x32-10 used above, evaluated for n counters and keys
 * (host arrays ctr[n][4], key[n][2], out[n][4]); for verification. */
bt_status bt_philox4x32_10(bt_ctx *ctx, const uint32_t *ctr, const uint32_t *key, uint32_t *out, int32_t n);

/* Continuous-batching pricing server --------------------------------------- */
/* Not in the paper (its SPMD scheme prices one problem at a time): a server
 * that prices a stream of single-option requests of mixed N and payoff. A
 * scheduler thread admits requests in arrival order while a slot is free and
 * the device pool has room for the request's tables and per-item partials
 * (admission by memory), keeps up to n_streams path-sum launches in flight,
 * each over work items of all admitted requests (smallest remaining work
 * first), and finalises a request with the same fixed-order reduction as
 * bt_price_exact, so each result is identical alone and in the mix. */
typedef struct bt_server bt_server;
typedef struct {
    int32_t max_active;            /* requests admitted at once (slots); 0 = 1024          */
    int32_t n_streams;             /* path-sum launches in flight; 0 = 6                    */
    int32_t max_items_per_launch;  /* 2^10-prefix work items per launch; 0 = 4864           */
    int32_t use_fp64;              /* precision bt_serve_replay submits with: 0 = FP32_COMP, 1 = FP64 */
    size_t device_budget_bytes;    /* device memory for slots, tables, partials; 0 = 8 GiB */
} bt_server_cfg;
typedef struct {
    int64_t submitted, completed, launches, items;
    int32_t active, pending;       /* admitted and waiting requests right now              */
    double p50_ms, p99_ms, mean_ms, max_ms;  /* latency = completion - submission        */
    double throughput_rps, paths_per_s;     /* over first submission .. last completion */
    double busy_s;                 /* scheduler time with GPU work in flight               */
    int32_t peak_active;           /* most requests admitted at one time                   */
    int32_t reserved;
    int64_t pool_bytes;            /* device pool for tables and partials                  */
} bt_server_stats_t;

/* Starts the scheduler thread; allocates device_budget_bytes from the context
 * (BT_EBUDGET if that exceeds the context's budget). */
bt_status bt_server_start(bt_ctx *ctx, const bt_server_cfg *cfg, bt_server **out);
/* Queues one option, priced at precision `prec`; returns at once with a
 * ticket. Requests of both precisions share the server (each launch runs one
 * precision's kernel). Validation errors as bt_price_exact; BT_EBUDGET if one
 * request alone exceeds the pool. */
bt_status bt_submit(bt_server *srv, const bt_option *opt, bt_precision prec, uint64_t *ticket);
/* Waits up to timeout_ms for the ticket's result (BT_ETIMEOUT on expiry; the
 * request stays queued). A ticket can be collected once. */
bt_status bt_wait(bt_server *srv, uint64_t ticket, int32_t timeout_ms, bt_result *out);
/* Non-blocking: *done = 1 and the result if finished (collects the ticket). */
bt_status bt_poll(bt_server *srv, uint64_t ticket, bt_result *out, int32_t *done);
bt_status bt_server_stats(bt_server *srv, bt_server_stats_t *out);
/* Finishes all queued requests, stops the thread, frees its memory; results
 * not yet collected are discarded. No other call on srv may be running (a
 * thread blocked in bt_wait must have returned) or follow. */
bt_status bt_server_stop(bt_server *srv);
/* Replays an arrival schedule (seconds from the call) of n single-option
 * requests: mode 1 through a server started with cfg, mode 0 as plain
 * pricing -- one bt_price_exact per request in arrival order. results are in
 * request order; latency_ms[i] = completion of request i minus its
 * scheduled arrival, on the same clock for both modes; wall_s the span. */
bt_status bt_serve_replay(bt_ctx *ctx, const bt_server_cfg *cfg, const bt_option *opts, const double *arrival_s,
                          int32_t n, int32_t mode, bt_result *results, double *latency_ms, double *wall_s);

/* Allocation-free exhaustive pricing --------------------------------------- */
/* The paper has no counterpart: this exists for callers that cannot allocate
 * device memory while they run -- for example an application whose own
 * allocator owns the device, or a latency-sensitive loop that cannot afford
 * cudaMalloc/cudaFree (cudaFree synchronises the whole device).
 *
 * Same computation and results as bt_price_exact (host arrays opts[0..n) in,
 * out[0..n) out, synchronous on `stream`, NULL = the legacy default stream),
 * but every intermediate buffer lives in one fixed device array of
 * BT_NOALLOC_SCRATCH_BYTES that the library defines statically: no context is
 * needed and nothing is allocated (no cudaMalloc, cudaFree, or any allocating
 * library routine). Every GPU that loads the library holds that array until
 * the process exits.
 *
 * The first call on a device (with that device current) looks up the array's
 * device address; make that first call before any stream capture.
 *
 * All calls on a device share the array, and two calls whose GPU work
 * overlapped would race on it. The function prevents that: it holds a
 * process-wide lock from its first copy until its stream has drained, and it
 * clears the parts that must start at zero on every call.
 *
 * Limits: n <= BT_NOALLOC_MAX_OPTIONS, and the batch's tables and per-item
 * partials must fit in the array (for example 64 options with N <= 30, or a
 * single option up to N = 40); beyond either, BT_EUNSUPPORTED with a message
 * giving the bytes needed. Other errors as bt_price_exact. */
#define BT_NOALLOC_SCRATCH_BYTES (8u << 20)
#define BT_NOALLOC_MAX_OPTIONS 64
bt_status bt_price_exact_noalloc(const bt_option *opts, int32_t n, bt_precision prec, bt_result *out,
                                 void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BTREE_H */
