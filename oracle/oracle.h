/*
 * CPU oracle for expected values over the Bernoulli paths of a recombinant
 * binomial tree (Popuri, Raim, Neerchal, Gobbert, arXiv 1701.03512).
 *
 * TEST INFRASTRUCTURE ONLY. This library is a plain, slow, FP64 restatement
 * of what the paper computes. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it. It shares no code, header, table or
 * constant generator with the CUDA library: nothing in the product links or
 * calls it, and it calls nothing of the product.
 *
 * Conventions (the paper's notation):
 *   path x = (x_1..x_N), 1 = up (Section 1); a path index b in [0, 2^N) holds
 *   x_t in bit (N - t), so x_1 is the most significant bit -- the rank bits
 *   of Section 3 come first (Listing 1 prepends the rank's bits).
 *   S_t = S0 u^{U_t} d^{t - U_t}, U_t = x_1 + ... + x_t   (Algorithm 1 grid)
 *   p(x) = p^{U_N} (1-p)^{N-U_N}                           (Section 2)
 *   V = e^{-qT} sum_x p(x) V_N(x)                          (eq. f13)
 * The rate q of the paper is called `rate` here.
 */
#ifndef BT_ORACLE_H
#define BT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Payoffs. Numbering agrees with the product's public header (an interface
 * both sides must share); the definitions below are the oracle's own. */
enum {
    ORC_EURO_CALL = 0, ORC_EURO_PUT = 1,
    ORC_ARITH_CALL = 2, ORC_ARITH_PUT = 3,
    ORC_GEO_CALL = 4, ORC_GEO_PUT = 5,
    ORC_LOOK_CALL = 6, ORC_LOOK_PUT = 7
};
enum { ORC_TREE_CRR = 0, ORC_TREE_SEYDEL = 1, ORC_TREE_EXPLICIT = 2 };

typedef struct {
    int32_t N;
    int32_t payoff;
    double S0, K, u, d, p;
    double disc; /* e^{-qT} */
} orc_model;

/* Tree parameters (Section 2, A1-A3). Returns 0 on success, -1 if p is not in
 * (0,1) or an input is out of range. */
int orc_tree(int kind, int N, double sigma, double rate, double T,
             double *u, double *d, double *p);

/* Build a model from option fields; explicit trees pass u,d,p through. */
int orc_model_make(int N, int kind, int payoff, double S0, double K, double rate,
                   double sigma, double T, double u, double d, double p, orc_model *m);

/* Payoff of one path index b (Listing 1's calc_payoff, Section 5 payoffs). */
double orc_path_payoff(const orc_model *m, uint64_t b);
/* Probability of one path index (Listing 1's calc_path_prob, Section 2). */
double orc_path_prob(const orc_model *m, uint64_t b);

/* Plain enumeration of sum_{b in [lo,hi)} p(x_b) V_N(x_b) (undiscounted),
 * Neumaier-compensated; eq. f14 without the discount factor. */
void orc_sum_range(const orc_model *m, uint64_t lo, uint64_t hi, double *sum, double *comp);

/* Full exhaustive value by the SPMD scheme of Section 3: M = 2^r workers,
 * worker m takes the paths whose first r steps are the bits of m (eq. f14),
 * partial values are added in rank order (eq. f15). nthreads is rounded down
 * to a power of two not above 2^N. Returns the discounted value. */
double orc_price_exhaustive(const orc_model *m, int nthreads);

/* Same partition, over the path-index range [lo,hi) only (for bounded CPU
 * baselines); returns the undiscounted sum. */
double orc_sum_range_mt(const orc_model *m, uint64_t lo, uint64_t hi, int nthreads);

/* eq. f11: per-leaf path-probability sums by enumeration, out[i] for i=0..N. */
void orc_leaf_prob_sums(const orc_model *m, double *out);

/* eq. f8: European value from the leaf distribution (binomial weights). */
double orc_price_european_closed(const orc_model *m);
/* Textbook backward induction on the Algorithm 1 grid (European only). */
double orc_price_european_backward(const orc_model *m);

/* Exact geometric-average Asian by dynamic programming over
 * (step, up-count U_t, running sum of up-counts W_t); O(N^4). */
double orc_price_geometric_dp(const orc_model *m);
/* Exact fixed-strike lookback (max for calls, min for puts over S_1..S_N) by
 * dynamic programming over (level 2U_t - t, running extreme level); needs
 * u*d = 1 (A1). O(N^3). */
double orc_price_lookback_dp(const orc_model *m);
/* Exact arithmetic Asian by meet in the middle: the last L steps' relative
 * partial sums are sorted once, and every prefix adds the in-the-money part
 * of that sorted list through compensated cumulative sums. An independent
 * exact algorithm for the same sum as eq. f13 (not the paper's method). */
double orc_price_asian_mitm(const orc_model *m, int L);

/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): out = bijection of ctr
 * under key. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Bernoulli threshold: x = (r < thr) for a uniform 32-bit r. */
uint64_t orc_bernoulli_threshold(double p);

/* Partitioned Monte Carlo (Section 4, eq. mc9/mc12). Strata m in [0, 2^mb)
 * fix x_1..x_mb to the bits of m (MSB first). Each stratum draws Rm suffixes;
 * step t (t > mb) of sample i of stratum m uses word (t-mb-1)%4 of
 * Philox(ctr = ((t-mb-1)/4, i, shared ? 0 : m, stream), key = (seed_lo, seed_hi)).
 * Outputs (undiscounted theta): theta_s, var_s = sum_m P(D_m)^2 s_m^2 / Rm with
 * the unbiased s_m^2; per-stratum means/variances if the arrays are non-null.
 * shared != 0 selects the Shared-Sample estimator of the Remark (eq. mc16):
 * the same Rm suffix draws under every prefix; var_s is then its variance
 * estimate (1/R) * sample variance of sum_m V(z_m, y_i) P(D_m). */
void orc_mc(const orc_model *m, int mb, int64_t Rm, uint64_t seed, uint32_t stream, int shared,
            double *theta, double *var, double *stratum_mean, double *stratum_var,
            double *stratum_prob);

/* One stratum z of orc_mc (same draws): mean, unbiased variance, P(D_z). */
void orc_mc_stratum(const orc_model *m, int mb, uint64_t z, int64_t Rm, uint64_t seed, uint32_t stream,
                    double *mean, double *var, double *prob);

/* Exact conditional moments per stratum by enumeration (small N):
 * mean_m = E[V | D_m], var_m = Var[V | D_m], prob_m = P(D_m). */
void orc_stratum_moments(const orc_model *m, int mb, double *mean, double *var, double *prob);

/* Time-varying trees (eq. f13 with per-step moves and probabilities; the
 * case Section 2 names where eq. f8 no longer applies): step t multiplies the
 * price by u[t-1] (up, probability p[t-1]) or by d[t-1]; the tree need not
 * recombine. p(x) = prod_t p_t^{x_t} (1-p_t)^{1-x_t}. Payoffs as above. */
typedef struct {
    int32_t N;
    int32_t payoff;
    double S0, K;
    double disc;                 /* e^{-qT} */
    const double *u, *d, *p;     /* N entries each, step 1 first */
} orc_steps_model;

/* Path walk in the shape of Listing 1: rebuild path b step by step. */
double orc_steps_path_payoff(const orc_steps_model *m, uint64_t b);
double orc_steps_path_prob(const orc_steps_model *m, uint64_t b);
/* Undiscounted Neumaier sum of p(x) V_N(x) over path indices [lo, hi). */
void orc_steps_sum_range(const orc_steps_model *m, uint64_t lo, uint64_t hi, double *sum, double *comp);
/* Discounted value by the Section 3 partition over nthreads workers (rounded
 * down to a power of two), partials added in rank order (eq. f14, f15). */
double orc_steps_price(const orc_steps_model *m, int nthreads);

/* Several payoffs of one time-varying tree in one enumeration: out[j] is the
 * discounted value of payoff pay[j] with strike K[j] (the model's own payoff
 * and K are not used), each path walked once for all of them; same partition
 * and reduction order as orc_steps_price. */
void orc_steps_price_multi(const orc_steps_model *m, int n, const int32_t *pay, const double *K, int nthreads,
                           double *out);

/* Trees with b branches per node (the end of Section 3: the partition of the
 * paths applies to trees with more than two branches, e.g. trinomial trees).
 * A path is N digits x_t in 0..b-1, the first step the most significant digit
 * of the path index in base b; digit k of step t multiplies the price by
 * f[t-1][k] with probability q[t-1][k] (each row of q sums to 1).
 * p(x) = prod_t q[t-1][x_t]. Payoffs as above. */
typedef struct {
    int32_t N, b;
    int32_t payoff, pad;
    double S0, K;
    double disc;                 /* e^{-qT} */
    const double *f, *q;         /* N x b each, step 1 first */
} orc_branch_model;

double orc_branch_path_payoff(const orc_branch_model *m, uint64_t idx);
double orc_branch_path_prob(const orc_branch_model *m, uint64_t idx);
/* Discounted value: b^N paths split into nthreads contiguous index ranges
 * (Section 3's partition by leading digits when nthreads is a power of b),
 * partials added in rank order. Needs b^N < 2^63. */
double orc_branch_price(const orc_branch_model *m, int nthreads);
/* As orc_steps_price_multi for a b-ary tree: out[j] for payoff pay[j], strike K[j]. */
void orc_branch_price_multi(const orc_branch_model *m, int n, const int32_t *pay, const double *K, int nthreads,
                            double *out);
/* eq. expval for a payoff given as a function of the whole path: the value
 * e^{-qT} sum_x p(x) V(x) on the tree m (a time-varying binomial tree is b = 2
 * with factors (d_t, u_t) and probabilities (1 - p_t, p_t); m->payoff and m->K
 * are not used). Paths are visited in index order and passed to fn in blocks:
 * fn(user, count, N, S, x, v) receives S[i N + t - 1] = S_t and x[i N + t - 1]
 * = the digit of step t of the block's path i, and writes its payoff to v[i].
 * Single-threaded. */
typedef void (*orc_payoff_fn)(void *user, int32_t count, int32_t N, const double *S, const int32_t *x, double *v);
double orc_functional_price(const orc_branch_model *m, orc_payoff_fn fn, void *user);

/* European value by backward induction on a recombining b-ary lattice with
 * the same moves at every step (f[0], q[0] used for all steps; f_k = u^{k - c}
 * with c = (b-1)/2 so that node (t, j) has price S0 u^{j - c t}). */
double orc_branch_european_backward(const orc_branch_model *m);

/* Pathwise Greeks by enumeration for CRR trees: grad = dV/d(S0, sigma, rate, K).
 * Returns the value. */
double orc_greeks_crr(int N, int payoff, double S0, double K, double rate, double sigma,
                      double T, double grad[4]);

#ifdef __cplusplus
}
#endif
#endif
