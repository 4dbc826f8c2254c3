/*
 * CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Plain serial FP64 code, compiled with -ffp-contract=off so that every
 * expression rounds as written. Each function names the passage of
 * arXiv 1701.03512 it restates. Nothing here is tuned for speed.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Compensated (Neumaier) summation and double-double helpers               */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } nsum;

static void nsum_add(nsum *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double nsum_get(const nsum *a) { return a->s + a->c; }

typedef struct { double hi, lo; } dd;

static dd two_sum(double a, double b) {
    dd r; double s = a + b; double bb = s - a;
    r.hi = s; r.lo = (a - (s - bb)) + (b - bb); return r;
}
static dd fast_two_sum(double a, double b) {
    dd r; double s = a + b; r.hi = s; r.lo = b - (s - a); return r;
}
static dd dd_add(dd x, dd y) {
    dd s = two_sum(x.hi, y.hi);
    double e = s.lo + x.lo + y.lo;
    return fast_two_sum(s.hi, e);
}
static dd dd_mul_d(dd x, double b) {
    double p = x.hi * b;
    double e = fma(x.hi, b, -p);
    e += x.lo * b;
    return fast_two_sum(p, e);
}
static dd dd_from(double a) { dd r; r.hi = a; r.lo = 0.0; return r; }
static double dd_get(dd x) { return x.hi + x.lo; }

/* ------------------------------------------------------------------------ */
/* Tree parameters: Section 2, assumptions A1-A3 and the formulas for u, p   */
/* ------------------------------------------------------------------------ */
int orc_tree(int kind, int N, double sigma, double rate, double T, double *u, double *d, double *p) {
    if (N < 1 || !(T > 0.0) || !(sigma > 0.0) || !isfinite(rate)) return -1;
    double dt = T / (double)N;
    double uu;
    if (kind == ORC_TREE_CRR) {
        /* Cox-Ross-Rubinstein: u = e^{sigma sqrt(dt)}. */
        uu = exp(sigma * sqrt(dt));
    } else if (kind == ORC_TREE_SEYDEL) {
        /* Section 2 (following Seydel Sec. 1.4): beta = (e^{-q dt} + e^{(q+sigma^2) dt}) / 2 and
         * u = beta + sqrt(beta^2 - 1). The text prints "+1" under the root; only "-1"
         * gives ud = 1 together with the second-moment match and reproduces the
         * exact values printed in Section 5. */
        double beta = 0.5 * (exp(-rate * dt) + exp((rate + sigma * sigma) * dt));
        uu = beta + sqrt(beta * beta - 1.0);
    } else {
        return -1;
    }
    double dd_ = 1.0 / uu;                      /* A1: ud = 1 */
    double pp = (exp(rate * dt) - dd_) / (uu - dd_); /* A3: E[S_{t+1}|S_t] = S_t e^{q dt} */
    if (!(pp > 0.0 && pp < 1.0)) return -1;
    *u = uu; *d = dd_; *p = pp;
    return 0;
}

int orc_model_make(int N, int kind, int payoff, double S0, double K, double rate, double sigma,
                   double T, double u, double d, double p, orc_model *m) {
    if (N < 1 || N > 100000 || payoff < 0 || payoff > 7) return -1;
    if (!(S0 > 0.0) || !(K >= 0.0) || !(T > 0.0)) return -1;
    if (kind == ORC_TREE_EXPLICIT) {
        if (!(d > 0.0 && u > d && p > 0.0 && p < 1.0)) return -1;
    } else if (orc_tree(kind, N, sigma, rate, T, &u, &d, &p) != 0) {
        return -1;
    }
    m->N = N; m->payoff = payoff; m->S0 = S0; m->K = K;
    m->u = u; m->d = d; m->p = p;
    m->disc = exp(-rate * T);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: the grid S_{ij} = S0 u^j d^{i-j}, and its logarithms         */
/* ------------------------------------------------------------------------ */
typedef struct {
    int N;
    double *S;   /* S[t*(N+1) + j] */
    double *lnS; /* ln S[t*(N+1) + j] */
    double *w;   /* w[k] = p^k (1-p)^{N-k} */
} grid_t;

static int grid_make(const orc_model *m, grid_t *g) {
    int N = m->N;
    g->N = N;
    g->S = (double *)malloc(sizeof(double) * (size_t)(N + 1) * (size_t)(N + 1));
    g->lnS = (double *)malloc(sizeof(double) * (size_t)(N + 1) * (size_t)(N + 1));
    g->w = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    if (!g->S || !g->lnS || !g->w) return -1;
    double lu = log(m->u), ld = log(m->d), ls = log(m->S0);
    for (int i = 0; i <= N; ++i)
        for (int j = 0; j <= i; ++j) {
            g->S[i * (N + 1) + j] = m->S0 * pow(m->u, (double)j) * pow(m->d, (double)(i - j));
            g->lnS[i * (N + 1) + j] = ls + (double)j * lu + (double)(i - j) * ld;
        }
    for (int k = 0; k <= N; ++k) g->w[k] = pow(m->p, (double)k) * pow(1.0 - m->p, (double)(N - k));
    return 0;
}
static void grid_free(grid_t *g) { free(g->S); free(g->lnS); free(g->w); }

/* Payoff of a price summary; X is the payoff's underlying quantity. */
static double payoff_of(int payoff, double K, double X) {
    switch (payoff) {
    case ORC_EURO_CALL: case ORC_ARITH_CALL: case ORC_GEO_CALL: case ORC_LOOK_CALL:
        return X > K ? X - K : 0.0;      /* eq. call */
    default:
        return K > X ? K - X : 0.0;      /* eq. put */
    }
}

/* The payoff's underlying quantity along path b, stepping t = 1..N:
 *   European: S_N (Section 2); arithmetic Asian: (1/N) sum_{t=1}^N S_t (Section 5);
 *   geometric Asian: exp((1/N) sum_{t=1}^N ln S_t); lookback: max / min over
 *   t = 1..N of S_t (Section 5, fixed-strike lookback). */
static double path_quantity(const orc_model *m, const grid_t *g, uint64_t b, int *Uout) {
    int N = m->N, U = 0;
    double sum = 0.0, lsum = 0.0, mx = -INFINITY, mn = INFINITY, St = m->S0;
    for (int t = 1; t <= N; ++t) {
        int x = (int)((b >> (N - t)) & 1u);
        U += x;
        St = g->S[t * (N + 1) + U];
        sum += St;
        lsum += g->lnS[t * (N + 1) + U];
        if (St > mx) mx = St;
        if (St < mn) mn = St;
    }
    *Uout = U;
    switch (m->payoff) {
    case ORC_EURO_CALL: case ORC_EURO_PUT: return St;
    case ORC_ARITH_CALL: case ORC_ARITH_PUT: return sum / (double)N;
    case ORC_GEO_CALL: case ORC_GEO_PUT: return exp(lsum / (double)N);
    case ORC_LOOK_CALL: return mx;
    default: return mn;
    }
}

double orc_path_payoff(const orc_model *m, uint64_t b) {
    grid_t g; if (grid_make(m, &g)) return NAN;
    int U; double X = path_quantity(m, &g, b, &U);
    double v = payoff_of(m->payoff, m->K, X);
    grid_free(&g); return v;
}

double orc_path_prob(const orc_model *m, uint64_t b) {
    int N = m->N, U = 0;
    for (int t = 1; t <= N; ++t) U += (int)((b >> (N - t)) & 1u);
    return pow(m->p, (double)U) * pow(1.0 - m->p, (double)(N - U));
}

/* eq. f14 (undiscounted): the sum of p(x) V_N(x) over a set of path indices.
 * The loop has the shape of Listing 1: rebuild the path, cost it in O(N),
 * accumulate probability times payoff. */
static void sum_range_grid(const orc_model *m, const grid_t *g, uint64_t lo, uint64_t hi, nsum *acc) {
    for (uint64_t b = lo; b < hi; ++b) {
        int U;
        double X = path_quantity(m, g, b, &U);
        double v = payoff_of(m->payoff, m->K, X);
        nsum_add(acc, g->w[U] * v);
    }
}

void orc_sum_range(const orc_model *m, uint64_t lo, uint64_t hi, double *sum, double *comp) {
    grid_t g; nsum acc = {0.0, 0.0};
    if (m->N > 62 || grid_make(m, &g)) { *sum = NAN; *comp = 0.0; return; }
    sum_range_grid(m, &g, lo, hi, &acc);
    grid_free(&g);
    *sum = acc.s; *comp = acc.c;
}

typedef struct {
    const orc_model *m; const grid_t *g; uint64_t lo, hi; nsum acc;
} worker_t;

static void *worker_run(void *arg) {
    worker_t *w = (worker_t *)arg;
    w->acc.s = 0.0; w->acc.c = 0.0;
    sum_range_grid(w->m, w->g, w->lo, w->hi, &w->acc);
    return NULL;
}

/* Runs contiguous ranges on threads and adds the partial sums in range order
 * (eq. f15's reduce, done deterministically). */
static double run_ranges(const orc_model *m, const grid_t *g, const uint64_t *bounds, int M) {
    worker_t *ws = (worker_t *)calloc((size_t)M, sizeof(worker_t));
    pthread_t *th = (pthread_t *)calloc((size_t)M, sizeof(pthread_t));
    int *started = (int *)calloc((size_t)M, sizeof(int));
    for (int r = 0; r < M; ++r) {
        ws[r].m = m; ws[r].g = g; ws[r].lo = bounds[r]; ws[r].hi = bounds[r + 1];
        started[r] = (M > 1) && pthread_create(&th[r], NULL, worker_run, &ws[r]) == 0;
        if (!started[r]) worker_run(&ws[r]);
    }
    nsum tot = {0.0, 0.0};
    for (int r = 0; r < M; ++r) {
        if (started[r]) pthread_join(th[r], NULL);
        nsum_add(&tot, ws[r].acc.s);
        nsum_add(&tot, ws[r].acc.c);
    }
    free(ws); free(th); free(started);
    return nsum_get(&tot);
}

/* Section 3: M = 2^r processes; process m owns B_m^N, the 2^{N-r} paths whose
 * first r steps are m's r-digit binary representation (z_{r-1} = x_1). */
double orc_price_exhaustive(const orc_model *m, int nthreads) {
    grid_t g; if (m->N > 62 || grid_make(m, &g)) return NAN;
    int r = 0;
    while (r < m->N && (2 << r) <= nthreads) ++r;
    int M = 1 << r;
    uint64_t *bounds = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(M + 1));
    for (int k = 0; k <= M; ++k) bounds[k] = (uint64_t)k << (m->N - r);
    double s = run_ranges(m, &g, bounds, M);
    free(bounds); grid_free(&g);
    return m->disc * s;
}

double orc_sum_range_mt(const orc_model *m, uint64_t lo, uint64_t hi, int nthreads) {
    grid_t g; if (m->N > 62 || grid_make(m, &g)) return NAN;
    int M = nthreads < 1 ? 1 : nthreads;
    uint64_t n = hi - lo;
    uint64_t *bounds = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(M + 1));
    for (int k = 0; k <= M; ++k) bounds[k] = lo + (uint64_t)(((unsigned __int128)n * (unsigned)k) / (unsigned)M);
    double s = run_ranges(m, &g, bounds, M);
    free(bounds); grid_free(&g);
    return s;
}

/* eq. f11: the probability of reaching leaf i is the sum of p(x) over the
 * paths with x'1 = i; summed here path by path. */
void orc_leaf_prob_sums(const orc_model *m, double *out) {
    int N = m->N;
    if (N > 40) return;
    nsum *acc = (nsum *)calloc((size_t)N + 1, sizeof(nsum));
    uint64_t n = (uint64_t)1 << N;
    for (uint64_t b = 0; b < n; ++b) {
        int U = 0;
        for (int t = 1; t <= N; ++t) U += (int)((b >> (N - t)) & 1u);
        nsum_add(&acc[U], orc_path_prob(m, b));
    }
    for (int i = 0; i <= N; ++i) out[i] = nsum_get(&acc[i]);
    free(acc);
}

/* eq. f8: V = e^{-qT} sum_i C(N,i) p^i (1-p)^{N-i} V_{Ni}, V_{Ni} from the
 * Algorithm 1 leaf prices. */
double orc_price_european_closed(const orc_model *m) {
    int N = m->N;
    nsum acc = {0.0, 0.0};
    double c = 1.0; /* C(N,i), exact in double for N <= 60; via lgamma beyond */
    for (int i = 0; i <= N; ++i) {
        if (i > 0) c = c * (double)(N - i + 1) / (double)i;
        double S = m->S0 * pow(m->u, (double)i) * pow(m->d, (double)(N - i));
        double pr;
        if (N <= 60) pr = c * pow(m->p, (double)i) * pow(1.0 - m->p, (double)(N - i));
        else pr = exp(lgamma((double)N + 1.0) - lgamma((double)i + 1.0) - lgamma((double)(N - i) + 1.0) +
                      (double)i * log(m->p) + (double)(N - i) * log1p(-m->p));
        nsum_add(&acc, pr * payoff_of(m->payoff, m->K, S));
    }
    return m->disc * nsum_get(&acc);
}

/* Backward induction on the Algorithm 1 grid: E_i[j] = p E_{i+1}[j+1] + (1-p) E_{i+1}[j],
 * then discount the root by e^{-qT}. */
double orc_price_european_backward(const orc_model *m) {
    int N = m->N;
    double *E = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    for (int j = 0; j <= N; ++j) {
        double S = m->S0 * pow(m->u, (double)j) * pow(m->d, (double)(N - j));
        E[j] = payoff_of(m->payoff, m->K, S);
    }
    for (int i = N - 1; i >= 0; --i)
        for (int j = 0; j <= i; ++j) E[j] = m->p * E[j + 1] + (1.0 - m->p) * E[j];
    double v = m->disc * E[0];
    free(E);
    return v;
}

/* Geometric Asian: sum_{t=1}^N ln S_t = N ln S0 + W ln u + (N(N+1)/2 - W) ln d with
 * W = sum_t U_t, so the payoff depends on the path only through W. The DP
 * carries the probability mass of (U_t, W_t) forward one step at a time. */
double orc_price_geometric_dp(const orc_model *m) {
    int N = m->N;
    if (m->payoff != ORC_GEO_CALL && m->payoff != ORC_GEO_PUT) return NAN;
    int Wmax = N * (N + 1) / 2;
    size_t sz = (size_t)(N + 1) * (size_t)(Wmax + 1);
    double *cur = (double *)calloc(sz, sizeof(double));
    double *nxt = (double *)calloc(sz, sizeof(double));
    cur[0] = 1.0; /* t = 0: U = 0, W = 0 */
    for (int t = 0; t < N; ++t) {
        memset(nxt, 0, sz * sizeof(double));
        int wt = t * (t + 1) / 2;
        for (int k = 0; k <= t; ++k)
            for (int W = 0; W <= wt; ++W) {
                double pm = cur[(size_t)k * (Wmax + 1) + W];
                if (pm == 0.0) continue;
                nxt[(size_t)(k + 1) * (Wmax + 1) + W + k + 1] += pm * m->p;   /* up */
                nxt[(size_t)k * (Wmax + 1) + W + k] += pm * (1.0 - m->p);     /* down */
            }
        double *tmp = cur; cur = nxt; nxt = tmp;
    }
    double lu = log(m->u), ld = log(m->d), ls = log(m->S0);
    nsum acc = {0.0, 0.0};
    for (int k = 0; k <= N; ++k)
        for (int W = 0; W <= Wmax; ++W) {
            double pm = cur[(size_t)k * (Wmax + 1) + W];
            if (pm == 0.0) continue;
            double lg = ls + ((double)W * lu + (double)(Wmax - W) * ld) / (double)N;
            nsum_add(&acc, pm * payoff_of(m->payoff, m->K, exp(lg)));
        }
    free(cur); free(nxt);
    return m->disc * nsum_get(&acc);
}

/* Fixed-strike lookback with ud = 1 (A1): S_t = S0 u^{l_t}, l_t = 2U_t - t.
 * The DP carries the mass of (l_t, running extreme level over t' = 1..t). */
double orc_price_lookback_dp(const orc_model *m) {
    int N = m->N;
    if (m->payoff != ORC_LOOK_CALL && m->payoff != ORC_LOOK_PUT) return NAN;
    if (fabs(m->u * m->d - 1.0) > 1e-12) return NAN;
    int is_call = (m->payoff == ORC_LOOK_CALL);
    int W = 2 * N + 1; /* levels -N..N */
    size_t sz = (size_t)W * (size_t)W;
    double *cur = (double *)calloc(sz, sizeof(double));
    double *nxt = (double *)calloc(sz, sizeof(double));
#define IDX(l, e) ((size_t)((l) + N) * (size_t)W + (size_t)((e) + N))
    /* t = 1: the running extreme starts at S_1 (S_0 is excluded). */
    cur[IDX(1, 1)] = m->p;
    cur[IDX(-1, -1)] = 1.0 - m->p;
    for (int t = 1; t < N; ++t) {
        memset(nxt, 0, sz * sizeof(double));
        for (int l = -t; l <= t; ++l)
            for (int e = -t; e <= t; ++e) {
                double pm = cur[IDX(l, e)];
                if (pm == 0.0) continue;
                int lu = l + 1, ld = l - 1;
                int eu = is_call ? (e > lu ? e : lu) : (e < lu ? e : lu);
                int ed = is_call ? (e > ld ? e : ld) : (e < ld ? e : ld);
                nxt[IDX(lu, eu)] += pm * m->p;
                nxt[IDX(ld, ed)] += pm * (1.0 - m->p);
            }
        double *tmp = cur; cur = nxt; nxt = tmp;
    }
    nsum acc = {0.0, 0.0};
    for (int l = -N; l <= N; ++l)
        for (int e = -N; e <= N; ++e) {
            double pm = cur[IDX(l, e)];
            if (pm == 0.0) continue;
            double X = m->S0 * pow(m->u, (double)e);
            nsum_add(&acc, pm * payoff_of(m->payoff, m->K, X));
        }
#undef IDX
    free(cur); free(nxt);
    return m->disc * nsum_get(&acc);
}

/* ------------------------------------------------------------------------ */
/* Meet in the middle for the arithmetic Asian                               */
/* ------------------------------------------------------------------------ */
typedef struct { double f, w; } fw_t;
static int fw_cmp(const void *a, const void *b) {
    double x = ((const fw_t *)a)->f, y = ((const fw_t *)b)->f;
    return (x > y) - (x < y);
}

/* A = (Sigma_P + S_P f_s) / N with Sigma_P = sum_{t<=P} S_t and f_s the sum of
 * the last L prices relative to S_P. The payoff is max(a + b f_s, 0) (call) with
 * a = Sigma_P/N - K, b = S_P/N > 0, so a prefix is in the money exactly on the
 * suffixes with f_s above -a/b. */
double orc_price_asian_mitm(const orc_model *m, int L) {
    int N = m->N;
    if (m->payoff != ORC_ARITH_CALL && m->payoff != ORC_ARITH_PUT) return NAN;
    if (L < 1 || L > N || L > 26) return NAN;
    int P = N - L;
    int is_call = (m->payoff == ORC_ARITH_CALL);
    size_t ns = (size_t)1 << L;
    fw_t *suf = (fw_t *)malloc(sizeof(fw_t) * ns);
    /* relative price after j suffix steps with k ups: u^k d^{j-k} */
    double *rel = (double *)malloc(sizeof(double) * (size_t)(L + 1) * (size_t)(L + 1));
    for (int j = 0; j <= L; ++j)
        for (int k = 0; k <= j; ++k) rel[j * (L + 1) + k] = pow(m->u, (double)k) * pow(m->d, (double)(j - k));
    for (size_t s = 0; s < ns; ++s) {
        int k = 0; double f = 0.0;
        for (int j = 1; j <= L; ++j) {
            k += (int)((s >> (L - j)) & 1u);
            f += rel[j * (L + 1) + k];
        }
        suf[s].f = f;
        suf[s].w = pow(m->p, (double)k) * pow(1.0 - m->p, (double)(L - k));
    }
    qsort(suf, ns, sizeof(fw_t), fw_cmp);
    /* lower cumulative sums: lowW[i] = sum_{s<i} w_s, lowF[i] = sum_{s<i} w_s f_s */
    dd *lowW = (dd *)malloc(sizeof(dd) * (ns + 1));
    dd *lowF = (dd *)malloc(sizeof(dd) * (ns + 1));
    lowW[0] = dd_from(0.0); lowF[0] = dd_from(0.0);
    for (size_t i = 0; i < ns; ++i) {
        lowW[i + 1] = dd_add(lowW[i], dd_from(suf[i].w));
        dd wf; double pr = suf[i].w * suf[i].f; wf.hi = pr; wf.lo = fma(suf[i].w, suf[i].f, -pr);
        lowF[i + 1] = dd_add(lowF[i], wf);
    }
    dd totW = lowW[ns], totF = lowF[ns];
    dd total = dd_from(0.0);
    size_t np = (size_t)1 << P;
    for (size_t q = 0; q < np; ++q) {
        int k = 0; double SP = m->S0, sig = 0.0;
        for (int t = 1; t <= P; ++t) {
            k += (int)((q >> (P - t)) & 1u);
            SP = m->S0 * pow(m->u, (double)k) * pow(m->d, (double)(t - k));
            sig += SP;
        }
        double a = sig / (double)N - m->K, b = SP / (double)N;
        double wp = pow(m->p, (double)k) * pow(1.0 - m->p, (double)(P - k));
        double theta = -a / b;
        dd part;
        if (is_call) {
            /* first index with f > theta */
            size_t lo = 0, hi = ns;
            while (lo < hi) { size_t mid = (lo + hi) / 2; if (suf[mid].f > theta) hi = mid; else lo = mid + 1; }
            dd W = dd_add(totW, dd_mul_d(lowW[lo], -1.0));
            dd F = dd_add(totF, dd_mul_d(lowF[lo], -1.0));
            part = dd_add(dd_mul_d(W, a), dd_mul_d(F, b));
        } else {
            /* first index with f >= theta: suffixes below it are in the money */
            size_t lo = 0, hi = ns;
            while (lo < hi) { size_t mid = (lo + hi) / 2; if (suf[mid].f >= theta) hi = mid; else lo = mid + 1; }
            part = dd_add(dd_mul_d(lowW[lo], -a), dd_mul_d(lowF[lo], -b));
        }
        total = dd_add(total, dd_mul_d(part, wp));
    }
    free(suf); free(rel); free(lowW); free(lowF);
    return m->disc * dd_get(total);
}

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon et al., SC'11)                                     */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u; /* Weyl key schedule */
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

uint64_t orc_bernoulli_threshold(double p) {
    double x = floor(p * 4294967296.0 + 0.5);
    if (x < 1.0) x = 1.0;
    if (x > 4294967295.0) x = 4294967295.0;
    return (uint64_t)x;
}

/* State of a path after some steps: enough to finish any payoff. */
typedef struct { int t, U; double S, sum, lsum, mx, mn; } pstate;

static void pstate_step(const orc_model *m, const grid_t *g, pstate *s, int x) {
    s->t += 1; s->U += x;
    double St = g->S[s->t * (m->N + 1) + s->U];
    s->S = St; s->sum += St; s->lsum += g->lnS[s->t * (m->N + 1) + s->U];
    if (St > s->mx) s->mx = St;
    if (St < s->mn) s->mn = St;
}
static double pstate_payoff(const orc_model *m, const pstate *s) {
    double X;
    switch (m->payoff) {
    case ORC_EURO_CALL: case ORC_EURO_PUT: X = s->S; break;
    case ORC_ARITH_CALL: case ORC_ARITH_PUT: X = s->sum / (double)m->N; break;
    case ORC_GEO_CALL: case ORC_GEO_PUT: X = exp(s->lsum / (double)m->N); break;
    case ORC_LOOK_CALL: X = s->mx; break;
    default: X = s->mn; break;
    }
    return payoff_of(m->payoff, m->K, X);
}
static void prefix_state(const orc_model *m, const grid_t *g, int mb, uint64_t z, pstate *s) {
    s->t = 0; s->U = 0; s->S = m->S0; s->sum = 0.0; s->lsum = 0.0; s->mx = -INFINITY; s->mn = INFINITY;
    for (int t = 1; t <= mb; ++t) pstate_step(m, g, s, (int)((z >> (mb - t)) & 1u));
}

/* One Monte Carlo draw: finish the path from the stratum's prefix state. */
static double mc_draw(const orc_model *m, const grid_t *g, const pstate *pre, int mb, uint64_t thr,
                      uint32_t i, uint32_t c2, uint32_t stream, const uint32_t key[2]) {
    pstate s = *pre;
    uint32_t blk[4];
    for (int t = mb + 1; t <= m->N; ++t) {
        uint32_t j = (uint32_t)(t - mb - 1);
        if ((j & 3u) == 0u) {
            uint32_t ctr[4] = {j >> 2, i, c2, stream};
            orc_philox4x32_10(ctr, key, blk);
        }
        int x = (uint64_t)blk[j & 3u] < thr;
        pstate_step(m, g, &s, x);
    }
    return pstate_payoff(m, &s);
}

/* Section 4. Partitioned MC: theta_s = sum_m theta_hat^{(m)} P(D_m) (eq. mc12); the
 * variance of the estimator is sum_m P(D_m)^2 Var[V|D_m] / R_m, estimated with the
 * unbiased per-stratum sample variance. Shared-Sample MC (Remark, eq. mc16):
 * theta_tilde = (1/R) sum_i sum_m V(z_m, y_i) P(D_m). */
void orc_mc(const orc_model *m, int mb, int64_t Rm, uint64_t seed, uint32_t stream, int shared,
            double *theta, double *var, double *stratum_mean, double *stratum_var, double *stratum_prob) {
    grid_t g;
    if (mb < 0 || mb > m->N || mb > 24 || Rm < 1 || grid_make(m, &g)) { *theta = NAN; *var = NAN; return; }
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint64_t thr = orc_bernoulli_threshold(m->p);
    int64_t M = (int64_t)1 << mb;
    pstate *pre = (pstate *)malloc(sizeof(pstate) * (size_t)M);
    double *prob = (double *)malloc(sizeof(double) * (size_t)M);
    for (int64_t z = 0; z < M; ++z) {
        prefix_state(m, &g, mb, (uint64_t)z, &pre[z]);
        prob[z] = pow(m->p, (double)pre[z].U) * pow(1.0 - m->p, (double)(mb - pre[z].U));
    }
    if (!shared) {
        nsum th = {0.0, 0.0}, vv = {0.0, 0.0};
        for (int64_t z = 0; z < M; ++z) {
            /* Welford running mean and sum of squared deviations */
            double mean = 0.0, M2 = 0.0;
            for (int64_t i = 0; i < Rm; ++i) {
                double v = mc_draw(m, &g, &pre[z], mb, thr, (uint32_t)i, (uint32_t)z, stream, key);
                double delta = v - mean;
                mean += delta / (double)(i + 1);
                M2 += delta * (v - mean);
            }
            double s2 = Rm > 1 ? M2 / (double)(Rm - 1) : 0.0;
            if (stratum_mean) stratum_mean[z] = mean;
            if (stratum_var) stratum_var[z] = s2;
            if (stratum_prob) stratum_prob[z] = prob[z];
            nsum_add(&th, prob[z] * mean);
            nsum_add(&vv, prob[z] * prob[z] * s2 / (double)Rm);
        }
        *theta = nsum_get(&th); *var = nsum_get(&vv);
    } else {
        double mean = 0.0, M2 = 0.0;
        for (int64_t i = 0; i < Rm; ++i) {
            nsum h = {0.0, 0.0};
            for (int64_t z = 0; z < M; ++z) {
                double v = mc_draw(m, &g, &pre[z], mb, thr, (uint32_t)i, 0u, stream, key);
                nsum_add(&h, prob[z] * v);
            }
            double hv = nsum_get(&h);
            double delta = hv - mean;
            mean += delta / (double)(i + 1);
            M2 += delta * (hv - mean);
        }
        *theta = mean;
        *var = Rm > 1 ? M2 / (double)(Rm - 1) / (double)Rm : 0.0;
        if (stratum_prob) for (int64_t z = 0; z < M; ++z) stratum_prob[z] = prob[z];
    }
    free(pre); free(prob); grid_free(&g);
}

/* One stratum z of the Partitioned estimator, with the same draws as orc_mc:
 * its sample mean, unbiased sample variance and P(D_z). */
void orc_mc_stratum(const orc_model *m, int mb, uint64_t z, int64_t Rm, uint64_t seed, uint32_t stream,
                    double *mean, double *var, double *prob) {
    grid_t g;
    *mean = NAN; *var = NAN; *prob = NAN;
    if (mb < 0 || mb > m->N || mb > 24 || Rm < 1 || (z >> mb) != 0 || grid_make(m, &g)) return;
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint64_t thr = orc_bernoulli_threshold(m->p);
    pstate pre;
    prefix_state(m, &g, mb, z, &pre);
    double mu = 0.0, M2 = 0.0;
    for (int64_t i = 0; i < Rm; ++i) {
        double v = mc_draw(m, &g, &pre, mb, thr, (uint32_t)i, (uint32_t)z, stream, key);
        double delta = v - mu;
        mu += delta / (double)(i + 1);
        M2 += delta * (v - mu);
    }
    *mean = mu;
    *var = Rm > 1 ? M2 / (double)(Rm - 1) : 0.0;
    *prob = pow(m->p, (double)pre.U) * pow(1.0 - m->p, (double)(mb - pre.U));
    grid_free(&g);
}

/* Exact E[V|D_m] and Var[V|D_m] by enumerating the suffixes of every stratum. */
void orc_stratum_moments(const orc_model *m, int mb, double *mean, double *var, double *prob) {
    grid_t g;
    if (grid_make(m, &g)) return;
    int L = m->N - mb;
    uint64_t M = (uint64_t)1 << mb, ns = (uint64_t)1 << L;
    for (uint64_t z = 0; z < M; ++z) {
        pstate pre; prefix_state(m, &g, mb, z, &pre);
        prob[z] = pow(m->p, (double)pre.U) * pow(1.0 - m->p, (double)(mb - pre.U));
        nsum mu = {0.0, 0.0};
        for (uint64_t y = 0; y < ns; ++y) {
            pstate s = pre; int k = 0;
            for (int j = 1; j <= L; ++j) { int x = (int)((y >> (L - j)) & 1u); k += x; pstate_step(m, &g, &s, x); }
            double w = pow(m->p, (double)k) * pow(1.0 - m->p, (double)(L - k));
            nsum_add(&mu, w * pstate_payoff(m, &s));
        }
        double mval = nsum_get(&mu);
        nsum vs = {0.0, 0.0};
        for (uint64_t y = 0; y < ns; ++y) {
            pstate s = pre; int k = 0;
            for (int j = 1; j <= L; ++j) { int x = (int)((y >> (L - j)) & 1u); k += x; pstate_step(m, &g, &s, x); }
            double w = pow(m->p, (double)k) * pow(1.0 - m->p, (double)(L - k));
            double dv = pstate_payoff(m, &s) - mval;
            nsum_add(&vs, w * dv * dv);
        }
        mean[z] = mval; var[z] = nsum_get(&vs);
    }
    grid_free(&g);
}

/* ------------------------------------------------------------------------ */
/* Pathwise Greeks for CRR trees (not in the paper; a derivative of eq. f13)  */
/* ------------------------------------------------------------------------ */
/* V = e^{-qT} sum_x p(x; p) V_N(x; S0, u, K), u = e^{sigma sqrt(dt)}, d = 1/u,
 * p = (e^{q dt} - d)/(u - d). Differentiate every path term: the weight through
 * p, the payoff through S0, u and K (S_t = S0 u^{2U_t - t}). */
double orc_greeks_crr(int N, int payoff, double S0, double K, double rate, double sigma, double T,
                      double grad[4]) {
    orc_model m;
    if (orc_model_make(N, ORC_TREE_CRR, payoff, S0, K, rate, sigma, T, 0, 0, 0, &m)) return NAN;
    grid_t g; if (grid_make(&m, &g)) return NAN;
    double dt = T / (double)N, sq = sqrt(dt);
    double u = m.u, p = m.p, E = exp(rate * dt);
    double D = u - 1.0 / u, num = E - 1.0 / u;
    double dp_du = ((1.0 / (u * u)) * D - num * (1.0 + 1.0 / (u * u))) / (D * D);
    double dp_dr = dt * E / D;
    double du_ds = sq * u;
    int is_call = (payoff == ORC_EURO_CALL || payoff == ORC_ARITH_CALL || payoff == ORC_GEO_CALL ||
                   payoff == ORC_LOOK_CALL);
    nsum V = {0, 0}, dS = {0, 0}, dK = {0, 0}, dU = {0, 0}, dP = {0, 0};
    uint64_t n = (uint64_t)1 << N;
    for (uint64_t b = 0; b < n; ++b) {
        int U = 0; double sum = 0.0, dsum = 0.0, lsum_lvl = 0.0, St = S0;
        double mx = -INFINITY, mn = INFINITY; int lmx = 0, lmn = 0;
        double lsum = 0.0;
        for (int t = 1; t <= N; ++t) {
            U += (int)((b >> (N - t)) & 1u);
            int l = 2 * U - t;
            St = g.S[t * (N + 1) + U];
            sum += St; dsum += (double)l * St / u;
            lsum += g.lnS[t * (N + 1) + U]; lsum_lvl += (double)l;
            if (St > mx) { mx = St; lmx = l; }
            if (St < mn) { mn = St; lmn = l; }
        }
        double X, dX_du;
        switch (payoff) {
        case ORC_EURO_CALL: case ORC_EURO_PUT: X = St; dX_du = (double)(2 * U - N) * St / u; break;
        case ORC_ARITH_CALL: case ORC_ARITH_PUT: X = sum / (double)N; dX_du = dsum / (double)N; break;
        case ORC_GEO_CALL: case ORC_GEO_PUT: X = exp(lsum / (double)N); dX_du = X * lsum_lvl / ((double)N * u); break;
        case ORC_LOOK_CALL: X = mx; dX_du = (double)lmx * mx / u; break;
        default: X = mn; dX_du = (double)lmn * mn / u; break;
        }
        double pay = payoff_of(payoff, K, X);
        double w = g.w[U];
        double dw_dp = w * ((double)U / p - (double)(N - U) / (1.0 - p));
        int itm = pay > 0.0;
        double sgn = is_call ? 1.0 : -1.0;
        nsum_add(&V, w * pay);
        nsum_add(&dP, dw_dp * pay);
        if (itm) {
            nsum_add(&dS, w * sgn * X / S0);
            nsum_add(&dK, w * (-sgn));
            nsum_add(&dU, w * sgn * dX_du);
        }
    }
    double disc = m.disc;
    double v = disc * nsum_get(&V);
    double dVdu = disc * nsum_get(&dU), dVdp = disc * nsum_get(&dP);
    grad[0] = disc * nsum_get(&dS);
    grad[1] = (dVdu + dVdp * dp_du) * du_ds;
    grad[2] = dVdp * dp_dr - T * v;
    grad[3] = disc * nsum_get(&dK);
    grid_free(&g);
    return v;
}

/* ------------------------------------------------------------------------ */
/* Trees given move by move: time-varying binomial trees (eq. f13 with       */
/* per-step u_t, d_t, p_t) and trees with b branches per node (end of        */
/* Section 3). One walk per path gives every payoff's quantity.              */
/* ------------------------------------------------------------------------ */
typedef struct { double SN, sum, lsum, mx, mn; } price_summary;

/* The payoff's underlying quantity from a path's prices (the definitions of
 * path_quantity above: S_N, the average, the geometric average, max, min over
 * t = 1..N). */
static double summary_quantity(int payoff, int N, const price_summary *s) {
    switch (payoff) {
    case ORC_EURO_CALL: case ORC_EURO_PUT: return s->SN;
    case ORC_ARITH_CALL: case ORC_ARITH_PUT: return s->sum / (double)N;
    case ORC_GEO_CALL: case ORC_GEO_PUT: return exp(s->lsum / (double)N);
    case ORC_LOOK_CALL: return s->mx;
    default: return s->mn;
    }
}

/* Walks one path: x[t-1] is the digit taken at step t, fac[(t-1) b + k] and
 * lnf[(t-1) b + k] the factor of digit k at step t and its logarithm,
 * prob[(t-1) b + k] its probability. S_t = S_{t-1} fac, ln S_t = ln S_{t-1} +
 * ln fac (so sum_t ln S_t needs no logarithm per step), and the path's
 * probability is the product of the probabilities of its moves. */
static double walk_moves(int N, int b, double S0, const double *fac, const double *lnf, const double *prob,
                         const int *x, price_summary *s) {
    double St = S0, lS = log(S0), w = 1.0;
    s->sum = 0.0; s->lsum = 0.0; s->mx = -INFINITY; s->mn = INFINITY;
    for (int t = 1; t <= N; ++t) {
        const int k = (t - 1) * b + x[t - 1];
        St = St * fac[k];
        lS = lS + lnf[k];
        w = w * prob[k];
        s->sum += St;
        s->lsum += lS;
        if (St > s->mx) s->mx = St;
        if (St < s->mn) s->mn = St;
    }
    s->SN = St;
    return w;
}

/* Digits of path index idx, the first step most significant (Section 3's rank
 * digits come first): x[t-1] = digit of step t in base b. */
static void path_digits(uint64_t idx, int N, int b, int *x) {
    for (int t = N; t >= 1; --t) {
        x[t - 1] = (int)(idx % (uint64_t)b);
        idx /= (uint64_t)b;
    }
}

/* A tree given move by move in one layout: b factors and b probabilities per
 * step, with the logarithms of the factors. */
typedef struct {
    int N, b;
    double S0;
    double *fac, *lnf, *prob;
} moves_t;

static int moves_from_steps(const orc_steps_model *m, moves_t *mv) {
    mv->N = m->N; mv->b = 2; mv->S0 = m->S0;
    mv->fac = (double *)malloc(sizeof(double) * 2 * (size_t)m->N);
    mv->lnf = (double *)malloc(sizeof(double) * 2 * (size_t)m->N);
    mv->prob = (double *)malloc(sizeof(double) * 2 * (size_t)m->N);
    if (!mv->fac || !mv->lnf || !mv->prob) return -1;
    for (int t = 0; t < m->N; ++t) {   /* digit 0 = down, digit 1 = up */
        mv->fac[2 * t] = m->d[t]; mv->fac[2 * t + 1] = m->u[t];
        mv->prob[2 * t] = 1.0 - m->p[t]; mv->prob[2 * t + 1] = m->p[t];
        mv->lnf[2 * t] = log(m->d[t]); mv->lnf[2 * t + 1] = log(m->u[t]);
    }
    return 0;
}

static int moves_from_branch(const orc_branch_model *m, moves_t *mv) {
    const size_t n = (size_t)m->N * (size_t)m->b;
    mv->N = m->N; mv->b = m->b; mv->S0 = m->S0;
    mv->fac = (double *)malloc(sizeof(double) * n);
    mv->lnf = (double *)malloc(sizeof(double) * n);
    mv->prob = (double *)malloc(sizeof(double) * n);
    if (!mv->fac || !mv->lnf || !mv->prob) return -1;
    for (size_t i = 0; i < n; ++i) {
        mv->fac[i] = m->f[i];
        mv->prob[i] = m->q[i];
        mv->lnf[i] = log(m->f[i]);
    }
    return 0;
}

static void moves_free(moves_t *mv) { free(mv->fac); free(mv->lnf); free(mv->prob); }

/* eq. f14 (undiscounted) for several payoffs at once: for every path index in
 * [lo, hi), in order, rebuild the path, cost it in O(N) (Listing 1's loop) and
 * add p(x) V_j(x) to accumulator j, V_j the payoff pay[j] with strike K[j]. */
static void moves_sum(const moves_t *mv, int n, const int32_t *pay, const double *K, uint64_t lo, uint64_t hi,
                      nsum *acc) {
    int x[64];
    price_summary s;
    double X[8];
    if (lo >= hi) return;
    path_digits(lo, mv->N, mv->b, x);
    for (uint64_t idx = lo; idx < hi; ++idx) {
        const double w = walk_moves(mv->N, mv->b, mv->S0, mv->fac, mv->lnf, mv->prob, x, &s);
        for (int k = 0; k < 8; ++k) X[k] = NAN;   /* each payoff kind's quantity, once per path */
        for (int j = 0; j < n; ++j) {
            if (isnan(X[pay[j]])) X[pay[j]] = summary_quantity(pay[j], mv->N, &s);
            nsum_add(&acc[j], w * payoff_of(pay[j], K[j], X[pay[j]]));
        }
        /* the next path index: add one in base b (the last step least significant) */
        for (int t = mv->N - 1; t >= 0 && ++x[t] == mv->b; --t) x[t] = 0;
    }
}

typedef struct {
    const moves_t *mv; int n; const int32_t *pay; const double *K;
    uint64_t lo, hi; nsum *acc;
} moves_worker_t;

static void *moves_worker_run(void *arg) {
    moves_worker_t *w = (moves_worker_t *)arg;
    for (int j = 0; j < w->n; ++j) { w->acc[j].s = 0.0; w->acc[j].c = 0.0; }
    moves_sum(w->mv, w->n, w->pay, w->K, w->lo, w->hi, w->acc);
    return NULL;
}

/* Section 3's partition: the b^N path indices split into M contiguous ranges
 * (for M a power of b, rank m owns the paths whose leading digits are m's),
 * partial sums added in rank order (eq. f15). out[j] = disc * sum for payoff j. */
static void moves_price(const moves_t *mv, double disc, int n, const int32_t *pay, const double *K, int M,
                        double *out) {
    uint64_t total = 1;
    for (int t = 0; t < mv->N; ++t) total *= (uint64_t)mv->b;
    if (M < 1) M = 1;
    if ((uint64_t)M > total) M = (int)total;
    moves_worker_t *ws = (moves_worker_t *)calloc((size_t)M, sizeof(moves_worker_t));
    nsum *accs = (nsum *)calloc((size_t)M * (size_t)n, sizeof(nsum));
    pthread_t *th = (pthread_t *)calloc((size_t)M, sizeof(pthread_t));
    int *started = (int *)calloc((size_t)M, sizeof(int));
    for (int k = 0; k < M; ++k) {
        ws[k].mv = mv; ws[k].n = n; ws[k].pay = pay; ws[k].K = K; ws[k].acc = accs + (size_t)k * n;
        ws[k].lo = (uint64_t)(((unsigned __int128)total * (unsigned)k) / (unsigned)M);
        ws[k].hi = (uint64_t)(((unsigned __int128)total * (unsigned)(k + 1)) / (unsigned)M);
        started[k] = (M > 1) && pthread_create(&th[k], NULL, moves_worker_run, &ws[k]) == 0;
        if (!started[k]) moves_worker_run(&ws[k]);
    }
    for (int k = 0; k < M; ++k)
        if (started[k]) pthread_join(th[k], NULL);
    for (int j = 0; j < n; ++j) {
        nsum tot = {0.0, 0.0};
        for (int k = 0; k < M; ++k) {      /* eq. f15 in rank order */
            nsum_add(&tot, accs[(size_t)k * n + j].s);
            nsum_add(&tot, accs[(size_t)k * n + j].c);
        }
        out[j] = disc * nsum_get(&tot);
    }
    free(ws); free(accs); free(th); free(started);
}

double orc_steps_path_payoff(const orc_steps_model *m, uint64_t b) {
    moves_t mv; int x[64]; price_summary s;
    if (m->N < 1 || m->N > 62 || moves_from_steps(m, &mv)) return NAN;
    path_digits(b, m->N, 2, x);
    walk_moves(m->N, 2, m->S0, mv.fac, mv.lnf, mv.prob, x, &s);
    moves_free(&mv);
    return payoff_of(m->payoff, m->K, summary_quantity(m->payoff, m->N, &s));
}

double orc_steps_path_prob(const orc_steps_model *m, uint64_t b) {
    int N = m->N;
    double w = 1.0;
    for (int t = 1; t <= N; ++t) {
        int x = (int)((b >> (N - t)) & 1u);
        w *= x ? m->p[t - 1] : 1.0 - m->p[t - 1];
    }
    return w;
}

void orc_steps_sum_range(const orc_steps_model *m, uint64_t lo, uint64_t hi, double *sum, double *comp) {
    moves_t mv; nsum acc = {0.0, 0.0};
    const int32_t pay = m->payoff;
    if (m->N < 1 || m->N > 62 || moves_from_steps(m, &mv)) { *sum = NAN; *comp = 0.0; return; }
    moves_sum(&mv, 1, &pay, &m->K, lo, hi, &acc);
    moves_free(&mv);
    *sum = acc.s; *comp = acc.c;
}

/* Section 3: M = 2^r workers (nthreads rounded down to a power of two), worker
 * m owns B_m^N, the paths whose first r steps are m's bits. */
static int pow2_workers(int N, int nthreads) {
    int r = 0;
    while ((2 << r) <= nthreads && r + 1 <= N) ++r;
    return nthreads < 2 ? 1 : 1 << r;
}

void orc_steps_price_multi(const orc_steps_model *m, int n, const int32_t *pay, const double *K, int nthreads,
                           double *out) {
    moves_t mv;
    if (m->N < 1 || m->N > 62 || n < 1 || moves_from_steps(m, &mv)) {
        for (int j = 0; j < n; ++j) out[j] = NAN;
        return;
    }
    moves_price(&mv, m->disc, n, pay, K, pow2_workers(m->N, nthreads), out);
    moves_free(&mv);
}

double orc_steps_price(const orc_steps_model *m, int nthreads) {
    const int32_t pay = m->payoff;
    double v;
    orc_steps_price_multi(m, 1, &pay, &m->K, nthreads, &v);
    return v;
}

/* ------------------------------------------------------------------------ */
/* b-ary trees (end of Section 3)                                            */
/* ------------------------------------------------------------------------ */
static int branch_paths_ok(const orc_branch_model *m) {
    if (m->N < 1 || m->N > 62 || m->b < 2) return 0;
    uint64_t total = 1;
    for (int t = 0; t < m->N; ++t) {
        if (total > ((uint64_t)1 << 62) / (uint64_t)m->b) return 0;
        total *= (uint64_t)m->b;
    }
    return 1;
}

double orc_branch_path_payoff(const orc_branch_model *m, uint64_t idx) {
    moves_t mv; int x[64]; price_summary s;
    if (!branch_paths_ok(m) || moves_from_branch(m, &mv)) return NAN;
    path_digits(idx, m->N, m->b, x);
    walk_moves(m->N, m->b, m->S0, mv.fac, mv.lnf, mv.prob, x, &s);
    moves_free(&mv);
    return payoff_of(m->payoff, m->K, summary_quantity(m->payoff, m->N, &s));
}

double orc_branch_path_prob(const orc_branch_model *m, uint64_t idx) {
    int x[64];
    if (!branch_paths_ok(m)) return NAN;
    path_digits(idx, m->N, m->b, x);
    double w = 1.0;
    for (int t = 1; t <= m->N; ++t) w *= m->q[(t - 1) * m->b + x[t - 1]];
    return w;
}

void orc_branch_price_multi(const orc_branch_model *m, int n, const int32_t *pay, const double *K, int nthreads,
                            double *out) {
    moves_t mv;
    if (!branch_paths_ok(m) || n < 1 || moves_from_branch(m, &mv)) {
        for (int j = 0; j < n; ++j) out[j] = NAN;
        return;
    }
    moves_price(&mv, m->disc, n, pay, K, nthreads, out);
    moves_free(&mv);
}

double orc_branch_price(const orc_branch_model *m, int nthreads) {
    const int32_t pay = m->payoff;
    double v;
    orc_branch_price_multi(m, 1, &pay, &m->K, nthreads, &v);
    return v;
}

/* eq. expval: E[V(x)] = sum_x p(x) V(x) for any function V of the whole path,
 * on a tree given move by move. Paths are visited in index order (Listing 1's
 * loop); their prices and digits are handed to `fn` in blocks, and p(x) V(x)
 * is added in path order with Neumaier compensation. One thread (the
 * callback may not be reentrant). */
#define ORC_FN_BLOCK 2048
double orc_functional_price(const orc_branch_model *m, orc_payoff_fn fn, void *user) {
    moves_t mv;
    if (!branch_paths_ok(m) || !fn || moves_from_branch(m, &mv)) return NAN;
    const int N = m->N, b = m->b;
    uint64_t total = 1;
    for (int t = 0; t < N; ++t) total *= (uint64_t)b;
    double *S = (double *)malloc(sizeof(double) * ORC_FN_BLOCK * (size_t)N);
    int32_t *X = (int32_t *)malloc(sizeof(int32_t) * ORC_FN_BLOCK * (size_t)N);
    double *w = (double *)malloc(sizeof(double) * ORC_FN_BLOCK);
    double *v = (double *)malloc(sizeof(double) * ORC_FN_BLOCK);
    nsum acc = {0.0, 0.0};
    int x[64];
    for (uint64_t lo = 0; lo < total; lo += ORC_FN_BLOCK) {
        const int cnt = (int)((total - lo) < ORC_FN_BLOCK ? (total - lo) : ORC_FN_BLOCK);
        for (int i = 0; i < cnt; ++i) {
            path_digits(lo + (uint64_t)i, N, b, x);   /* path index lo + i, first step most significant */
            double St = m->S0, wi = 1.0;
            for (int t = 1; t <= N; ++t) {
                const int k = (t - 1) * b + x[t - 1];
                St = St * mv.fac[k];
                wi = wi * mv.prob[k];
                S[(size_t)i * N + t - 1] = St;
                X[(size_t)i * N + t - 1] = x[t - 1];
            }
            w[i] = wi;
        }
        fn(user, cnt, N, S, X, v);
        for (int i = 0; i < cnt; ++i) nsum_add(&acc, w[i] * v[i]);
    }
    free(S); free(X); free(w); free(v);
    moves_free(&mv);
    return m->disc * nsum_get(&acc);
}

double orc_branch_european_backward(const orc_branch_model *m) {
    /* node (t, j), j = 0..(b-1) t, price S0 u^{j - c t} with u = f[0][b-1]^{1/c} */
    const int N = m->N, b = m->b;
    const double c = 0.5 * (double)(b - 1);
    const double u = pow(m->f[b - 1], 1.0 / c);
    const int W = (b - 1) * N + 1;
    double *V = (double *)malloc(sizeof(double) * (size_t)W);
    for (int j = 0; j < W; ++j) V[j] = payoff_of(m->payoff, m->K, m->S0 * pow(u, (double)j - c * N));
    for (int t = N - 1; t >= 0; --t)
        for (int j = 0; j <= (b - 1) * t; ++j) {
            double v = 0.0;
            for (int k = 0; k < b; ++k) v += m->q[k] * V[j + k];
            V[j] = v;
        }
    double r = m->disc * V[0];
    free(V);
    return r;
}
