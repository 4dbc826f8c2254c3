/* Payoff plug-ins for the exhaustive expected value over Bernoulli paths.
 *
 * The paper's object is the expected value of a function of the whole path,
 * E V(X) = sum over x in {0,1}^N of p(x) V(x) (eq. expval; eq. f13 for
 * option payoffs). The built-in passes of libbtree reduce their eight payoffs
 * to an affine form in one per-suffix number; a plug-in instead supplies any
 * V as a small state machine along the path, and this generic pass evaluates
 * it on every path.
 *
 * A plug-in is a struct named Payoff with
 *
 *     struct state { ... };                               // trivially copyable
 *     __device__ static state start(double S0, const double *param);
 *     __device__ static state step(const state &s, double S, int t, int x, const double *param);
 *     __device__ static double value(const state &s, int N, const double *param);
 *
 * so that V(x) = value(step(...step(start(S0), S_1, 1, x_1)..., S_N, N, x_N))
 * with x_t the move of step t (1 = up), S_t the price after it, and param the
 * option's eight user parameters. A functional of the bits alone (the
 * general V of eq. expval) ignores S.
 * It is compiled either into the caller's own CUDA code (instantiate
 * btp::run<Payoff> in a kernel) or at run time from source with
 * bt_plugin_compile (btree.h), which appends the plug-in source to this
 * header and builds it for the current GPU.
 *
 * The pass: an option's path index splits into P = N - L prefix steps and
 * L = min(N, 12) suffix steps. A work item is 256 prefixes, one per thread;
 * a thread walks its prefix once, then visits its 2^L suffixes in order as a
 * depth-first walk that keeps the state of every level, so consecutive
 * suffixes share their common first steps and a path costs two state steps
 * on average. Weights and the sum are FP64; the block's sum goes to one
 * partial per work item, in a fixed order. This header has no includes: it
 * is also the source that the run-time compiler sees. */
#ifndef BTREE_PAYOFF_CUH
#define BTREE_PAYOFF_CUH

namespace btp {

#define BTP_MAX_L 12
#define BTP_THREADS 256
#define BTP_PARAMS 8

struct job {
    int N, L, P, pad;
    long long item_begin, n_items;  /* items of this option: ceil(2^P / 256) */
    const double *steps;            /* device: (u_t, d_t, p_t) for t = 1..N */
    double S0;
    double param[BTP_PARAMS];
};

struct args {
    const job *jobs;
    int n_jobs, pad;
    long long n_items;              /* all options */
    double *partials;               /* one per work item */
    unsigned long long *counter;    /* zero before the launch */
};

template <class Payoff>
__device__ void run(const args &a) {
    typedef typename Payoff::state state;
    __shared__ double red[BTP_THREADS / 32];
    __shared__ long long s_item;
    __shared__ int s_job;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned long long i = atomicAdd(a.counter, 1ull);
            s_item = i < (unsigned long long)a.n_items ? (long long)i : -1;
            if (s_item >= 0) {
                int lo = 0, hi = a.n_jobs - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (a.jobs[mid].item_begin <= s_item) lo = mid;
                    else hi = mid - 1;
                }
                s_job = lo;
            }
        }
        __syncthreads();
        if (s_item < 0) return;
        const job &J = a.jobs[s_job];
        const long long item = s_item - J.item_begin;
        const long long q = item * BTP_THREADS + threadIdx.x;  /* this thread's prefix */
        double acc = 0.0;
        if (q < (1ll << J.P)) {
            /* prefix walk: steps 1..P, the most significant bit first */
            double S = J.S0, w = 1.0;
            state st = Payoff::start(J.S0, J.param);
            for (int t = 1; t <= J.P; ++t) {
                const bool up = (q >> (J.P - t)) & 1;
                const double *f = J.steps + 3 * (t - 1);
                S *= up ? f[0] : f[1];
                w *= up ? f[2] : 1.0 - f[2];
                st = Payoff::step(st, S, t, up, J.param);
            }
            /* suffix leaves in order; level d holds the state after d suffix steps */
            state ss[BTP_MAX_L + 1];
            double sS[BTP_MAX_L + 1], sw[BTP_MAX_L + 1];
            ss[0] = st;
            sS[0] = S;
            sw[0] = w;
            const int L = J.L;
            const long long n_leaves = 1ll << L;
            for (long long s = 0; s < n_leaves; ++s) {
                /* the first suffix step that differs from the previous leaf */
                const int d0 = s == 0 ? 0 : L - 1 - __ffsll(s) + 1;
                for (int d = d0; d < L; ++d) {
                    const bool up = (s >> (L - 1 - d)) & 1;
                    const int t = J.P + d + 1;
                    const double *f = J.steps + 3 * (t - 1);
                    sS[d + 1] = sS[d] * (up ? f[0] : f[1]);
                    sw[d + 1] = sw[d] * (up ? f[2] : 1.0 - f[2]);
                    ss[d + 1] = Payoff::step(ss[d], sS[d + 1], t, up, J.param);
                }
                acc = fma(sw[L], Payoff::value(ss[L], J.N, J.param), acc);
            }
        }
        /* block sum in a fixed order */
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int i = 0; i < BTP_THREADS / 32; ++i) t += red[i];
            a.partials[J.item_begin + item] = t;
        }
    }
}

}  // namespace btp

#endif
