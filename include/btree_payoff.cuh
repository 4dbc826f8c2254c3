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
 * with x_t the move of step t (a digit 0..b-1 in a tree with b branches per
 * node; 1 = up, 0 = down in a binomial tree), S_t the price after it, and
 * param the option's eight user parameters. A functional of the moves alone
 * (the general V of eq. expval) ignores S.
 * It is compiled either into the caller's own CUDA code (instantiate
 * btp::run<Payoff> in a kernel) or at run time from source with
 * bt_plugin_compile (btree.h), which appends the plug-in source to this
 * header and builds it for the current GPU.
 *
 * The pass: a path is N digits in base b, the first step the most
 * significant (the leading digits are Section 3's partition); its index
 * splits into P = N - L prefix steps and L suffix steps, b^L <= 4096. A work
 * item is 256 prefixes, one per thread; a thread walks its prefix once, then
 * visits its b^L suffixes in order as a depth-first walk (an odometer over
 * the suffix digits) that keeps the state of every level, so consecutive
 * suffixes share their common first steps and a path costs about
 * b/(b-1) state steps. Weights and the sum are FP64; the block's sum goes to
 * one partial per work item, in a fixed order. This header has no includes:
 * it is also the source that the run-time compiler sees. */
#ifndef BTREE_PAYOFF_CUH
#define BTREE_PAYOFF_CUH

namespace btp {

#define BTP_MAX_L 12
#define BTP_THREADS 256
#define BTP_PARAMS 8

struct job {
    int N, L, P, b;                 /* steps, suffix and prefix steps, branches */
    long long item_begin, n_items;  /* items of this option: ceil(b^P / 256) */
    long long n_prefixes, n_leaves; /* b^P, b^L */
    const double *moves;            /* device: step t at 2b (t-1): factor of digit 0..b-1,
                                       then the probability of digit 0..b-1 */
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
        if (q < J.n_prefixes) {
            const int b = J.b;
            /* prefix walk: steps 1..P, the most significant digit first */
            double S = J.S0, w = 1.0;
            state st = Payoff::start(J.S0, J.param);
            long long place = J.n_prefixes / b;
            for (int t = 1; t <= J.P; ++t, place /= b) {
                const int x = (int)((q / place) % b);
                const double *mv = J.moves + 2 * b * (t - 1);
                S *= mv[x];
                w *= mv[b + x];
                st = Payoff::step(st, S, t, x, J.param);
            }
            /* suffix leaves in order; level d holds the state after d suffix steps */
            state ss[BTP_MAX_L + 1];
            double sS[BTP_MAX_L + 1], sw[BTP_MAX_L + 1];
            int dig[BTP_MAX_L];
            ss[0] = st;
            sS[0] = S;
            sw[0] = w;
            const int L = J.L;
            for (int d = 0; d < L; ++d) dig[d] = 0;
            for (long long s = 0; s < J.n_leaves; ++s) {
                /* advance the odometer; d0 is the first suffix step that changed */
                int d0 = 0;
                if (s > 0) {
                    d0 = L - 1;
                    while (dig[d0] == b - 1) dig[d0--] = 0;
                    ++dig[d0];
                }
                for (int d = d0; d < L; ++d) {
                    const int x = dig[d];
                    const int t = J.P + d + 1;
                    const double *mv = J.moves + 2 * b * (t - 1);
                    sS[d + 1] = sS[d] * mv[x];
                    sw[d + 1] = sw[d] * mv[b + x];
                    ss[d + 1] = Payoff::step(ss[d], sS[d + 1], t, x, J.param);
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
