// The generic pass of btree_payoff.cuh instantiated for the built-in payoffs,
// for trees with b branches per node (the end of Section 3). A path walk
// keeps the running sum, log-sum (geometric payoffs only), extremes and the
// last price; param[0] = K, param[1] = the bt_payoff code.
#include <cuda_runtime.h>
#include <math.h>

#include "btree.h"
#include "btree_payoff.cuh"

struct builtin_payoff {
    struct state {
        double sum, lsum, mx, mn, S;
    };
    __device__ static state start(double S0, const double *) {
        state s;
        s.sum = 0.0;
        s.lsum = 0.0;
        s.mx = 0.0;
        s.mn = 1e300;
        s.S = S0;
        return s;
    }
    __device__ static state step(const state &s, double S, int, int, const double *p) {
        const int pay = (int)p[1];
        state r;
        r.sum = s.sum + S;
        r.lsum = (pay == BT_ASIAN_GEO_CALL || pay == BT_ASIAN_GEO_PUT) ? s.lsum + log(S) : 0.0;
        r.mx = fmax(s.mx, S);
        r.mn = fmin(s.mn, S);
        r.S = S;
        return r;
    }
    __device__ static double value(const state &s, int N, const double *p) {
        const int pay = (int)p[1];
        double X;
        switch (pay) {
        case BT_EURO_CALL: case BT_EURO_PUT: X = s.S; break;
        case BT_ASIAN_ARITH_CALL: case BT_ASIAN_ARITH_PUT: X = s.sum / (double)N; break;
        case BT_ASIAN_GEO_CALL: case BT_ASIAN_GEO_PUT: X = exp(s.lsum / (double)N); break;
        case BT_LOOKBACK_FIXED_CALL: X = s.mx; break;
        default: X = s.mn; break;
        }
        return (pay & 1) ? fmax(p[0] - X, 0.0) : fmax(X - p[0], 0.0);
    }
};

extern "C" __global__ void __launch_bounds__(BTP_THREADS) k_branch_builtin(btp::args a) {
    btp::run<builtin_payoff>(a);
}

extern "C" int bt_branch_builtin_grid(int device) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_branch_builtin, BTP_THREADS, 0);
    return sms * (per < 1 ? 1 : per);
}

extern "C" int bt_launch_branch_builtin(const btp::args *a, int grid, void *stream) {
    k_branch_builtin<<<grid, BTP_THREADS, 0, (cudaStream_t)stream>>>(*a);
    return (int)cudaGetLastError();
}
