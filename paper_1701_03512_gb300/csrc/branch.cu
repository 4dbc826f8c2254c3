// The generic pass of btree_payoff.cuh instantiated for the built-in payoffs,
// for trees with b branches per node (the end of Section 3). A path walk
// keeps the last price and the one running quantity the payoff needs (sum,
// log-sum or extreme); param[0] = K, param[1] = the bt_payoff code,
// param[2] = 1/N.
#include <cuda_runtime.h>
#include <math.h>

#include "btree.h"
#include "btree_payoff.cuh"

struct builtin_payoff {
    struct state {
        double acc, S;  // running sum, log-sum or extreme (by payoff); the last price
    };
    __device__ static state start(double S0, const double *p) {
        const int pay = (int)p[1];
        state s;
        s.acc = pay == BT_LOOKBACK_FIXED_PUT ? 1e300 : 0.0;
        s.S = S0;
        return s;
    }
    // one update of the quantity the payoff needs (the payoff is the same for
    // the whole work item, so the branch is uniform)
    __device__ static state step(const state &s, double S, int, int, const double *p) {
        const int pay = (int)p[1];
        state r;
        r.S = S;
        switch (pay) {
        case BT_ASIAN_ARITH_CALL: case BT_ASIAN_ARITH_PUT: r.acc = s.acc + S; break;
        case BT_ASIAN_GEO_CALL: case BT_ASIAN_GEO_PUT: r.acc = s.acc + log(S); break;
        case BT_LOOKBACK_FIXED_CALL: r.acc = fmax(s.acc, S); break;
        case BT_LOOKBACK_FIXED_PUT: r.acc = fmin(s.acc, S); break;
        default: r.acc = 0.0; break;
        }
        return r;
    }
    // param[2] = 1/N
    __device__ static double value(const state &s, int, const double *p) {
        const int pay = (int)p[1];
        double X;
        switch (pay) {
        case BT_EURO_CALL: case BT_EURO_PUT: X = s.S; break;
        case BT_ASIAN_ARITH_CALL: case BT_ASIAN_ARITH_PUT: X = s.acc * p[2]; break;
        case BT_ASIAN_GEO_CALL: case BT_ASIAN_GEO_PUT: X = exp(s.acc * p[2]); break;
        default: X = s.acc; break;
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
