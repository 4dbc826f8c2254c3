// Device pieces shared by the exhaustive kernels (exact.cu, steps.cu): the
// work-item loop, the block reduction and the FP32 per-prefix scaling.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "bt_internal.h"
#include "df.cuh"

struct __align__(16) smem_job {
    bt_job J;
    bt_jparams P;
    int64_t item;
    int job;
};

__device__ static int find_job(const bt_job *jobs, int n_jobs, int64_t item) {
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].item_begin <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Deterministic block sum of two doubles; result valid in thread 0.
__device__ __forceinline__ double2 block_sum2(double x, double y, double2 *red) {
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_down_sync(0xffffffffu, x, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) red[w] = make_double2(x, y);
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    if (threadIdx.x == 0) {
        for (int i = 0; i < BT_THREADS / 32; ++i) {
            r.x += red[i].x;
            r.y += red[i].y;
        }
    }
    return r;
}

// Loads the next work item and (if it changed) its job into shared memory.
// Returns false when the run has no items left.
template <typename SufT>
__device__ __forceinline__ bool next_item(const bt_exact_args &a, smem_job &sj, SufT *s_suf, const SufT *g_suf,
                                          int &cur_job) {
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long i = atomicAdd(a.counter, 1ull);
        sj.item = (i < (unsigned long long)a.n_run_items) ? (int64_t)a.shard + (int64_t)i * a.n_shards : -1;
        if (sj.item >= 0) sj.job = find_job(a.jobs, a.n_jobs, sj.item);
    }
    __syncthreads();
    if (sj.item < 0) return false;
    if (sj.job != cur_job) {
        cur_job = sj.job;
        if (threadIdx.x == 0) {
            sj.J = a.jobs[cur_job];
            sj.P = a.prm[sj.J.prm_off];
        }
        __syncthreads();
        const SufT *src = g_suf + sj.J.off_suf;
        for (int i = threadIdx.x; i < sj.J.suf_len; i += BT_THREADS) s_suf[i] = src[i];
        __syncthreads();
    }
    return true;
}

// The FP32 per-prefix scale of the rounding design (exact.cu header):
// lambda = 2^-e (256 - h)/256 with 2^e bounding |tau + f| over [fmin, fmax]
// and h a 7-bit hash of the prefix index q; A = lambda tau split into A_hi on
// the grid 2^(gexp - e - 8) (so lambda f_hi + A_hi is exact for f_hi on the
// grid 2^gexp) and the remainder, stored negated; 1/lambda as an FP32 pair.
struct scale32 {
    float B, Ah, nAl;
    df32 rinv;
};
__device__ __forceinline__ scale32 scale_prefix(const df32 &tau, const bt_jparams &P, int64_t q) {
    scale32 r;
    float m1 = fabsf(__fadd_rn(tau.hi, P.fmin_f)), m2 = fabsf(__fadd_rn(tau.hi, P.fmax_f));
    float mmax = fmaxf(m1, m2) * (1.0f + 0x1p-10f);
    int e = ((__float_as_int(mmax) >> 23) & 0xff) - 126;  // mmax < 2^e
    e = max(-120, min(120, e));
    const unsigned hd = ((unsigned)q * 0x9E3779B1u) >> 25;        // 7-bit dither
    const float lam = ldexpf((float)(256u - hd) * 0x1p-8f, -e);    // 9-bit mantissa, exact
    r.B = lam;
    const df32 A = df_mul_f(tau, lam);
    const int gq = P.gexp - e - 8;
    const float Ah = ldexpf(rintf(ldexpf(A.hi, -gq)), gq);
    r.Ah = Ah;
    r.nAl = -__fadd_rn(__fsub_rn(A.hi, Ah), A.lo);
    // 1/lambda: r0 = rcp, correction from the exact residual 1 - lam r0
    const float r0 = 1.0f / lam;
    const float res = __fmaf_rn(-lam, r0, 1.0f);
    r.rinv = fast_two_sum(r0, r0 * res);
    return r;
}
