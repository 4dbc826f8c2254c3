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

// Loads the next work item and (if it changed) its job into shared memory; `load(J)` copies
// the job's suffix table (all threads take part). Returns false when the run has no items left.
template <typename Load>
__device__ __forceinline__ bool next_item_with(const bt_exact_args &a, smem_job &sj, int &cur_job, Load load) {
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
        load(sj.J);
        __syncthreads();
    }
    return true;
}

// The same with the suffix table copied entry by entry.
template <typename SufT>
__device__ __forceinline__ bool next_item(const bt_exact_args &a, smem_job &sj, SufT *s_suf, const SufT *g_suf,
                                          int &cur_job) {
    return next_item_with(a, sj, cur_job, [&](const bt_job &J) {
        const SufT *src = g_suf + J.off_suf;
        for (int i = threadIdx.x; i < J.suf_len; i += BT_THREADS) s_suf[i] = src[i];
    });
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

// ---------------------------------------------------------------------------
// Per-prefix state of the lattice passes (exact.cu, greeks.cu)
// ---------------------------------------------------------------------------
__device__ __forceinline__ df32 pw2(const bt_pow *t, int e) {
    bt_pow v = t[e];
    return df_make(v.hi, v.lo);
}

struct pref32 {
    float B, Ah, nAl;
    df32 om;   // w_low * beta * 2^e
    df32 cst;  // w_low * C (lookback)
};

// Per-prefix affine form of the payoff in the suffix factor f:
// payoff = beta * max(+-(tau + f), 0) + C, with tau, beta, C as FP32 pairs.
struct pstate {
    df32 tau, beta, cst;
};
__device__ __forceinline__ pstate prefix_state(const bt_job &J, const bt_jparams &P, const bt_exact_args &a,
                                               int64_t q) {
    const int64_t h = q >> J.M;
    const int m = (int)(q & ((1ll << J.M) - 1));
    const bt_pentry eh = a.ph[J.off_ph + h];
    const bt_pentry em = a.pm[J.off_pm + m];
    const int lvl = eh.lvl + em.lvl;
    const bt_pow *pw = a.pw + J.off_pow + J.N + 1;
    df32 tau, beta, cst = df_make(0.0f, 0.0f);
    switch (J.field) {
    case BT_F_ARITH: {
        // tau = Sigma_P / S_P - N K / S_P, Sigma_P / S_P = u^{-Delta_m} R_h + R_m
        df32 Rp = df_add(df_mul(pw2(pw, -em.lvl), df_make(eh.R_hi, eh.R_lo)), df_make(em.R_hi, em.R_lo));
        df32 X = df_mul(df_from2(P.NKoS0_2), pw2(pw, -lvl));
        tau = df_sub(Rp, X);
        beta = df_mul(df_from2(P.S0oN_2), pw2(pw, lvl));
        break;
    }
    case BT_F_EURO:
        tau = df_neg(df_mul(df_from2(P.KoS0_2), pw2(pw, -lvl)));
        beta = df_mul(df_from2(P.S0_2), pw2(pw, lvl));
        break;
    case BT_F_GEO: {
        const int I = (int)eh.D + J.M * (int)eh.lvl + (int)em.D + J.L * lvl;
        const bt_pow *g = a.pw + J.off_geo - J.geo_imin;
        tau = df_neg(df_mul(df_from2(P.KoS0_2), pw2(g, -I)));
        beta = df_mul(df_from2(P.S0_2), pw2(g, I));
        break;
    }
    case BT_F_LOOKMAX: {
        const int lam = max((int)eh.mx, (int)eh.lvl + (int)em.mx);
        df32 kk = df_mul(df_from2(P.KoS0_2), pw2(pw, -lvl));
        if (lam > -BT_LVL_NONE / 2) {
            // tau = -max(M_P, K) / S_P,  C = max(M_P - K, 0)
            df32 rr = pw2(pw, lam - lvl);
            tau = df_neg(df_gt(rr, kk) ? rr : kk);
            df32 c = df_sub(df_mul(df_from2(P.S0_2), pw2(pw, lam)), df_from2(P.K_2));
            if (c.hi > 0.0f) cst = c;
        } else {
            tau = df_neg(kk);
        }
        beta = df_mul(df_from2(P.S0_2), pw2(pw, lvl));
        break;
    }
    default: {  // BT_F_LOOKMIN
        const int lam = min((int)eh.mn, (int)eh.lvl + (int)em.mn);
        df32 kk = df_mul(df_from2(P.KoS0_2), pw2(pw, -lvl));
        if (lam < BT_LVL_NONE / 2) {
            // tau = -min(m_P, K) / S_P,  C = max(K - m_P, 0)
            df32 rr = pw2(pw, lam - lvl);
            tau = df_neg(df_gt(rr, kk) ? kk : rr);
            df32 c = df_sub(df_from2(P.K_2), df_mul(df_from2(P.S0_2), pw2(pw, lam)));
            if (c.hi > 0.0f) cst = c;
        } else {
            tau = df_neg(kk);
        }
        beta = df_mul(df_from2(P.S0_2), pw2(pw, lvl));
        break;
    }
    }
    pstate st;
    st.tau = tau;
    st.beta = beta;
    st.cst = cst;
    return st;
}

// Per-prefix affine coefficients: y = B * (tau + f) with B = 2^-e chosen so that
// |y| <= 1 over the whole suffix range, so that max(y, 0) is a saturating add.
__device__ __forceinline__ pref32 prefix32(const bt_job &J, const bt_jparams &P, const bt_exact_args &a,
                                           int64_t q, bool valid) {
    pref32 r;
    if (!valid) {
        r.B = 0.0f;
        r.Ah = __int_as_float(0x7fc00000);
        r.nAl = r.Ah;
        r.om = df_make(0.0f, 0.0f);
        r.cst = df_make(0.0f, 0.0f);
        return r;
    }
    const pstate st = prefix_state(J, P, a, q);
    const df32 tau = st.tau, beta = st.beta, cst = st.cst;
    const scale32 sc = scale_prefix(tau, P, q);
    r.B = sc.B;
    r.Ah = sc.Ah;
    r.nAl = sc.nAl;
    const df32 rinv = sc.rinv;
    const int c = __popc((unsigned)(q & ((1 << BT_LOW_BITS) - 1)));
    r.om = df_mul(df_mul(df_from2(P.wl2[c]), beta), rinv);
    r.cst = df_mul(df_from2(P.wl2[c]), cst);
    return r;
}

// Payoffs/lambda of eight suffixes under one prefix: y = lambda (tau_hi + f_hi)
// exactly, c = -lambda (tau_lo + f_lo), z = sat(+-(y - c)); returns the
// eight-wide addition tree of the call (MODE & CALL) and put z.
// g + t as (sum, compensation): Fast2Sum (|g| >= |t| after the first add).
__device__ __forceinline__ void fast_acc(float &g, float &e, float t) {
    const float sN = __fadd_rn(g, t);
    e = __fadd_rn(e, __fsub_rn(t, __fsub_rn(sN, g)));
    g = sN;
}

// g += m * (th + tl) for an unnormalised pair (th, tl): exact product of the
// high part (TwoProd), then TwoSum into g; m is a small integer (or 0).
__device__ __forceinline__ void acc_pair(df32 &g, float m, float th, float tl) {
    const df32 p = two_prod(m, th);
    const float lo = __fmaf_rn(m, tl, p.lo);
    const df32 t = two_sum(g.hi, p.hi);
    g.hi = t.hi;
    g.lo = __fadd_rn(g.lo, __fadd_rn(t.lo, lo));
}

// Per-prefix pair coefficients of the class pass: tau, w_low * beta and
// w_low * C (zero for a prefix past the end of the job).
__device__ __forceinline__ void prefix_cls(const bt_job &J, const bt_jparams &P, const bt_exact_args &a, int64_t q,
                                           bool valid, df32 &tau, df32 &om, df32 &cst) {
    if (!valid) {
        tau = om = cst = df_make(0.0f, 0.0f);
        return;
    }
    const pstate st = prefix_state(J, P, a, q);
    const df32 wl = df_from2(P.wl2[__popc((unsigned)(q & ((1 << BT_LOW_BITS) - 1)))]);
    tau = st.tau;
    om = df_mul(wl, st.beta);
    cst = df_mul(wl, st.cst);
}

