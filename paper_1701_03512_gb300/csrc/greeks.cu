// Pathwise derivatives of eq. f13 on the lattice: the derivative pass behind
// bt_greeks_exact (host side in greeks_host.cpp).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bt_internal.h"
#include "df.cuh"
#include "exact_common.cuh"

struct neu_fwd {
    double s, c;
};
__device__ __forceinline__ void neu_fwd_add(neu_fwd &a, double x) {
    const double t = a.s + x;
    if (fabs(a.s) >= fabs(x)) a.c += (a.s - t) + x;
    else a.c += (x - t) + a.s;
    a.s = t;
}

// ---------------------------------------------------------------------------
// Pathwise derivatives of eq. f13 (the adjoint pass behind the Greeks)
//
// With payoff = C + beta * max(s (tau + f), 0) = C + max(s (a + b f), 0)
// (a = beta tau, b = beta, s = +1 call / -1 put), for one prefix and all its
// suffixes (sum_s w_s = 1):
//   sum_s w_s d payoff/du = C' + s (a' N_w + b' F_w + b F'_w),
//   N_w = sum_ITM w_s, F_w = sum_ITM w_s f_s, F'_w = sum_ITM w_s df_s/du;
//   sum_s w_s 1[payoff > 0] = 1 if C > 0 else N_w;
//   sum_s w_s k_s payoff = (beta/lambda) sum_k k W(k) G_k + C L p.
// The kernel accumulates these per prefix next to the value; the host turns
// them into dV/dS0, dV/dsigma, dV/drate, dV/dK by the chain rule through u, p.
// ---------------------------------------------------------------------------
struct prefd {
    float b, bp, ap, Cp, C;
};

__device__ __forceinline__ prefd prefix_deriv(const bt_job &J, const bt_jparams &P, const bt_exact_args &a,
                                              int64_t q) {
    prefd r;
    const int64_t h = q >> J.M;
    const int m = (int)(q & ((1ll << J.M) - 1));
    const bt_pentry eh = a.ph[J.off_ph + h];
    const bt_pentry em = a.pm[J.off_pm + m];
    const int lvl = eh.lvl + em.lvl;
    const bt_pow *pw = a.pw + J.off_pow + J.N + 1;
    const float u = (float)P.u, S0 = (float)P.S0, K = (float)P.K, N = (float)J.N;
    const float SP = S0 * pw[lvl].hi;
    r.b = SP;
    r.bp = (float)lvl * SP / u;
    r.ap = 0.0f;
    r.Cp = 0.0f;
    r.C = 0.0f;
    switch (J.field) {
    case BT_F_ARITH: {
        // a = Sigma_P/N - K, a' = S_P Q_P / (N u), Q_P = u^{-Delta_m} Q_h + l_H R_m + Q_m
        const float QP = pw[-em.lvl].hi * eh.Q + (float)eh.lvl * em.R_hi + em.Q;
        r.b = SP / N;
        r.bp = (float)lvl * SP / (N * u);
        r.ap = SP * QP / (N * u);
        break;
    }
    case BT_F_GEO: {
        const int I = (int)eh.D + J.M * (int)eh.lvl + (int)em.D + J.L * lvl;
        const bt_pow *g = a.pw + J.off_geo - J.geo_imin;
        const float c = S0 * g[I].hi;
        r.b = c;
        r.bp = c * (float)I / (N * u);
        break;
    }
    case BT_F_EURO:
        break;
    case BT_F_LOOKMAX: {
        const int lam = max((int)eh.mx, (int)eh.lvl + (int)em.mx);
        if (lam > -BT_LVL_NONE / 2) {
            const float M = S0 * pw[lam].hi;
            if (M > K) {
                r.ap = -(float)lam * M / u;
                r.Cp = (float)lam * M / u;
                r.C = M - K;
            }
        }
        break;
    }
    default: {
        const int lam = min((int)eh.mn, (int)eh.lvl + (int)em.mn);
        if (lam < BT_LVL_NONE / 2) {
            const float M = S0 * pw[lam].hi;
            if (M < K) {
                r.ap = -(float)lam * M / u;
                r.Cp = -(float)lam * M / u;
                r.C = K - M;
            }
        }
        break;
    }
    }
    return r;
}

// Per-prefix combination and block sum of the derivative pass: value, the
// up-count moment (for dV/dp), the u-derivative and the in-the-money mass.
template <int MODE, bool CLS>
__device__ __forceinline__ void greeks_tail(const bt_exact_args &a, const smem_job &sj, int64_t item_local,
                                            const df32 *accV, const df32 *accK, const df32 *Nw, const df32 *Fw,
                                            const df32 *Dw, double *red4) {
    const bt_job &J = sj.J;
    const bt_jparams &P = sj.P;
    const int64_t qbase = item_local << BT_LOW_BITS;
    const int64_t nP = 1ll << J.P;
    const double sgn = (MODE & BT_MODE_CALL) ? 1.0 : -1.0;
    double tV = 0.0, tK = 0.0, tD = 0.0, tP = 0.0;
#pragma unroll
    for (int j = 0; j < BT_PT; ++j) {
        const int64_t q = qbase + threadIdx.x + j * BT_THREADS;
        if (q >= nP) continue;
        df32 om, cw;  // w_low * beta (/ lambda in the per-path pass) and w_low * C
        if (CLS) {
            df32 tq;
            prefix_cls(J, P, a, q, true, tq, om, cw);
        } else {
            const pref32 pr = prefix32(J, P, a, q, true);
            om = pr.om;
            cw = pr.cst;
        }
        const prefd dv = prefix_deriv(J, P, a, q);
        const double wl = P.wl[__popc((unsigned)(q & ((1 << BT_LOW_BITS) - 1)))];
        const double kq = (double)__popcll((unsigned long long)q);
        const double cq = df_to_double(cw);  // w_low * C as an FP32 pair, as in the value kernel
        const double Vq = df_to_double(df_mul(om, accV[j])) + cq;
        tV += Vq;
        tK += kq * Vq + df_to_double(df_mul(om, accK[j])) + cq * (double)J.L * P.p;
        tD += wl * ((double)dv.Cp +
                    sgn * ((double)dv.ap * df_to_double(Nw[j]) + (double)dv.bp * df_to_double(Fw[j]) +
                           (double)dv.b * df_to_double(Dw[j])));
        tP += wl * (dv.C > 0.0f ? 1.0 : df_to_double(Nw[j]));
    }
    // deterministic block sum of four doubles
    for (int o = 16; o > 0; o >>= 1) {
        tV += __shfl_down_sync(0xffffffffu, tV, o);
        tK += __shfl_down_sync(0xffffffffu, tK, o);
        tD += __shfl_down_sync(0xffffffffu, tD, o);
        tP += __shfl_down_sync(0xffffffffu, tP, o);
    }
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red4[4 * wid + 0] = tV;
        red4[4 * wid + 1] = tK;
        red4[4 * wid + 2] = tD;
        red4[4 * wid + 3] = tP;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[4] = {0.0, 0.0, 0.0, 0.0};
        for (int i = 0; i < BT_THREADS / 32; ++i)
            for (int c = 0; c < 4; ++c) r[c] += red4[4 * i + c];
        const double wh = P.wh[__popcll((unsigned long long)item_local)];
        a.partials4[J.part_off + item_local] = make_double4(r[0] * wh, r[1] * wh, r[2] * wh, r[3] * wh);
    }
}

// Per-path derivative pass over eight suffixes under one prefix: the
// payoff/lambda tree (as tree8), the in-the-money count and the tree of
// df_s/du over the in-the-money suffixes.
template <int MODE>
__device__ __forceinline__ void greeks8(const float4 *f4, const float4 *d4, float B, float Ah, float nAl, float &tz,
                                        float &td, float &cn) {
    const float fh[BT_UNROLL] = {f4[0].x, f4[0].z, f4[1].x, f4[1].z, f4[2].x, f4[2].z, f4[3].x, f4[3].z};
    const float fl[BT_UNROLL] = {f4[0].y, f4[0].w, f4[1].y, f4[1].w, f4[2].y, f4[2].w, f4[3].y, f4[3].w};
    const float fd[BT_UNROLL] = {d4[0].x, d4[0].y, d4[0].z, d4[0].w, d4[1].x, d4[1].y, d4[1].z, d4[1].w};
    float z[BT_UNROLL], t[BT_UNROLL];
#pragma unroll
    for (int i = 0; i < BT_UNROLL; ++i) {
        const float y = __fmaf_rn(B, fh[i], Ah);
        const float c = __fmaf_rn(B, fl[i], nAl);
        z[i] = (MODE & BT_MODE_CALL) ? __saturatef(__fsub_rn(y, c)) : __saturatef(__fsub_rn(c, y));
        // in the money as a number, on the FMA pipe (a compare and two selects would load the ALU
        // pipe, the busier one in this loop): sat(z 2^126) is 1 for every positive normal z and 0
        // out of the money; the NaN padding saturates to 0. Only a positive z below 2^-126 (a
        // cancellation of y - c to 1e-38) would count as a fraction of a path, far below the
        // derivatives' stated accuracy.
        const float ind = __saturatef(__fmul_rn(z[i], 0x1p126f));
        cn = __fadd_rn(cn, ind);
        t[i] = __fmul_rn(ind, fd[i]);
    }
#pragma unroll
    for (int w = 1; w < BT_UNROLL; w *= 2)
#pragma unroll
        for (int i = 0; i < BT_UNROLL; i += 2 * w) {
            z[i] = __fadd_rn(z[i], z[i + w]);
            t[i] = __fadd_rn(t[i], t[i + w]);
        }
    tz = __fadd_rn(tz, z[0]);
    td = __fadd_rn(td, t[0]);
}

// One work item of the derivative pass (per-path table). Per up-count group
// and prefix: sum of payoff/lambda (eight trees per Fast2Sum), in-the-money
// count (exact) and sum of df_s/du (eight trees per TwoSum). The sum of f over
// the in-the-money suffixes follows from the payoff sum: each in-the-money z
// is lambda |tau + f|, so sum f = +-sum z / lambda - tau N_w.
template <int MODE>
__device__ __forceinline__ void item_greeks(const bt_exact_args &a, const smem_job &sj, const float2 *s_suf,
                                            const float *s_sufd, double *red4) {
    const bt_job &J = sj.J;
    const bt_jparams &P = sj.P;
    const int64_t item_local = sj.item - J.item_begin + J.item_offset;
    const int64_t qbase = item_local << BT_LOW_BITS;
    const int64_t nP = 1ll << J.P;
    float B[BT_PT], Ah[BT_PT], nAl[BT_PT];
#pragma unroll
    for (int j = 0; j < BT_PT; ++j) {
        const int64_t q = qbase + threadIdx.x + j * BT_THREADS;
        pref32 pr = prefix32(J, P, a, q, q < nP);
        B[j] = pr.B;
        Ah[j] = pr.Ah;
        nAl[j] = pr.nAl;
    }
    df32 accV[BT_PT], accK[BT_PT], Nw[BT_PT], Dw[BT_PT];
#pragma unroll
    for (int j = 0; j < BT_PT; ++j) accV[j] = accK[j] = Nw[j] = Dw[j] = df_make(0.0f, 0.0f);
    for (int k = 0; k <= J.L; ++k) {
        const int s0 = J.goff[k], s1 = J.goff[k + 1];
        float g[BT_PT], e[BT_PT], cd[BT_PT], ed[BT_PT], cn[BT_PT];
#pragma unroll
        for (int j = 0; j < BT_PT; ++j) g[j] = e[j] = cd[j] = ed[j] = cn[j] = 0.0f;
        int s = s0;
        for (; s + 8 * BT_UNROLL <= s1; s += 8 * BT_UNROLL) {
            float tz[BT_PT], td[BT_PT];
#pragma unroll
            for (int j = 0; j < BT_PT; ++j) tz[j] = td[j] = 0.0f;
#pragma unroll 1
            for (int r = 0; r < 8; ++r) {
                const int sr = s + r * BT_UNROLL;
                float4 f4[BT_UNROLL / 2], d4[BT_UNROLL / 4];
#pragma unroll
                for (int i = 0; i < BT_UNROLL / 2; ++i) f4[i] = *reinterpret_cast<const float4 *>(s_suf + sr + 2 * i);
#pragma unroll
                for (int i = 0; i < BT_UNROLL / 4; ++i) d4[i] = *reinterpret_cast<const float4 *>(s_sufd + sr + 4 * i);
#pragma unroll
                for (int j = 0; j < BT_PT; ++j) greeks8<MODE>(f4, d4, B[j], Ah[j], nAl[j], tz[j], td[j], cn[j]);
            }
#pragma unroll
            for (int j = 0; j < BT_PT; ++j) {
                fast_acc(g[j], e[j], tz[j]);
                const df32 ts = two_sum(cd[j], td[j]);
                cd[j] = ts.hi;
                ed[j] = __fadd_rn(ed[j], ts.lo);
            }
        }
        for (; s < s1; s += BT_UNROLL) {
            float4 f4[BT_UNROLL / 2], d4[BT_UNROLL / 4];
#pragma unroll
            for (int i = 0; i < BT_UNROLL / 2; ++i) f4[i] = *reinterpret_cast<const float4 *>(s_suf + s + 2 * i);
#pragma unroll
            for (int i = 0; i < BT_UNROLL / 4; ++i) d4[i] = *reinterpret_cast<const float4 *>(s_sufd + s + 4 * i);
#pragma unroll
            for (int j = 0; j < BT_PT; ++j) {
                float tz = 0.0f, td = 0.0f;
                greeks8<MODE>(f4, d4, B[j], Ah[j], nAl[j], tz, td, cn[j]);
                fast_acc(g[j], e[j], tz);
                const df32 ts = two_sum(cd[j], td);
                cd[j] = ts.hi;
                ed[j] = __fadd_rn(ed[j], ts.lo);
            }
        }
        const df32 w = df_from2(P.W2[k]);
#pragma unroll
        for (int j = 0; j < BT_PT; ++j) {
            const df32 wg = df_mul(w, fast_two_sum(g[j], e[j]));
            accV[j] = df_add_pos(accV[j], wg);
            accK[j] = df_add_pos(accK[j], df_mul_f(wg, (float)k));
            Nw[j] = df_add_pos(Nw[j], df_mul_f(w, cn[j]));
            Dw[j] = df_add(Dw[j], df_mul(w, two_sum(cd[j], ed[j])));
        }
    }
    df32 Fw[BT_PT];
#pragma unroll
    for (int j = 0; j < BT_PT; ++j) {
        const int64_t q = qbase + threadIdx.x + j * BT_THREADS;
        Fw[j] = df_make(0.0f, 0.0f);
        if (q >= nP) continue;
        const df32 tau = prefix_state(J, P, a, q).tau;
        const df32 zl = df_mul(accV[j], scale_prefix(tau, P, q).rinv);  // sum of |tau + f| over ITM
        Fw[j] = df_sub((MODE & BT_MODE_CALL) ? zl : df_neg(zl), df_mul(tau, Nw[j]));
    }
    greeks_tail<MODE, false>(a, sj, item_local, accV, accK, Nw, Fw, Dw, red4);
}

// Derivative pass over a class table: per class the in-the-money test and
// the sums of multiplicity x (payoff, 1, f, df/du) in FP32 pairs.
template <int MODE>
__device__ __forceinline__ void item_greeks_cls(const bt_exact_args &a, const smem_job &sj, const float2 *s_suf,
                                                const float *s_sufd, double *red4) {
    const bt_job &J = sj.J;
    const bt_jparams &P = sj.P;
    const int64_t item_local = sj.item - J.item_begin + J.item_offset;
    const int64_t qbase = item_local << BT_LOW_BITS;
    const int64_t nP = 1ll << J.P;
    const float4 *s_cls = reinterpret_cast<const float4 *>(s_suf);
    const float2 *s_cd = reinterpret_cast<const float2 *>(s_sufd);
    df32 tau[BT_PT];
#pragma unroll
    for (int j = 0; j < BT_PT; ++j) {
        const int64_t q = qbase + threadIdx.x + j * BT_THREADS;
        df32 om, cw;
        prefix_cls(J, P, a, q, q < nP, tau[j], om, cw);
    }
    df32 accV[BT_PT], accK[BT_PT], Fw[BT_PT], Dw[BT_PT], Nw[BT_PT];
#pragma unroll
    for (int j = 0; j < BT_PT; ++j) accV[j] = accK[j] = Fw[j] = Dw[j] = Nw[j] = df_make(0.0f, 0.0f);
    for (int k = 0; k <= J.L; ++k) {
        df32 g[BT_PT], cf[BT_PT], cd[BT_PT];
        float cn[BT_PT];
#pragma unroll
        for (int j = 0; j < BT_PT; ++j) {
            g[j] = cf[j] = cd[j] = df_make(0.0f, 0.0f);
            cn[j] = 0.0f;
        }
        for (int s = J.goff[k]; s < J.goff[k + 1]; ++s) {
            const float4 e = s_cls[s];
            const float2 fd = s_cd[s];
#pragma unroll
            for (int j = 0; j < BT_PT; ++j) {
                const df32 t0 = two_sum(tau[j].hi, e.x);
                const float tl = __fadd_rn(t0.lo, __fadd_rn(tau[j].lo, e.y));
                const float ts = __fadd_rn(t0.hi, tl);
                const bool itm = (MODE & BT_MODE_CALL) ? ts > 0.0f : ts < 0.0f;
                const float m = itm ? e.z : 0.0f;
                acc_pair(g[j], (MODE & BT_MODE_CALL) ? m : -m, t0.hi, tl);
                cn[j] += m;
                acc_pair(cf[j], m, e.x, e.y);
                acc_pair(cd[j], m, fd.x, fd.y);
            }
        }
        const df32 w = df_from2(P.W2[k]);
#pragma unroll
        for (int j = 0; j < BT_PT; ++j) {
            const df32 wg = df_mul(w, fast_two_sum(g[j].hi, g[j].lo));
            accV[j] = df_add_pos(accV[j], wg);
            accK[j] = df_add_pos(accK[j], df_mul_f(wg, (float)k));
            Nw[j] = df_add_pos(Nw[j], df_mul_f(w, cn[j]));
            Fw[j] = df_add(Fw[j], df_mul(w, fast_two_sum(cf[j].hi, cf[j].lo)));
            Dw[j] = df_add(Dw[j], df_mul(w, two_sum(cd[j].hi, cd[j].lo)));
        }
    }
    greeks_tail<MODE, true>(a, sj, item_local, accV, accK, Nw, Fw, Dw, red4);
}

__global__ void __launch_bounds__(BT_THREADS, 2) k_greeks32(bt_exact_args a) {
    extern __shared__ float4 smem_raw[];
    float2 *s_suf = reinterpret_cast<float2 *>(smem_raw);
    float *s_sufd = reinterpret_cast<float *>(s_suf + BT_SUF_MAX_EVEN);  // 16-byte aligned for float4 loads
    __shared__ smem_job sj;
    __shared__ double red4[4 * (BT_THREADS / 32)];
    int cur_job = -1;
    for (;;) {
        const int prev = cur_job;
        if (!next_item<float2>(a, sj, s_suf, a.suf32, cur_job)) break;
        if (cur_job != prev) {
            const float *src = a.sufd + sj.J.off_suf;
            for (int i = threadIdx.x; i < sj.J.suf_len; i += BT_THREADS) s_sufd[i] = src[i];
            __syncthreads();
        }
        if (sj.J.cls) {
            if (sj.J.mode == BT_MODE_CALL) item_greeks_cls<BT_MODE_CALL>(a, sj, s_suf, s_sufd, red4);
            else item_greeks_cls<BT_MODE_PUT>(a, sj, s_suf, s_sufd, red4);
        } else if (sj.J.mode == BT_MODE_CALL) {
            item_greeks<BT_MODE_CALL>(a, sj, s_suf, s_sufd, red4);
        } else {
            item_greeks<BT_MODE_PUT>(a, sj, s_suf, s_sufd, red4);
        }
    }
}

// Fixed-order per-job sums of the four partials.
__global__ void k_greeks_finalize(const bt_job *jobs, int n_jobs, const double4 *partials, double4 *sums) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_jobs) return;
    const bt_job J = jobs[j];
    neu_fwd v = {0, 0}, k = {0, 0}, d = {0, 0}, p = {0, 0};
    for (int i = 0; i < J.n_items; ++i) {
        const double4 x = partials[J.part_off + i];
        neu_fwd_add(v, x.x);
        neu_fwd_add(k, x.y);
        neu_fwd_add(d, x.z);
        neu_fwd_add(p, x.w);
    }
    sums[j] = make_double4(v.s + v.c, k.s + k.c, d.s + d.c, p.s + p.c);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
extern "C" int bt_launch_greeks(const bt_exact_args *a, int grid, void *stream) {
    if (a->n_run_items <= 0) return 0;
    const size_t sm = (size_t)BT_SUF_MAX_EVEN * sizeof(float2) + (size_t)BT_SUF_MAX * sizeof(float);
    cudaFuncSetAttribute(k_greeks32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    {  // persistent grid: every SM's resident blocks, no more
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_greeks32, BT_THREADS, sm);
        if (sms > 0 && per > 0) grid = sms * per;
    }
    if ((int64_t)grid > a->n_run_items) grid = (int)a->n_run_items;
    k_greeks32<<<grid, BT_THREADS, sm, (cudaStream_t)stream>>>(*a);
    return (int)cudaGetLastError();
}

extern "C" int bt_launch_greeks_finalize(const bt_job *d_jobs, int n_jobs, const double4 *partials, double4 *sums,
                                         void *stream) {
    if (n_jobs <= 0) return 0;
    k_greeks_finalize<<<(n_jobs + 63) / 64, 64, 0, (cudaStream_t)stream>>>(d_jobs, n_jobs, partials, sums);
    return (int)cudaGetLastError();
}

