// Exhaustive expected value over all 2^N Bernoulli paths (eq. f13), sm_103a.
//
// A path index b of an N-step tree splits into a prefix (the first P = N - L
// steps, the high bits -- Section 3's rank bits) and a suffix (the last L
// steps). With u d = 1 (A1) and levels l_t = 2 U_t - t, S_t = S0 u^{l_t}, every
// payoff here is, for a fixed prefix, an affine function of one per-suffix
// number f_s:
//     payoff(prefix, suffix) = beta_p * max(+-(tau_p + f_s), 0) + C_p
// (tau_p, beta_p, C_p from the prefix; the sign selects call or put). The path
// weight factorises as p(x) = w_p * w_s with w_s = p^k (1-p)^{L-k} depending
// only on the suffix's up-count k. So one block of threads holds the suffix
// table (sorted by k) in shared memory, each thread holds four prefixes in
// registers, and every path costs one FP32 FMA for lambda (tau + f), one FMA
// for the low-order correction, one saturating add for max(., 0) and its
// share of an eight-wide addition tree (a call and a put of the same tree
// share the two FMAs). Eight trees are added in turn and enter the group sum
// through one Fast2Sum (compensated), group sums are folded with the weight
// w(k) by error-free transformations, prefixes are combined in FP32 pairs,
// and the block's total goes to FP64 (eq. f14); block partials are added in
// a fixed order per option (eq. f15).
//
// The European, geometric and lookback payoffs take a table of recombined
// suffix classes instead (k_class_tables, item32_cls): within an up-count
// group their f_s depends on one integer key, so each class is evaluated once
// per prefix in FP32-pair arithmetic and weighted by its multiplicity. The
// arithmetic Asian below 2^28 paths (N <= 27) takes the same pass with every
// suffix its own class (k_tables writes that table): with fewer paths the
// per-path roundings would not average below 1e-9.
//
// Rounding design of the FP32 path. The per-prefix scale lambda = 2^-e
// (256 - h)/256, with 2^e bounding |tau + f| over the suffix range and h a
// 7-bit hash of the prefix index, keeps |lambda (tau + f)| <= 1 so that
// max(., 0) is a saturating add. The suffix table stores f_hi on the fixed grid
// 2^gexp (gexp = ceil(log2 max f) - 10, at most 10 significant bits) and the
// exact remainder f_lo; the prefix rounds A = lambda tau to the grid
// 2^(gexp - e - 8). Then lambda f_hi + A_hi is exact in
// FP32 on every path, and the only rounding of the payoff is one
// correctly-rounded FP32 result -- unbiased, unlike a rounding of a rounded
// value. The hash makes prefixes that share tau (the structured payoffs) scale
// differently, so those single roundings also average out across prefixes.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bt_internal.h"
#include "df.cuh"
#include "exact_common.cuh"

// ---------------------------------------------------------------------------
// Tree parameters (Section 2, A1-A3) on the device
// ---------------------------------------------------------------------------
__device__ static int dev_tree(const bt_option &o, double *u, double *d, double *p) {
    double dt = o.T / (double)o.N;
    double uu;
    if (o.tree_kind == BT_TREE_CRR) {
        uu = exp(o.sigma * sqrt(dt));
    } else if (o.tree_kind == BT_TREE_SEYDEL) {
        double beta = 0.5 * (exp(-o.rate * dt) + exp((o.rate + o.sigma * o.sigma) * dt));
        uu = beta + sqrt(beta * beta - 1.0);
    } else {
        *u = o.u;
        *d = o.d;
        *p = o.p;
        return o.p > 0.0 && o.p < 1.0;
    }
    double dd = 1.0 / uu;
    double pp = (exp(o.rate * dt) - dd) / (uu - dd);
    *u = uu;
    *d = dd;
    *p = pp;
    return pp > 0.0 && pp < 1.0;
}

__device__ static double ipow(double x, int n) {
    double r = 1.0;
    for (int i = 0; i < n; ++i) r *= x;
    return r;
}

// One warp per job: the record is zeroed, then lane 0 writes the scalars and the lanes write the
// weight tables entry by entry (lane k: p^k (1-p)^(L-k), ...), so that the slow FP64 powers run
// side by side instead of one after another. Each entry has the same formula as in a serial loop.
static_assert(sizeof(bt_jparams) % sizeof(double) == 0, "bt_jparams is zeroed in doubles");
__global__ void k_params(const bt_option *opts, const bt_job *jobs, bt_jparams *prm, int n_jobs) {
    const int j = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= n_jobs) return;
    const bt_job &J = jobs[j];
    const bt_option o = opts[J.opt];
    bt_jparams *P = prm + J.prm_off;
    double *z = reinterpret_cast<double *>(P);
    for (int i = lane; i < (int)(sizeof(bt_jparams) / sizeof(double)); i += 32) z[i] = 0.0;
    __syncwarp();
    double u, d, p;
    const int ok = dev_tree(o, &u, &d, &p);   // every lane, the same values
    const double q = 1.0 - p;
    const int L = J.L;
    const int plo = J.P < BT_LOW_BITS ? J.P : BT_LOW_BITS;
    const int phi = J.P - plo;
    static_assert(BT_MAX_L < 32 && BT_LOW_BITS < 32 && BT_MAX_N_EXACT - 1 - BT_LOW_BITS < 32, "one lane per entry");
    if (lane <= L) {
        P->W[lane] = ipow(p, lane) * ipow(q, L - lane);
        P->W2[lane] = split2(P->W[lane]);
    }
    if (lane <= plo) {
        P->wl[lane] = ipow(p, lane) * ipow(q, plo - lane);
        P->wl2[lane] = split2(P->wl[lane]);
    }
    if (lane <= phi) P->wh[lane] = pow(p, (double)lane) * pow(q, (double)(phi - lane));
    if (lane != 0) return;
    P->ok = ok;
    P->u = u;
    P->d = d;
    P->p = p;
    P->disc = exp(-o.rate * o.T);
    const double lnu = log(u);
    P->lnu = lnu;
    P->S0 = o.S0;
    P->K = o.K;
    P->NKoS0 = (double)J.N * o.K / o.S0;
    P->KoS0 = o.K / o.S0;
    P->S0oN = o.S0 / (double)J.N;
    double fmin, fmax;
    switch (J.field) {
    case BT_F_ARITH: {
        double a = 0.0, b = 0.0, ru = 1.0, rd = 1.0;
        for (int i = 1; i <= L; ++i) {
            ru *= u;
            rd *= d;
            a += rd;
            b += ru;
        }
        fmin = a;
        fmax = b;
        break;
    }
    case BT_F_GEO: {
        double e = (double)L * (double)(L + 1) / (2.0 * (double)J.N);
        fmin = exp(-e * lnu);
        fmax = exp(e * lnu);
        break;
    }
    case BT_F_EURO:
        fmin = exp(-(double)L * lnu);
        fmax = exp((double)L * lnu);
        break;
    case BT_F_LOOKMAX:
        fmin = exp(-lnu);
        fmax = exp((double)L * lnu);
        break;
    default:
        fmin = exp(-(double)L * lnu);
        fmax = exp(lnu);
        break;
    }
    P->fmin = fmin;
    P->fmax = fmax;
    P->NKoS0_2 = split2((double)J.N * o.K / o.S0);
    P->KoS0_2 = split2(o.K / o.S0);
    P->S0oN_2 = split2(o.S0 / (double)J.N);
    P->S0_2 = split2(o.S0);
    P->K_2 = split2(o.K);
    P->fmin_f = (float)fmin;
    P->fmax_f = (float)fmax;
    int ef;
    frexp(fmax, &ef);  // fmax <= 2^ef
    P->gexp = ef - 10;
}

// ---------------------------------------------------------------------------
// Suffix table (sorted by up-count, groups padded with NaN) and the
// two-level prefix tables, in FP64
// ---------------------------------------------------------------------------
__device__ static int binom_small(int n, int k) {
    if (k < 0 || k > n) return 0;
    int r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// Rank of a k-subset among all k-subsets in colexicographic order (the
// combinatorial number system): sum over the i-th set bit c_i of C(c_i, i).
__device__ static int colex_rank(unsigned s) {
    int r = 0, i = 0;
    while (s) {
        int c = __ffs(s) - 1;
        ++i;
        r += binom_small(c, i);
        s &= s - 1;
    }
    return r;
}

// Walk `bits` steps of `x` (MSB first) from level 0 and return the block's
// summary: end level, max/min level, level sum, the backward-relative
// partial sum R = sum_t u^{l_t - l_end} (R_t = R_{t-1} * u^{-(l_t - l_{t-1})} + 1)
// and its level-weighted form Q = sum_t l_t u^{l_t - l_end}.
__device__ static bt_pentry walk_block(uint64_t x, int bits, double u, double d) {
    bt_pentry e;
    int lvl = 0, mx = -BT_LVL_NONE, mn = BT_LVL_NONE, D = 0;
    double R = 0.0, Q = 0.0;
    for (int t = 1; t <= bits; ++t) {
        int up = (int)((x >> (bits - t)) & 1u);
        lvl += up ? 1 : -1;
        R = R * (up ? d : u) + 1.0;
        Q = Q * (up ? d : u) + (double)lvl;
        mx = lvl > mx ? lvl : mx;
        mn = lvl < mn ? lvl : mn;
        D += lvl;
    }
    e.R64 = R;
    float2 r2 = split2(R);
    e.R_hi = r2.x;
    e.R_lo = r2.y;
    e.lvl = (int16_t)lvl;
    e.mx = (int16_t)mx;
    e.mn = (int16_t)mn;
    e.D = (int16_t)D;
    e.Q = (float)Q;
    e.pad = 0;
    return e;
}

__global__ void k_tables(const bt_job *jobs, const bt_jparams *prm, int prec, float2 *suf32, double *suf64,
                         bt_pentry *ph, bt_pentry *pm, bt_pow *pw, float *sufd) {
    const int j = blockIdx.y;
    const bt_job J = jobs[j];
    const bt_jparams &Pj = prm[J.prm_off];
    const double u = Pj.u, d = Pj.d, lnu = Pj.lnu;
    // class jobs get their suffix table from k_class_tables, except the
    // arithmetic Asian's: its classes are its suffixes, one path each
    const bool acls = J.cls && J.field == BT_F_ARITH;
    const int64_t nsuf = (J.cls && !acls) ? 0 : 1ll << J.L;
    const int64_t nsl = (J.cls && !acls) ? 0 : acls ? J.suf_len / 2 : J.suf_len;
    const int64_t nh = 1ll << J.H, nm = 1ll << J.M;
    const int64_t npow = 2 * J.N + 3;
    const int64_t total = nsuf + nsl + nh + nm + npow + J.geo_len;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx;
        if (i < nsuf) {  // suffix entry
            unsigned s = (unsigned)i;
            int k = __popc(s);
            int lvl = 0, mx = -BT_LVL_NONE, mn = BT_LVL_NONE, D = 0;
            double r = 1.0, f = 0.0, fl = 0.0;
            for (int t = 1; t <= J.L; ++t) {
                int up = (int)((s >> (J.L - t)) & 1u);
                lvl += up ? 1 : -1;
                r *= up ? u : d;
                f += r;
                fl += (double)lvl * r;
                D += lvl;
                mx = lvl > mx ? lvl : mx;
                mn = lvl < mn ? lvl : mn;
            }
            double v;
            switch (J.field) {
            case BT_F_ARITH: v = f; break;
            case BT_F_GEO: v = exp((double)D * lnu / (double)J.N); break;
            case BT_F_EURO: v = exp((double)lvl * lnu); break;
            case BT_F_LOOKMAX: v = exp((double)mx * lnu); break;
            default: v = exp((double)mn * lnu); break;
            }
            int pos = J.goff[k] + colex_rank(s);
            if (acls) {  // class entry (f_hi, f_lo), (multiplicity 1, 0); with sufd, df/du as a pair
                suf32[J.off_suf + 2 * pos] = split2(v);
                suf32[J.off_suf + 2 * pos + 1] = make_float2(1.0f, 0.0f);
                if (sufd) {
                    const float2 dd = split2(fl / u);
                    sufd[J.off_suf + 2 * pos] = dd.x;
                    sufd[J.off_suf + 2 * pos + 1] = dd.y;
                }
                continue;
            }
            if (sufd) {  // df_s/du
                double dv;
                switch (J.field) {
                case BT_F_ARITH: dv = fl / u; break;
                case BT_F_GEO: dv = v * (double)D / ((double)J.N * u); break;
                case BT_F_EURO: dv = v * (double)lvl / u; break;
                case BT_F_LOOKMAX: dv = v * (double)mx / u; break;
                default: dv = v * (double)mn / u; break;
                }
                sufd[J.off_suf + pos] = (float)dv;
            }
            if (prec == BT_PREC_FP64) {
                suf64[J.off_suf + pos] = v;
            } else {
                // f_hi on the grid 2^gexp (exact in FP32), f_lo the exact remainder
                const int gx = Pj.gexp;
                const double fh = ldexp(rint(ldexp(v, -gx)), gx);
                suf32[J.off_suf + pos] = make_float2((float)fh, -(float)(v - fh));  // (f_hi, -f_lo)
            }
            continue;
        }
        i -= nsuf;
        if (i < nsl) {  // padding slots of each up-count group
            int pos = (int)i, k = 0;
            while (k < J.L && pos >= J.goff[k + 1]) ++k;
            if (pos - J.goff[k] >= binom_small(J.L, k) && acls) {  // zero-multiplicity classes
                suf32[J.off_suf + 2 * pos] = make_float2(0.0f, 0.0f);
                suf32[J.off_suf + 2 * pos + 1] = make_float2(0.0f, 0.0f);
                if (sufd) sufd[J.off_suf + 2 * pos] = sufd[J.off_suf + 2 * pos + 1] = 0.0f;
            } else if (pos - J.goff[k] >= binom_small(J.L, k)) {
                if (prec == BT_PREC_FP64) suf64[J.off_suf + pos] = nan("");
                else suf32[J.off_suf + pos] = make_float2(__int_as_float(0x7fc00000), 0.0f);
                if (sufd) sufd[J.off_suf + pos] = 0.0f;
            }
            continue;
        }
        i -= nsl;
        if (i < nh) {
            ph[J.off_ph + i] = walk_block((uint64_t)i, J.H, u, d);
            continue;
        }
        i -= nh;
        if (i < nm) {
            pm[J.off_pm + i] = walk_block((uint64_t)i, J.M, u, d);
            continue;
        }
        i -= nm;
        bt_pow e;
        if (i < npow) {
            e.v = exp((double)(i - (J.N + 1)) * lnu);
            float2 h = split2(e.v);
            e.hi = h.x;
            e.lo = h.y;
            pw[J.off_pow + i] = e;
            continue;
        }
        i -= npow;
        e.v = exp((double)(J.geo_imin + i) * lnu / (double)J.N);
        float2 h = split2(e.v);
        e.hi = h.x;
        e.lo = h.y;
        pw[J.off_geo + i] = e;
    }
}

// Suffix table of recombined classes (the FP32 geometric, European and
// lookback passes). Within an up-count group every suffix with the same key
// -- level sum D (f = u^{D/N}), end level (u^{l'_L}), max or min level
// (u^{max l'}, u^{min l'}) -- has the same f_s and the same weight, so the
// group's sum over suffixes is a sum over its distinct keys times their
// multiplicities. One block per job counts the keys of all 2^L suffixes in
// shared memory and writes, per group in ascending key order, two float2
// slots per class: (f_hi, f_lo) and (multiplicity, 0); with sufd, the pair
// (df/du hi, lo). Groups are padded with zero-multiplicity classes. The
// host plans the same class counts (same keys, same order) for goff.
#define BT_KEY_RANGE (2 * BT_KEY_SPAN + 1)
__global__ void k_class_tables(const bt_job *jobs, const bt_jparams *prm, float2 *suf32, float *sufd) {
    const bt_job J = jobs[blockIdx.x];
    if (!J.cls || J.field == BT_F_ARITH) return;  // the arithmetic Asian's classes come from k_tables
    __shared__ int hist[(BT_MAX_L + 1) * BT_KEY_RANGE];
    for (int i = threadIdx.x; i < (J.L + 1) * BT_KEY_RANGE; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (unsigned s = threadIdx.x; s < (1u << J.L); s += blockDim.x) {
        int lvl = 0, mx = -BT_LVL_NONE, mn = BT_LVL_NONE, D = 0;
        for (int t = 1; t <= J.L; ++t) {
            lvl += ((s >> (J.L - t)) & 1u) ? 1 : -1;
            mx = max(mx, lvl);
            mn = min(mn, lvl);
            D += lvl;
        }
        const int key = J.field == BT_F_GEO ? D : J.field == BT_F_EURO ? lvl : J.field == BT_F_LOOKMAX ? mx : mn;
        atomicAdd(&hist[__popc(s) * BT_KEY_RANGE + key + BT_KEY_SPAN], 1);
    }
    __syncthreads();
    const bt_jparams &P = prm[J.prm_off];
    const double lnu = P.lnu, u = P.u, N = (double)J.N;
    for (int k = threadIdx.x; k <= J.L; k += blockDim.x) {
        int pos = J.goff[k];
        const int end = J.goff[k + 1];
        for (int key = -BT_KEY_SPAN; key <= BT_KEY_SPAN && pos < end; ++key) {
            const int c = hist[k * BT_KEY_RANGE + key + BT_KEY_SPAN];
            if (!c) continue;
            const double x = J.field == BT_F_GEO ? (double)key / N : (double)key;
            const double v = exp(x * lnu);
            suf32[J.off_suf + 2 * pos] = split2(v);
            suf32[J.off_suf + 2 * pos + 1] = make_float2((float)c, 0.0f);
            if (sufd) {
                const float2 dv = split2(v * x / u);
                sufd[J.off_suf + 2 * pos] = dv.x;
                sufd[J.off_suf + 2 * pos + 1] = dv.y;
            }
            ++pos;
        }
        for (; pos < end; ++pos) {
            suf32[J.off_suf + 2 * pos] = make_float2(0.0f, 0.0f);
            suf32[J.off_suf + 2 * pos + 1] = make_float2(0.0f, 0.0f);
            if (sufd) {
                sufd[J.off_suf + 2 * pos] = 0.0f;
                sufd[J.off_suf + 2 * pos + 1] = 0.0f;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Prefix states and the path sums
// ---------------------------------------------------------------------------
template <int MODE>
__device__ __forceinline__ void tree8(const float4 *f4, float B, float Ah, float nAl, float &tc, float &tp) {
    float y[BT_UNROLL], c[BT_UNROLL];
#pragma unroll
    for (int i = 0; i < BT_UNROLL / 2; ++i) {
        y[2 * i] = __fmaf_rn(B, f4[i].x, Ah);
        c[2 * i] = __fmaf_rn(B, f4[i].y, nAl);
        y[2 * i + 1] = __fmaf_rn(B, f4[i].z, Ah);
        c[2 * i + 1] = __fmaf_rn(B, f4[i].w, nAl);
    }
    if (MODE & BT_MODE_CALL) {
        float z[BT_UNROLL];
#pragma unroll
        for (int i = 0; i < BT_UNROLL; ++i) z[i] = __saturatef(__fsub_rn(y[i], c[i]));
#pragma unroll
        for (int w = 1; w < BT_UNROLL; w *= 2)
#pragma unroll
            for (int i = 0; i < BT_UNROLL; i += 2 * w) z[i] = __fadd_rn(z[i], z[i + w]);
        tc = z[0];
    }
    if (MODE & BT_MODE_PUT) {
        float z[BT_UNROLL];
#pragma unroll
        for (int i = 0; i < BT_UNROLL; ++i) z[i] = __saturatef(__fsub_rn(c[i], y[i]));
#pragma unroll
        for (int w = 1; w < BT_UNROLL; w *= 2)
#pragma unroll
            for (int i = 0; i < BT_UNROLL; i += 2 * w) z[i] = __fadd_rn(z[i], z[i + w]);
        tp = z[0];
    }
}

template <int MODE>
__device__ __forceinline__ void item32(const bt_exact_args &a, const smem_job &sj, const float2 *s_suf,
                                       double2 *red) {
    const bt_job &J = sj.J;
    const bt_jparams &P = sj.P;
    const int64_t item_local = sj.item - J.item_begin + J.item_offset;
    const int64_t qbase = item_local << BT_LOW_BITS;
    const int64_t nP = 1ll << J.P;

    // the loop needs only the scaled affine form; w_low beta / lambda and C
    // are recomputed at the end (keeps registers for the sixteen-wide trees)
    float B[BT_PT], Ah[BT_PT], nAl[BT_PT];
#pragma unroll
    for (int j = 0; j < BT_PT; ++j) {
        const int64_t q = qbase + threadIdx.x + j * BT_THREADS;
        pref32 pr = prefix32(J, P, a, q, q < nP);
        B[j] = pr.B;
        Ah[j] = pr.Ah;
        nAl[j] = pr.nAl;
    }
    df32 accC[BT_PT], accP[BT_PT];
#pragma unroll
    for (int j = 0; j < BT_PT; ++j) accC[j] = accP[j] = df_make(0.0f, 0.0f);

    for (int k = 0; k <= J.L; ++k) {
        const int s0 = J.goff[k], s1 = J.goff[k + 1];
        // group sums as (sum, compensation) pairs
        float gc[BT_PT], ec[BT_PT], gp[BT_PT], ep[BT_PT];
#pragma unroll
        for (int j = 0; j < BT_PT; ++j) gc[j] = ec[j] = gp[j] = ep[j] = 0.0f;
        int s = s0;
        // 64 suffixes per step: eight eight-wide trees added in turn, one Fast2Sum
        for (; s + 8 * BT_UNROLL <= s1; s += 8 * BT_UNROLL) {
            float tc[BT_PT], tp[BT_PT];
#pragma unroll
            for (int j = 0; j < BT_PT; ++j) tc[j] = tp[j] = 0.0f;
#pragma unroll 2
            for (int r = 0; r < 8; ++r) {
                float4 f4[BT_UNROLL / 2];
#pragma unroll
                for (int i = 0; i < BT_UNROLL / 2; ++i)
                    f4[i] = *reinterpret_cast<const float4 *>(s_suf + s + r * BT_UNROLL + 2 * i);
#pragma unroll
                for (int j = 0; j < BT_PT; ++j) {
                    float uc, up;
                    tree8<MODE>(f4, B[j], Ah[j], nAl[j], uc, up);
                    if (MODE & BT_MODE_CALL) tc[j] = __fadd_rn(tc[j], uc);
                    if (MODE & BT_MODE_PUT) tp[j] = __fadd_rn(tp[j], up);
                }
            }
#pragma unroll
            for (int j = 0; j < BT_PT; ++j) {
                if (MODE & BT_MODE_CALL) fast_acc(gc[j], ec[j], tc[j]);
                if (MODE & BT_MODE_PUT) fast_acc(gp[j], ep[j], tp[j]);
            }
        }
        for (; s < s1; s += BT_UNROLL) {  // the last one to seven eights of the group
            float4 f4[BT_UNROLL / 2];
#pragma unroll
            for (int i = 0; i < BT_UNROLL / 2; ++i) f4[i] = *reinterpret_cast<const float4 *>(s_suf + s + 2 * i);
#pragma unroll
            for (int j = 0; j < BT_PT; ++j) {
                float uc, up;
                tree8<MODE>(f4, B[j], Ah[j], nAl[j], uc, up);
                if (MODE & BT_MODE_CALL) fast_acc(gc[j], ec[j], uc);
                if (MODE & BT_MODE_PUT) fast_acc(gp[j], ep[j], up);
            }
        }
        const df32 w = df_from2(P.W2[k]);
#pragma unroll
        for (int j = 0; j < BT_PT; ++j) {
            if (MODE & BT_MODE_CALL) accC[j] = df_add_pos(accC[j], df_mul(w, fast_two_sum(gc[j], ec[j])));
            if (MODE & BT_MODE_PUT) accP[j] = df_add_pos(accP[j], df_mul(w, fast_two_sum(gp[j], ep[j])));
        }
    }
    df32 totC = df_make(0.0f, 0.0f), totP = df_make(0.0f, 0.0f);
    df32 cst = df_make(0.0f, 0.0f);
#pragma unroll
    for (int j = 0; j < BT_PT; ++j) {
        const int64_t q = qbase + threadIdx.x + j * BT_THREADS;
        const pref32 pr = prefix32(J, P, a, q, q < nP);
        cst = df_add_pos(cst, pr.cst);
        if (MODE & BT_MODE_CALL) totC = df_add_pos(totC, df_mul(pr.om, accC[j]));
        if (MODE & BT_MODE_PUT) totP = df_add_pos(totP, df_mul(pr.om, accP[j]));
    }
    double vc = df_to_double(totC), vp = df_to_double(totP);
    if (J.field == BT_F_LOOKMAX) vc += df_to_double(cst);
    if (J.field == BT_F_LOOKMIN) vp += df_to_double(cst);
    double2 sum2 = block_sum2(vc, vp, red);
    if (threadIdx.x == 0) {
        const double wh = P.wh[__popcll((unsigned long long)item_local)];
        a.partials[J.part_off + item_local] = make_double2(sum2.x * wh, sum2.y * wh);
    }
}

// One work item over a class table (J.cls): for each prefix and up-count
// group, sum multiplicity * max(+-(tau + f), 0) over the group's classes with
// tau + f, the product and the sum all in FP32 pairs, then fold with W(k) as
// in item32. Identical classes are evaluated once, so there is no repeated
// FP32 rounding to correlate across the suffixes of a group.
template <int MODE>
__device__ __forceinline__ void item32_cls(const bt_exact_args &a, const smem_job &sj, const float2 *s_suf,
                                           double2 *red) {
    const bt_job &J = sj.J;
    const bt_jparams &P = sj.P;
    const int64_t item_local = sj.item - J.item_begin + J.item_offset;
    const int64_t qbase = item_local << BT_LOW_BITS;
    const int64_t nP = 1ll << J.P;
    const float4 *s_cls = reinterpret_cast<const float4 *>(s_suf);

    df32 tau[BT_PT], om[BT_PT];
    df32 cst = df_make(0.0f, 0.0f);
#pragma unroll
    for (int j = 0; j < BT_PT; ++j) {
        const int64_t q = qbase + threadIdx.x + j * BT_THREADS;
        df32 c;
        prefix_cls(J, P, a, q, q < nP, tau[j], om[j], c);
        cst = df_add_pos(cst, c);
    }
    df32 accC[BT_PT], accP[BT_PT];
#pragma unroll
    for (int j = 0; j < BT_PT; ++j) accC[j] = accP[j] = df_make(0.0f, 0.0f);

    for (int k = 0; k <= J.L; ++k) {
        df32 gc[BT_PT], gp[BT_PT];
#pragma unroll
        for (int j = 0; j < BT_PT; ++j) gc[j] = gp[j] = df_make(0.0f, 0.0f);
        for (int s = J.goff[k]; s < J.goff[k + 1]; s += BT_CLS_UNROLL) {
            float4 e[BT_CLS_UNROLL];
#pragma unroll
            for (int i = 0; i < BT_CLS_UNROLL; ++i) e[i] = s_cls[s + i];
#pragma unroll
            for (int j = 0; j < BT_PT; ++j) {
#pragma unroll
                for (int i = 0; i < BT_CLS_UNROLL; ++i) {
                    // tau + f as an unnormalised pair; its sign from the rounded sum
                    const df32 t0 = two_sum(tau[j].hi, e[i].x);
                    const float tl = __fadd_rn(t0.lo, __fadd_rn(tau[j].lo, e[i].y));
                    const float ts = __fadd_rn(t0.hi, tl);
                    if (MODE & BT_MODE_CALL) acc_pair(gc[j], ts > 0.0f ? e[i].z : 0.0f, t0.hi, tl);
                    if (MODE & BT_MODE_PUT) acc_pair(gp[j], ts < 0.0f ? -e[i].z : 0.0f, t0.hi, tl);
                }
            }
        }
        const df32 w = df_from2(P.W2[k]);
#pragma unroll
        for (int j = 0; j < BT_PT; ++j) {
            if (MODE & BT_MODE_CALL) accC[j] = df_add_pos(accC[j], df_mul(w, fast_two_sum(gc[j].hi, gc[j].lo)));
            if (MODE & BT_MODE_PUT) accP[j] = df_add_pos(accP[j], df_mul(w, fast_two_sum(gp[j].hi, gp[j].lo)));
        }
    }
    df32 totC = df_make(0.0f, 0.0f), totP = df_make(0.0f, 0.0f);
#pragma unroll
    for (int j = 0; j < BT_PT; ++j) {
        if (MODE & BT_MODE_CALL) totC = df_add_pos(totC, df_mul(om[j], accC[j]));
        if (MODE & BT_MODE_PUT) totP = df_add_pos(totP, df_mul(om[j], accP[j]));
    }
    double vc = df_to_double(totC), vp = df_to_double(totP);
    if (J.field == BT_F_LOOKMAX) vc += df_to_double(cst);
    if (J.field == BT_F_LOOKMIN) vp += df_to_double(cst);
    double2 sum = block_sum2(vc, vp, red);
    if (threadIdx.x == 0) {
        const double wh = P.wh[__popcll((unsigned long long)item_local)];
        a.partials[J.part_off + item_local] = make_double2(sum.x * wh, sum.y * wh);
    }
}

__global__ void __launch_bounds__(BT_THREADS, 2) k_exact32(bt_exact_args a) {
    extern __shared__ float4 smem_raw[];
    float2 *s_suf = reinterpret_cast<float2 *>(smem_raw);
    __shared__ smem_job sj;
    __shared__ double2 red[BT_THREADS / 32];
    int cur_job = -1;
    while (next_item<float2>(a, sj, s_suf, a.suf32, cur_job)) {
        if (sj.J.cls) {
            switch (sj.J.mode) {
            case BT_MODE_CALL: item32_cls<BT_MODE_CALL>(a, sj, s_suf, red); break;
            case BT_MODE_PUT: item32_cls<BT_MODE_PUT>(a, sj, s_suf, red); break;
            default: item32_cls<BT_MODE_BOTH>(a, sj, s_suf, red); break;
            }
            continue;
        }
        switch (sj.J.mode) {
        case BT_MODE_CALL: item32<BT_MODE_CALL>(a, sj, s_suf, red); break;
        case BT_MODE_PUT: item32<BT_MODE_PUT>(a, sj, s_suf, red); break;
        default: item32<BT_MODE_BOTH>(a, sj, s_suf, red); break;
        }
    }
}

// ---------------------------------------------------------------------------
// All-FP64 variant (the accuracy reference kernel): the same decomposition
// with every step in double precision.
// ---------------------------------------------------------------------------
struct pref64 {
    double tau, om, cst;
};

__device__ __forceinline__ pref64 prefix64(const bt_job &J, const bt_jparams &P, const bt_exact_args &a,
                                           int64_t q, bool valid) {
    pref64 r;
    if (!valid) {
        r.tau = nan("");
        r.om = 0.0;
        r.cst = 0.0;
        return r;
    }
    const int64_t h = q >> J.M;
    const int m = (int)(q & ((1ll << J.M) - 1));
    const bt_pentry eh = a.ph[J.off_ph + h];
    const bt_pentry em = a.pm[J.off_pm + m];
    const int lvl = eh.lvl + em.lvl;
    const bt_pow *pw = a.pw + J.off_pow + J.N + 1;
    double tau, beta, cst = 0.0;
    switch (J.field) {
    case BT_F_ARITH:
        tau = fma(pw[-em.lvl].v, eh.R64, em.R64) - P.NKoS0 * pw[-lvl].v;
        beta = P.S0oN * pw[lvl].v;
        break;
    case BT_F_EURO:
        tau = -P.KoS0 * pw[-lvl].v;
        beta = P.S0 * pw[lvl].v;
        break;
    case BT_F_GEO: {
        const int I = (int)eh.D + J.M * (int)eh.lvl + (int)em.D + J.L * lvl;
        const bt_pow *g = a.pw + J.off_geo - J.geo_imin;
        tau = -P.KoS0 * g[-I].v;
        beta = P.S0 * g[I].v;
        break;
    }
    case BT_F_LOOKMAX: {
        const int lam = max((int)eh.mx, (int)eh.lvl + (int)em.mx);
        const double kk = P.KoS0 * pw[-lvl].v;
        if (lam > -BT_LVL_NONE / 2) {
            tau = -fmax(pw[lam - lvl].v, kk);
            cst = fmax(P.S0 * pw[lam].v - P.K, 0.0);
        } else {
            tau = -kk;
        }
        beta = P.S0 * pw[lvl].v;
        break;
    }
    default: {
        const int lam = min((int)eh.mn, (int)eh.lvl + (int)em.mn);
        const double kk = P.KoS0 * pw[-lvl].v;
        if (lam < BT_LVL_NONE / 2) {
            tau = -fmin(pw[lam - lvl].v, kk);
            cst = fmax(P.K - P.S0 * pw[lam].v, 0.0);
        } else {
            tau = -kk;
        }
        beta = P.S0 * pw[lvl].v;
        break;
    }
    }
    const int c = __popc((unsigned)(q & ((1 << BT_LOW_BITS) - 1)));
    r.tau = tau;
    r.om = P.wl[c] * beta;
    r.cst = P.wl[c] * cst;
    return r;
}

template <int MODE>
__device__ __forceinline__ void item64(const bt_exact_args &a, const smem_job &sj, const double *s_suf,
                                       double2 *red) {
    const bt_job &J = sj.J;
    const bt_jparams &P = sj.P;
    const int64_t item_local = sj.item - J.item_begin + J.item_offset;
    const int64_t qbase = item_local << BT_LOW_BITS;
    const int64_t nP = 1ll << J.P;
    double tau[BT_PT64], om[BT_PT64], cst = 0.0;
#pragma unroll
    for (int j = 0; j < BT_PT64; ++j) {
        const int64_t q = qbase + threadIdx.x + j * BT_THREADS;
        pref64 pr = prefix64(J, P, a, q, q < nP);
        tau[j] = pr.tau;
        om[j] = pr.om;
        cst += pr.cst;
    }
    double accC[BT_PT64], accP[BT_PT64];
#pragma unroll
    for (int j = 0; j < BT_PT64; ++j) accC[j] = accP[j] = 0.0;
    for (int k = 0; k <= J.L; ++k) {
        const int s0 = J.goff[k], s1 = J.goff[k + 1];
        double gc[BT_PT64], gp[BT_PT64];
#pragma unroll
        for (int j = 0; j < BT_PT64; ++j) gc[j] = gp[j] = 0.0;
        for (int s = s0; s < s1; ++s) {
            const double f = s_suf[s];
#pragma unroll
            for (int j = 0; j < BT_PT64; ++j) {
                const double y = tau[j] + f;
                // NaN (padding or a masked prefix) contributes nothing
                if (MODE & BT_MODE_CALL) gc[j] += y > 0.0 ? y : 0.0;
                if (MODE & BT_MODE_PUT) gp[j] += y < 0.0 ? -y : 0.0;
            }
        }
        const double w = P.W[k];
#pragma unroll
        for (int j = 0; j < BT_PT64; ++j) {
            accC[j] = fma(w, gc[j], accC[j]);
            accP[j] = fma(w, gp[j], accP[j]);
        }
    }
    double vc = 0.0, vp = 0.0;
#pragma unroll
    for (int j = 0; j < BT_PT64; ++j) {
        vc = fma(om[j], accC[j], vc);
        vp = fma(om[j], accP[j], vp);
    }
    if (J.field == BT_F_LOOKMAX) vc += cst;
    if (J.field == BT_F_LOOKMIN) vp += cst;
    double2 s = block_sum2(vc, vp, red);
    if (threadIdx.x == 0) {
        const double wh = P.wh[__popcll((unsigned long long)item_local)];
        a.partials[J.part_off + item_local] = make_double2(s.x * wh, s.y * wh);
    }
}

__global__ void __launch_bounds__(BT_THREADS, 2) k_exact64(bt_exact_args a) {
    extern __shared__ double smem_d[];
    __shared__ smem_job sj;
    __shared__ double2 red[BT_THREADS / 32];
    int cur_job = -1;
    while (next_item<double>(a, sj, smem_d, a.suf64, cur_job)) {
        switch (sj.J.mode) {
        case BT_MODE_CALL: item64<BT_MODE_CALL>(a, sj, smem_d, red); break;
        case BT_MODE_PUT: item64<BT_MODE_PUT>(a, sj, smem_d, red); break;
        default: item64<BT_MODE_BOTH>(a, sj, smem_d, red); break;
        }
    }
}

// ---------------------------------------------------------------------------
// Per-option reduction of the block partials in a fixed order (eq. f15)
// ---------------------------------------------------------------------------
struct neu {
    double s, c;
};
__device__ __forceinline__ void neu_add(neu &a, double x) {
    double t = a.s + x;
    if (fabs(a.s) >= fabs(x)) a.c += (a.s - t) + x;
    else a.c += (x - t) + a.s;
    a.s = t;
}

__global__ void k_finalize(const bt_job *jobs, const bt_jparams *prm, int n_jobs, const double2 *partials,
                           int prec, bt_result *out) {
    // one block per job: thread t adds items t, t + BT_THREADS, ... (Neumaier), then a fixed-shape
    // tree over the lanes of each warp and over the warps (many warps keep the FP64 pipe busy where
    // a job has many items)
    __shared__ double sh[4][BT_THREADS / 32];
    const int j = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (j >= n_jobs) return;
    const bt_job J = jobs[j];
    neu c = {0.0, 0.0}, p = {0.0, 0.0};
    for (int64_t i = threadIdx.x; i < J.n_items; i += BT_THREADS) {
        double2 v = partials[J.part_off + i];
        neu_add(c, v.x);
        neu_add(p, v.y);
    }
    for (int o = 16; o > 0; o >>= 1) {
        double cs = __shfl_down_sync(0xffffffffu, c.s, o), cc = __shfl_down_sync(0xffffffffu, c.c, o);
        double ps = __shfl_down_sync(0xffffffffu, p.s, o), pc = __shfl_down_sync(0xffffffffu, p.c, o);
        neu_add(c, cs);
        c.c += cc;
        neu_add(p, ps);
        p.c += pc;
    }
    if (lane == 0) {
        sh[0][warp] = c.s;
        sh[1][warp] = c.c;
        sh[2][warp] = p.s;
        sh[3][warp] = p.c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < BT_THREADS / 32; ++w) {
            neu_add(c, sh[0][w]);
            c.c += sh[1][w];
            neu_add(p, sh[2][w]);
            p.c += sh[3][w];
        }
    }
    if (threadIdx.x == 0) {
        const bt_jparams &P = prm[J.prm_off];
        const double disc = P.disc;
        // stated error: FP64 1e-12; FP32_COMP 1e-9. The host gives the FP32
        // passes that round paths one by one only trees of 2^28 paths or
        // more with at least 2^BT_PER_PATH_MIN_NEFF_LOG2 effective paths
        // (the others go to passes without per-path rounding), where the
        // roundings average under 1e-9; class sums round no single path.
        const double rel = prec == BT_PREC_FP64 ? 1e-12 : 1e-9;
        const int64_t paths = 1ll << J.N;
        if (J.out_call >= 0) {
            bt_result r;
            r.value = disc * (c.s + c.c);
            r.err_est = rel * fabs(r.value);
            r.stderr_mc = 0.0;
            r.var_plain = 0.0;
            r.paths = paths;
            out[J.out_call] = r;
        }
        if (J.out_put >= 0) {
            bt_result r;
            r.value = disc * (p.s + p.c);
            r.err_est = rel * fabs(r.value);
            r.stderr_mc = 0.0;
            r.var_plain = 0.0;
            r.paths = paths;
            out[J.out_put] = r;
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
extern "C" int bt_launch_params(const bt_option *d_opts, const bt_job *d_jobs, bt_jparams *d_prm, int n_jobs,
                                void *stream) {
    if (n_jobs <= 0) return 0;
    k_params<<<(n_jobs + 3) / 4, 128, 0, (cudaStream_t)stream>>>(d_opts, d_jobs, d_prm, n_jobs);   // a warp per job
    return (int)cudaGetLastError();
}

extern "C" int bt_launch_tables(const bt_job *d_jobs, const bt_jparams *d_prm, int n_jobs, int max_len, int prec,
                                float2 *suf32, double *suf64, bt_pentry *ph, bt_pentry *pm, bt_pow *pw,
                                void *stream) {
    if (n_jobs <= 0) return 0;
    int bx = (max_len + 255) / 256;
    if (bx > 64) bx = 64;
    if (bx < 1) bx = 1;
    dim3 grid(bx, n_jobs);
    k_tables<<<grid, 256, 0, (cudaStream_t)stream>>>(d_jobs, d_prm, prec, suf32, suf64, ph, pm, pw, nullptr);
    if (prec == BT_PREC_FP32_COMP)
        k_class_tables<<<n_jobs, 256, 0, (cudaStream_t)stream>>>(d_jobs, d_prm, suf32, nullptr);
    return (int)cudaGetLastError();
}

extern "C" int bt_launch_tables_d(const bt_job *d_jobs, const bt_jparams *d_prm, int n_jobs, int max_len,
                                  float2 *suf32, float *sufd, bt_pentry *ph, bt_pentry *pm, bt_pow *pw,
                                  void *stream) {
    if (n_jobs <= 0) return 0;
    int bx = (max_len + 255) / 256;
    if (bx > 64) bx = 64;
    if (bx < 1) bx = 1;
    dim3 grid(bx, n_jobs);
    k_tables<<<grid, 256, 0, (cudaStream_t)stream>>>(d_jobs, d_prm, BT_PREC_FP32_COMP, suf32, nullptr, ph, pm, pw,
                                                     sufd);
    k_class_tables<<<n_jobs, 256, 0, (cudaStream_t)stream>>>(d_jobs, d_prm, suf32, sufd);
    return (int)cudaGetLastError();
}

static size_t exact_smem(int prec) {
    return prec == BT_PREC_FP64 ? (size_t)BT_SUF_MAX * sizeof(double) : (size_t)BT_SUF_MAX * sizeof(float2);
}

// Persistent grid of the path-sum kernel: SMs x resident blocks. Returns the
// negated cudaError_t if a query fails (the global error state is not read,
// so an earlier error of the caller's own is neither reported nor cleared).
extern "C" int bt_exact_grid_size(int prec, int device) {
    int sms = 0, per = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const size_t sm = exact_smem(prec);
    const void *k = prec == BT_PREC_FP64 ? (const void *)k_exact64 : (const void *)k_exact32;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, BT_THREADS, sm);
    if (e != cudaSuccess) return -(int)e;
    if (per < 1) per = 1;
    if (sms < 1) sms = 1;
    return sms * per;
}

extern "C" int bt_launch_exact(const bt_exact_args *a, int prec, int grid, void *stream) {
    if (a->n_run_items <= 0) return 0;
    if ((int64_t)grid > a->n_run_items) grid = (int)a->n_run_items;
    size_t sm = exact_smem(prec);
    if (prec == BT_PREC_FP64) {
        cudaFuncSetAttribute(k_exact64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_exact64<<<grid, BT_THREADS, sm, (cudaStream_t)stream>>>(*a);
    } else {
        cudaFuncSetAttribute(k_exact32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_exact32<<<grid, BT_THREADS, sm, (cudaStream_t)stream>>>(*a);
    }
    return (int)cudaGetLastError();
}

extern "C" int bt_launch_finalize(const bt_job *d_jobs, const bt_jparams *d_prm, int n_jobs, const double2 *partials,
                                  int shard, int n_shards, int prec, bt_result *d_out, void *stream) {
    (void)shard;
    (void)n_shards;
    if (n_jobs <= 0) return 0;
    k_finalize<<<n_jobs, BT_THREADS, 0, (cudaStream_t)stream>>>(d_jobs, d_prm, n_jobs, partials, prec, d_out);
    return (int)cudaGetLastError();
}
