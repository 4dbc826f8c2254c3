// Trees given move by move: eq. f13 with per-step moves and probabilities, and
// b branches per node (the end of Section 3), sm_103a.
//
// Step t multiplies the price by factor k of that step with probability k
// (digit k = 0..b-1; a time-varying binomial tree is b = 2 with digit 1 = up);
// the tree need not recombine, so every path is evaluated. A path index is N
// digits in base b, the first step most significant. The prefix/suffix
// split of exact.cu still applies, because the suffix steps sit at the same
// positions P+1..N under every prefix: with rho_j(s) = S_{P+j}/S_P the
// suffix's relative prices, each payoff is beta_q max(+-(tau_q + f_s), 0) + C_q
// with f_s = sum_j rho_j (arithmetic Asian), exp(sum_j ln rho_j / N)
// (geometric), rho_L (European), max_j or min_j rho_j (lookback). What
// changes is the weight: w(x) = w_q w_s with w_s the product over the suffix
// of p_t or 1 - p_t, a different number for every suffix. So each path's
// payoff is multiplied by its suffix weight and accumulated in one FMA
// instead of summing an up-count group before one multiplication. A call and
// a put of the same tree and strike share the pass (and the two FMAs of the
// affine form).
//
// Prefix states come from two-level tables over the steps 1..H and H+1..P
// (end factor and its inverse, backward-relative partial sum, extreme
// relative prices, geometric factor and its inverse, weight; FP64 and as FP32
// pairs), composed per prefix in pair arithmetic. The FP32 path keeps the
// rounding design of exact.cu (scaled affine form, exact lambda f_hi + A_hi,
// one rounding per payoff). The weight enters as one FP32 number per suffix,
// rounded from FP64 by error diffusion along ascending f_s (k_steps_weights, in
// 8 interleaved subsequences): the rounding residuals r_s = w_s - w32_s then
// have every partial sum over a run of consecutive f_s bounded by 8 FP32 ulps
// of the largest weight, and
// because a payoff is max(+-(tau + f_s), 0) -- an integral over thresholds of
// the indicator of f_s above (below) the threshold -- sum_s r_s payoff_s is
// bounded by that ulp times the payoff range (summation by parts) instead
// of growing with the number of suffixes.
//
// A job reuses bt_job: off_pow is the index of its first step in the move
// array (2b doubles per step: the b factors, then the b probabilities),
// off_ph and off_pm index the bt_spentry arena, off_suf the suffix arena (4
// floats or 2 doubles per entry), suf_len counts entries (b^L rounded up to a
// multiple of 8; padding has weight 0); n_prefix, n_mid, n_suffix are b^P,
// b^M and b^L.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bt_internal.h"
#include "df.cuh"
#include "exact_common.cuh"

#define BT_SBIG 1.0e30  // the minimum over an empty block

struct sblock {
    double rho, R, sum, mx, mn, lg, w;
};

// Walks `nd` steps of x (base-b digits, the first step most significant)
// whose moves are st[2b (t-1) + k] (factor of digit k) and st[2b (t-1) + b + k]
// (its probability); ext < 0 / > 0 takes every step's smallest / largest
// factor instead. Returns the end factor rho = S_end/S_start, the
// backward-relative partial sum R = sum_t S_t/S_end, the forward-relative sum
// sum_t S_t/S_start, extreme relative prices, sum of ln(S_t/S_start) and the
// block's weight.
__device__ static sblock walk_steps(uint64_t x, int nd, int b, const double *st, int ext = 0) {
    sblock blk;
    double rel = 1.0, R = 0.0, sum = 0.0, mx = 0.0, mn = BT_SBIG, lg = 0.0, w = 1.0;
    uint64_t place = 1;
    for (int t = 1; t < nd; ++t) place *= (uint64_t)b;
    for (int t = 1; t <= nd; ++t, place /= (uint64_t)b) {
        const double *mv = st + 2 * b * (t - 1);
        int k = (int)((x / place) % (uint64_t)b);
        if (ext != 0) {
            k = 0;
            for (int j = 1; j < b; ++j)
                if (ext > 0 ? mv[j] > mv[k] : mv[j] < mv[k]) k = j;
        }
        const double m = mv[k];
        const double p = mv[b + k];
        rel *= m;
        R = R / m + 1.0;
        sum += rel;
        mx = fmax(mx, rel);
        mn = fmin(mn, rel);
        lg += log(rel);
        w *= p;
    }
    blk.rho = rel;
    blk.R = R;
    blk.sum = sum;
    blk.mx = mx;
    blk.mn = mn;
    blk.lg = lg;
    blk.w = w;
    return blk;
}

// f_s of a suffix block for the job's field.
__device__ static double suffix_f(int field, const sblock &b, int N) {
    switch (field) {
    case BT_F_ARITH: return b.sum;
    case BT_F_GEO: return exp(b.lg / (double)N);
    case BT_F_EURO: return b.rho;
    case BT_F_LOOKMAX: return b.mx;
    default: return b.mn;
    }
}

// Parameters of move-by-move jobs: scalars and the suffix f range (every f_s is
// non-decreasing in each step's factor, so the smallest and the largest
// factors of every step bound it).
// One warp per job: the record is zeroed, lanes 0 and 1 walk the suffix extremes (the slow FP64
// work) side by side, lane 0 writes the scalars.
__global__ void k_steps_params(const bt_option *opts, const bt_job *jobs, const double *steps, bt_jparams *prm,
                               int n_jobs) {
    const int j = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= n_jobs) return;
    const bt_job &J = jobs[j];
    const bt_option o = opts[J.opt];
    bt_jparams *P = prm + J.prm_off;
    double *z = reinterpret_cast<double *>(P);
    for (int i = lane; i < (int)(sizeof(bt_jparams) / sizeof(double)); i += 32) z[i] = 0.0;
    __syncwarp();
    const int b = J.branches;
    const double *st = steps + 2 * b * (J.off_pow + J.P);
    double fv = 0.0;
    if (lane < 2) fv = suffix_f(J.field, walk_steps(0, J.L, b, st, lane == 0 ? -1 : +1), J.N);
    const double fmin = __shfl_sync(0xffffffffu, fv, 0), fmax = __shfl_sync(0xffffffffu, fv, 1);
    if (lane != 0) return;
    P->ok = 1;
    P->disc = exp(-o.rate * o.T);
    P->S0 = o.S0;
    P->K = o.K;
    P->NKoS0 = (double)J.N * o.K / o.S0;
    P->KoS0 = o.K / o.S0;
    P->S0oN = o.S0 / (double)J.N;
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

__device__ static bt_spentry make_spentry(const sblock &b, double e) {
    bt_spentry r;
    r.rho = b.rho;
    r.irho = 1.0 / b.rho;
    r.R = b.R;
    r.mx = b.mx;
    r.mn = b.mn;
    r.e = e;
    r.ie = 1.0 / e;
    r.w = b.w;
    r.rho2 = split2(r.rho);
    r.irho2 = split2(r.irho);
    r.R2 = split2(r.R);
    r.mx2 = split2(r.mx);
    r.mn2 = split2(r.mn);
    r.e2 = split2(r.e);
    r.ie2 = split2(r.ie);
    r.w2 = split2(r.w);
    return r;
}

// Tables of move-by-move jobs: suffix entries (f, w) and the two prefix
// tables. The geometric factor of a prefix block folds in the later steps
// that inherit its end price: e_h = exp((lg_h + (M + L) ln rho_h)/N) for the
// first block, e_m = exp((lg_m + L ln rho_m)/N) for the second.
__global__ void k_steps_tables(const bt_job *jobs, const bt_jparams *prm, const double *steps, int prec,
                               float4 *suf32, double2 *suf64, bt_spentry *tab) {
    const bt_job J = jobs[blockIdx.y];
    const bt_jparams &Pj = prm[J.prm_off];
    const int b = J.branches;
    const double *st = steps + 2 * b * J.off_pow;
    const int64_t nsuf = J.n_suffix, nh = J.n_prefix / J.n_mid, nm = J.n_mid;
    const int64_t total = J.suf_len + nh + nm;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx;
        if (i < J.suf_len) {
            double f = 0.0, w = 0.0;  // padding: weight 0
            if (i < nsuf) {
                const sblock s = walk_steps((uint64_t)i, J.L, b, st + 2 * b * J.P);
                f = suffix_f(J.field, s, J.N);
                w = s.w;
            }
            if (prec == BT_PREC_FP64) {
                suf64[J.off_suf + i] = make_double2(f, w);
            } else {
                const int gx = Pj.gexp;
                const double fh = ldexp(rint(ldexp(f, -gx)), gx);
                const float2 w2 = split2(w);
                suf32[J.off_suf + i] = make_float4((float)fh, -(float)(f - fh), w2.x, w2.y);
            }
            continue;
        }
        i -= J.suf_len;
        if (i < nh) {
            const sblock s = walk_steps((uint64_t)i, J.H, b, st);
            const double e = exp((s.lg + (double)(J.M + J.L) * log(s.rho)) / (double)J.N);
            tab[J.off_ph + i] = make_spentry(s, e);
            continue;
        }
        i -= nh;
        const sblock s = walk_steps((uint64_t)i, J.M, b, st + 2 * b * J.H);
        const double e = exp((s.lg + (double)J.L * log(s.rho)) / (double)J.N);
        tab[J.off_pm + i] = make_spentry(s, e);
    }
}

// FP32 suffix weights by error diffusion (one block per job, FP32 tables):
// the entries (f_hi, -f_lo, w_hi, w_lo) written by k_steps_tables are sorted
// by f = f_hi + f_lo (bitonic sort on the bit patterns of the FP64 values, which
// order like the values since every f_s > 0, with the suffix index in the low 13
// bits; padding keys after every suffix), then BT_DIFFUSE_LANES lanes of one warp each walk one of
// the interleaved subsequences r = lane, lane + BT_DIFFUSE_LANES, ... (each in
// ascending f) carrying the rounding residual: w32 = RN_f32(w + carry),
// carry = w + carry - w32, with w the FP32 pair (w_hi, w_lo) and the carry kept
// exactly by error-free sums (TwoSum, Fast2Sum), so that the residuals of any
// run of consecutive f telescope, per subsequence, to the difference of two
// carries, each at most half an FP32 ulp: BT_DIFFUSE_LANES ulps at most over
// the run. A weight of 0 (a branch of probability 0) stays 0. The entry keeps
// (f_hi, -f_lo, w32, 0).
// Compare-exchange of a thread's eight keys at distance J < 8 (element 8t + r against 8t + (r ^ J)),
// ascending where the element's bit k is clear.
template <int J>
__device__ __forceinline__ void sort_in_thread(unsigned long long (&v)[8], int k) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        if ((r ^ J) > r) {
            const bool asc = ((8 * (int)threadIdx.x + r) & k) == 0;
            const unsigned long long a = v[r], b = v[r ^ J];
            const unsigned long long lo = a < b ? a : b, hi = a < b ? b : a;
            v[r] = asc ? lo : hi;
            v[r ^ J] = asc ? hi : lo;
        }
    }
}

#ifndef BT_DIFFUSE_LANES
#define BT_DIFFUSE_LANES 8
#endif
static_assert(BT_DIFFUSE_LANES >= 1 && BT_DIFFUSE_LANES <= 32, "diffusion lanes of one warp");
#define BT_SORT_N (1 << BT_STEPS32_MAX_L)
#define BT_SORT_SMEM ((size_t)BT_SORT_N * (sizeof(unsigned long long) + sizeof(int16_t)))
__global__ void __launch_bounds__(1024) k_steps_weights(const bt_job *jobs, float4 *suf32) {
    const bt_job J = jobs[blockIdx.x];
    extern __shared__ unsigned long long key[];   // [BT_SORT_N], then idx
    int16_t *idx = reinterpret_cast<int16_t *>(key + BT_SORT_N);
    const int n = (int)J.n_suffix;
    float4 *tab = suf32 + J.off_suf;
    // Bitonic sort of BT_SORT_N keys, eight per thread in registers (thread t holds elements
    // 8t..8t+7): compare-exchange partners 8 or more apart but in the same warp come by shuffle,
    // those 256 or more apart through shared memory, the rest are in the same thread. A key is the
    // bit pattern of f (which orders like f, every f > 0) with its low 13 bits replaced by the
    // suffix index (so ties and f within 2^-39 relative of each other order by index); padding
    // keys are all ones.
    static_assert(BT_SORT_N == 8 * 1024 && BT_SORT_N <= (1 << 13), "eight keys per thread, 13-bit index");
    constexpr unsigned long long IDX = (1ull << 13) - 1;
    unsigned long long v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int e = 8 * threadIdx.x + r;
        if (e < n) {
            const float4 t = tab[e];
            v[r] = ((unsigned long long)__double_as_longlong((double)t.x - (double)t.y) & ~IDX) | (unsigned long long)e;
        } else {
            v[r] = ~0ull;
        }
    }
    for (int k = 2; k <= BT_SORT_N; k <<= 1) {
        for (int j = k >> 1; j >= 8; j >>= 1) {
            if (j >= 256) {
                __syncthreads();   // the previous exchange's reads are done
#pragma unroll
                for (int r = 0; r < 8; ++r) key[8 * threadIdx.x + r] = v[r];
                __syncthreads();
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int e = 8 * threadIdx.x + r;
                    const unsigned long long w = key[e ^ j];
                    const bool keep_min = ((e & k) == 0) == ((e & j) == 0);
                    v[r] = keep_min ? (v[r] < w ? v[r] : w) : (v[r] > w ? v[r] : w);
                }
            } else if (j >= 8) {
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int e = 8 * threadIdx.x + r;
                    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v[r], j >> 3);
                    const bool keep_min = ((e & k) == 0) == ((e & j) == 0);
                    v[r] = keep_min ? (v[r] < w ? v[r] : w) : (v[r] > w ? v[r] : w);
                }
            }
        }
        if (k >= 8) sort_in_thread<4>(v, k);   // j < 8: the partner is a register of this thread
        if (k >= 4) sort_in_thread<2>(v, k);
        sort_in_thread<1>(v, k);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) idx[8 * threadIdx.x + r] = (int16_t)(v[r] & IDX);
    __syncthreads();   // every exchange read of key[] is done before it holds the weights
    float2 *wp = reinterpret_cast<float2 *>(key);   // the keys are no longer needed
    for (int r = threadIdx.x; r < n; r += blockDim.x) {   // the weights in ascending f
        const float4 e = tab[idx[r]];
        wp[r] = make_float2(e.z, e.w);
    }
    __syncthreads();
    if (threadIdx.x < BT_DIFFUSE_LANES) {
        float carry = 0.0f;
        for (int r = threadIdx.x; r < n; r += BT_DIFFUSE_LANES) {
            const float2 w = wp[r];
            if (w.x == 0.0f) continue;               // probability 0: weight 0, carry kept
            const df32 t = two_sum(w.x, carry);      // w_hi + carry, exactly
            const float lo = __fadd_rn(t.lo, w.y);   // + w_lo (error 2^-24 of a 2^-24 term)
            const float h = __fadd_rn(t.hi, lo);     // the target rounded once to FP32
            carry = __fsub_rn(lo, __fsub_rn(h, t.hi));   // Fast2Sum remainder (|t.hi| >= |lo|)
            wp[r].x = h;
        }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        float4 &e = tab[idx[r]];
        e.z = wp[r].x;
        e.w = 0.0f;
    }
}

// Per-prefix affine form and weight in FP32 pairs.
struct sstate {
    df32 tau, beta, cst, w;
};
__device__ __forceinline__ sstate steps_state(const bt_job &J, const bt_jparams &P, const bt_spentry *tab,
                                              int64_t q) {
    const bt_spentry &eh = tab[J.off_ph + q / J.n_mid];
    const bt_spentry &em = tab[J.off_pm + q % J.n_mid];
    sstate r;
    const df32 rho_h = df_from2(eh.rho2), rho_m = df_from2(em.rho2);
    const df32 ir = df_mul(df_from2(eh.irho2), df_from2(em.irho2));  // S0 / S_P
    const df32 sp = df_mul(rho_h, rho_m);                              // S_P / S0
    const df32 kk = df_from2(P.KoS0_2);
    r.cst = df_make(0.0f, 0.0f);
    switch (J.field) {
    case BT_F_ARITH:
        // Sigma_P / S_P = R_h / rho_m + R_m
        r.tau = df_sub(df_add(df_mul(df_from2(eh.R2), df_from2(em.irho2)), df_from2(em.R2)),
                       df_mul(df_from2(P.NKoS0_2), ir));
        r.beta = df_mul(df_from2(P.S0oN_2), sp);
        break;
    case BT_F_EURO:
        r.tau = df_neg(df_mul(kk, ir));
        r.beta = df_mul(df_from2(P.S0_2), sp);
        break;
    case BT_F_GEO:
        r.tau = df_neg(df_mul(kk, df_mul(df_from2(eh.ie2), df_from2(em.ie2))));
        r.beta = df_mul(df_from2(P.S0_2), df_mul(df_from2(eh.e2), df_from2(em.e2)));
        break;
    case BT_F_LOOKMAX: {
        // M_P / S0 = max(mx_h, rho_h mx_m); tau = -max(M_P, K) / S_P, C = max(M_P - K, 0)
        const df32 a = df_from2(eh.mx2), b = df_mul(rho_h, df_from2(em.mx2));
        const df32 mr = df_gt(a, b) ? a : b;
        r.tau = df_neg(df_mul(df_gt(mr, kk) ? mr : kk, ir));
        if (df_gt(mr, kk)) r.cst = df_mul(df_from2(P.S0_2), df_sub(mr, kk));
        r.beta = df_mul(df_from2(P.S0_2), sp);
        break;
    }
    default: {
        const df32 a = df_from2(eh.mn2), b = df_mul(rho_h, df_from2(em.mn2));
        const df32 mr = df_gt(a, b) ? b : a;
        r.tau = df_neg(df_mul(df_gt(mr, kk) ? kk : mr, ir));
        if (df_gt(kk, mr)) r.cst = df_mul(df_from2(P.S0_2), df_sub(kk, mr));
        r.beta = df_mul(df_from2(P.S0_2), sp);
        break;
    }
    }
    r.w = df_mul(df_from2(eh.w2), df_from2(em.w2));
    return r;
}

// Weighted payoffs/lambda of eight suffixes under one prefix: per suffix
// y = lambda f_hi + A_hi (exact), c = lambda (-f_lo) - A_lo, z = sat(+-(y - c))
// (call: y - c, put: c - y), accumulated as w32 z by a chain of FMAs; a
// call and a put share y and c.
// The FP32 suffix table in shared memory: three arrays of BT_STEPS32_SUF floats (f_hi, -f_lo, w32)
// read four suffixes per 16-byte load.
#define BT_STEPS32_SUF (1 << BT_STEPS32_MAX_L)
#define BT_STEPS32_SMEM ((size_t)3 * BT_STEPS32_SUF * sizeof(float))
struct suf_soa {
    const float *fh, *nfl, *w;
};
struct suf8 {
    float fh[BT_UNROLL], nfl[BT_UNROLL], w[BT_UNROLL];
};
static_assert(BT_UNROLL == 8, "two float4 loads per array and chain");
__device__ __forceinline__ void load8(const suf_soa &t, int s, suf8 &v) {
    // s is a multiple of 8 (the table is padded to whole chains), so the float4 loads are aligned
    *reinterpret_cast<float4 *>(&v.fh[0]) = *reinterpret_cast<const float4 *>(t.fh + s);
    *reinterpret_cast<float4 *>(&v.fh[4]) = *reinterpret_cast<const float4 *>(t.fh + s + 4);
    *reinterpret_cast<float4 *>(&v.nfl[0]) = *reinterpret_cast<const float4 *>(t.nfl + s);
    *reinterpret_cast<float4 *>(&v.nfl[4]) = *reinterpret_cast<const float4 *>(t.nfl + s + 4);
    *reinterpret_cast<float4 *>(&v.w[0]) = *reinterpret_cast<const float4 *>(t.w + s);
    *reinterpret_cast<float4 *>(&v.w[4]) = *reinterpret_cast<const float4 *>(t.w + s + 4);
}
template <int MODE>
__device__ __forceinline__ void wchain8(const suf8 &v, float B, float Ah, float nAl, float &tc, float &tp) {
    float ac = 0.0f, ap = 0.0f;
#pragma unroll
    for (int i = 0; i < BT_UNROLL; ++i) {
        const float y = __fmaf_rn(B, v.fh[i], Ah);
        const float c = __fmaf_rn(B, v.nfl[i], nAl);
        if (MODE & BT_MODE_CALL) ac = __fmaf_rn(v.w[i], __saturatef(__fsub_rn(y, c)), ac);
        if (MODE & BT_MODE_PUT) ap = __fmaf_rn(v.w[i], __saturatef(__fsub_rn(c, y)), ap);
    }
    tc = ac;
    tp = ap;
}

// g + t as (sum, compensation): Fast2Sum (|g| >= |t| after the first add).
__device__ __forceinline__ void fast_acc_s(float &g, float &e, float t) {
    const float sN = __fadd_rn(g, t);
    e = __fadd_rn(e, __fsub_rn(t, __fsub_rn(sN, g)));
    g = sN;
}

// One work item, FP32: eight-suffix FMA chains of weighted payoffs, eight
// chains added in turn per Fast2Sum into the prefix's running sum; prefixes
// combined in pairs (w beta / lambda and C recomputed after the loop), the
// block in FP64.
template <int MODE>
__device__ __forceinline__ void item_steps32(const bt_exact_args &a, const smem_job &sj, const suf_soa &s_suf,
                                             const bt_spentry *tab, double2 *red) {
    const bt_job &J = sj.J;
    const bt_jparams &P = sj.P;
    const int64_t item_local = sj.item - J.item_begin + J.item_offset;
    const int64_t qbase = item_local << BT_LOW_BITS;
    const int64_t nP = J.n_prefix;
    float B[BT_PT], Ah[BT_PT], nAl[BT_PT];
#pragma unroll
    for (int j = 0; j < BT_PT; ++j) {
        const int64_t q = qbase + threadIdx.x + j * BT_THREADS;
        if (q < nP) {
            const scale32 sc = scale_prefix(steps_state(J, P, tab, q).tau, P, q);
            B[j] = sc.B;
            Ah[j] = sc.Ah;
            nAl[j] = sc.nAl;
        } else {
            B[j] = 0.0f;
            Ah[j] = nAl[j] = __int_as_float(0x7fc00000);  // sat(NaN) = 0
        }
    }
    float gc[BT_PT], ec[BT_PT], gp[BT_PT], ep[BT_PT];
#pragma unroll
    for (int j = 0; j < BT_PT; ++j) gc[j] = ec[j] = gp[j] = ep[j] = 0.0f;
    int s = 0;
    for (; s + 8 * BT_UNROLL <= J.suf_len; s += 8 * BT_UNROLL) {
        float tc[BT_PT], tp[BT_PT];
#pragma unroll
        for (int j = 0; j < BT_PT; ++j) tc[j] = tp[j] = 0.0f;
#pragma unroll 2
        for (int r = 0; r < 8; ++r) {
            suf8 v;
            load8(s_suf, s + r * BT_UNROLL, v);
#pragma unroll
            for (int j = 0; j < BT_PT; ++j) {
                float uc, up;
                wchain8<MODE>(v, B[j], Ah[j], nAl[j], uc, up);
                if (MODE & BT_MODE_CALL) tc[j] = __fadd_rn(tc[j], uc);
                if (MODE & BT_MODE_PUT) tp[j] = __fadd_rn(tp[j], up);
            }
        }
#pragma unroll
        for (int j = 0; j < BT_PT; ++j) {
            if (MODE & BT_MODE_CALL) fast_acc_s(gc[j], ec[j], tc[j]);
            if (MODE & BT_MODE_PUT) fast_acc_s(gp[j], ep[j], tp[j]);
        }
    }
    for (; s < J.suf_len; s += BT_UNROLL) {
        suf8 v;
        load8(s_suf, s, v);
#pragma unroll
        for (int j = 0; j < BT_PT; ++j) {
            float uc, up;
            wchain8<MODE>(v, B[j], Ah[j], nAl[j], uc, up);
            if (MODE & BT_MODE_CALL) fast_acc_s(gc[j], ec[j], uc);
            if (MODE & BT_MODE_PUT) fast_acc_s(gp[j], ep[j], up);
        }
    }
    df32 totC = df_make(0.0f, 0.0f), totP = df_make(0.0f, 0.0f), cst = df_make(0.0f, 0.0f);
#pragma unroll
    for (int j = 0; j < BT_PT; ++j) {
        const int64_t q = qbase + threadIdx.x + j * BT_THREADS;
        if (q >= nP) continue;
        const sstate st = steps_state(J, P, tab, q);
        const scale32 sc = scale_prefix(st.tau, P, q);
        const df32 om = df_mul(df_mul(st.w, st.beta), sc.rinv);
        if (MODE & BT_MODE_CALL) totC = df_add_pos(totC, df_mul(om, fast_two_sum(gc[j], ec[j])));
        if (MODE & BT_MODE_PUT) totP = df_add_pos(totP, df_mul(om, fast_two_sum(gp[j], ep[j])));
        cst = df_add_pos(cst, df_mul(st.w, st.cst));
    }
    double vc = df_to_double(totC), vp = df_to_double(totP);
    if (J.field == BT_F_LOOKMAX) vc += df_to_double(cst);
    if (J.field == BT_F_LOOKMIN) vp += df_to_double(cst);
    const double2 sum = block_sum2(vc, vp, red);
    if (threadIdx.x == 0) a.partials[J.part_off + item_local] = sum;
}

// One work item, FP64 (the accuracy reference): y = tau + f, payoff/beta =
// max(+-y, 0), weighted by w_s with one FMA.
template <int MODE>
__device__ __forceinline__ void item_steps64(const bt_exact_args &a, const smem_job &sj, const double2 *s_suf,
                                             const bt_spentry *tab, double2 *red) {
    const bt_job &J = sj.J;
    const bt_jparams &P = sj.P;
    const int64_t item_local = sj.item - J.item_begin + J.item_offset;
    const int64_t qbase = item_local << BT_LOW_BITS;
    const int64_t nP = J.n_prefix;
    double tau[BT_PT64], om[BT_PT64], cst = 0.0;
#pragma unroll
    for (int j = 0; j < BT_PT64; ++j) {
        const int64_t q = qbase + threadIdx.x + j * BT_THREADS;
        tau[j] = nan("");
        om[j] = 0.0;
        if (q >= nP) continue;
        const bt_spentry &eh = tab[J.off_ph + q / J.n_mid];
        const bt_spentry &em = tab[J.off_pm + q % J.n_mid];
        const double ir = eh.irho * em.irho, sp = eh.rho * em.rho, w = eh.w * em.w;
        double beta = P.S0 * sp, c = 0.0;
        switch (J.field) {
        case BT_F_ARITH:
            tau[j] = fma(eh.R, em.irho, em.R) - P.NKoS0 * ir;
            beta = P.S0oN * sp;
            break;
        case BT_F_EURO: tau[j] = -P.KoS0 * ir; break;
        case BT_F_GEO:
            tau[j] = -P.KoS0 * eh.ie * em.ie;
            beta = P.S0 * eh.e * em.e;
            break;
        case BT_F_LOOKMAX: {
            const double mr = fmax(eh.mx, eh.rho * em.mx);
            tau[j] = -fmax(mr, P.KoS0) * ir;
            c = fmax(P.S0 * mr - P.K, 0.0);
            break;
        }
        default: {
            const double mr = fmin(eh.mn, eh.rho * em.mn);
            tau[j] = -fmin(mr, P.KoS0) * ir;
            c = fmax(P.K - P.S0 * mr, 0.0);
            break;
        }
        }
        om[j] = w * beta;
        cst += w * c;
    }
    double accC[BT_PT64], accP[BT_PT64];
#pragma unroll
    for (int j = 0; j < BT_PT64; ++j) accC[j] = accP[j] = 0.0;
    for (int s = 0; s < J.suf_len; ++s) {
        const double2 fw = s_suf[s];
#pragma unroll
        for (int j = 0; j < BT_PT64; ++j) {
            const double y = tau[j] + fw.x;
            // NaN (a masked prefix) contributes nothing
            if (MODE & BT_MODE_CALL) accC[j] = fma(fw.y, y > 0.0 ? y : 0.0, accC[j]);
            if (MODE & BT_MODE_PUT) accP[j] = fma(fw.y, y < 0.0 ? -y : 0.0, accP[j]);
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
    const double2 sum = block_sum2(vc, vp, red);
    if (threadIdx.x == 0) a.partials[J.part_off + item_local] = sum;
}

__global__ void __launch_bounds__(BT_THREADS, 2) k_steps32(bt_exact_args a, const bt_spentry *tab) {
    extern __shared__ float4 s_suf4[];   // BT_STEPS32_SMEM bytes: f_hi, -f_lo, w32 arrays
    float *const s_f = reinterpret_cast<float *>(s_suf4);
    const suf_soa t = {s_f, s_f + BT_STEPS32_SUF, s_f + 2 * BT_STEPS32_SUF};
    __shared__ smem_job sj;
    __shared__ double2 red[BT_THREADS / 32];
    int cur_job = -1;
    const float4 *g_suf = reinterpret_cast<const float4 *>(a.suf32);
    // the job's (f_hi, -f_lo, w32, 0) entries split into the three arrays
    auto load = [&](const bt_job &J) {
        for (int i = threadIdx.x; i < J.suf_len; i += BT_THREADS) {
            const float4 e = g_suf[J.off_suf + i];
            s_f[i] = e.x;
            s_f[BT_STEPS32_SUF + i] = e.y;
            s_f[2 * BT_STEPS32_SUF + i] = e.z;
        }
    };
    while (next_item_with(a, sj, cur_job, load)) {
        switch (sj.J.mode) {
        case BT_MODE_CALL: item_steps32<BT_MODE_CALL>(a, sj, t, tab, red); break;
        case BT_MODE_PUT: item_steps32<BT_MODE_PUT>(a, sj, t, tab, red); break;
        default: item_steps32<BT_MODE_BOTH>(a, sj, t, tab, red); break;
        }
    }
}

__global__ void __launch_bounds__(BT_THREADS, 2) k_steps64(bt_exact_args a, const bt_spentry *tab) {
    extern __shared__ double2 s_suf2[];
    __shared__ smem_job sj;
    __shared__ double2 red[BT_THREADS / 32];
    int cur_job = -1;
    while (next_item<double2>(a, sj, s_suf2, reinterpret_cast<const double2 *>(a.suf64), cur_job)) {
        switch (sj.J.mode) {
        case BT_MODE_CALL: item_steps64<BT_MODE_CALL>(a, sj, s_suf2, tab, red); break;
        case BT_MODE_PUT: item_steps64<BT_MODE_PUT>(a, sj, s_suf2, tab, red); break;
        default: item_steps64<BT_MODE_BOTH>(a, sj, s_suf2, tab, red); break;
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
#define BT_STEPS_SMEM ((size_t)(1 << BT_STEPS_MAX_L) * 16)

extern "C" int bt_launch_steps_params(const bt_option *d_opts, const bt_job *d_jobs, const double *d_steps,
                                      bt_jparams *d_prm, int n_jobs, void *stream) {
    if (n_jobs <= 0) return 0;
    k_steps_params<<<(n_jobs + 3) / 4, 128, 0, (cudaStream_t)stream>>>(d_opts, d_jobs, d_steps, d_prm, n_jobs);   // a warp per job
    return (int)cudaGetLastError();
}

extern "C" int bt_launch_steps_tables(const bt_job *d_jobs, const bt_jparams *d_prm, const double *d_steps,
                                      int n_jobs, int max_len, int prec, float4 *suf32, double2 *suf64,
                                      bt_spentry *tab, void *stream) {
    if (n_jobs <= 0) return 0;
    int bx = (max_len + 255) / 256;
    if (bx > 64) bx = 64;
    if (bx < 1) bx = 1;
    dim3 grid(bx, n_jobs);
    k_steps_tables<<<grid, 256, 0, (cudaStream_t)stream>>>(d_jobs, d_prm, d_steps, prec, suf32, suf64, tab);
    if (prec == BT_PREC_FP32_COMP) {
        cudaError_t e = cudaFuncSetAttribute(k_steps_weights, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)BT_SORT_SMEM);
        if (e != cudaSuccess) return (int)e;
        k_steps_weights<<<n_jobs, 1024, BT_SORT_SMEM, (cudaStream_t)stream>>>(d_jobs, suf32);
    }
    return (int)cudaGetLastError();
}

// Persistent grid: SMs x resident blocks at the full suffix table size.
extern "C" int bt_launch_steps(const bt_exact_args *a, const bt_spentry *tab, int prec, int device, void *stream) {
    if (a->n_run_items <= 0) return 0;
    const void *k = prec == BT_PREC_FP64 ? (const void *)k_steps64 : (const void *)k_steps32;
    const size_t smem = prec == BT_PREC_FP64 ? BT_STEPS_SMEM : BT_STEPS32_SMEM;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, BT_THREADS, smem);
    if (e != cudaSuccess) return (int)e;
    if (per < 1) per = 1;
    int64_t grid = (int64_t)sms * per;
    if (grid > a->n_run_items) grid = a->n_run_items;
    if (prec == BT_PREC_FP64)
        k_steps64<<<(unsigned)grid, BT_THREADS, smem, (cudaStream_t)stream>>>(*a, tab);
    else
        k_steps32<<<(unsigned)grid, BT_THREADS, smem, (cudaStream_t)stream>>>(*a, tab);
    return (int)cudaGetLastError();
}
