// Partitioned (stratified) and Shared-Sample Monte Carlo (Section 4), sm_103a.
//
// Stratum m in [0, 2^mb) fixes the first mb steps of the path to the bits of m,
// most significant first (the rank bits of Section 3). Each stratum draws R
// suffixes of N - mb Bernoulli(p) steps; step t of sample i in stratum m takes
// word (t-mb-1) % 4 of Philox-4x32-10(counter = ((t-mb-1)/4, i, m, stream),
// key = (seed_lo, seed_hi)) and goes up iff that word is below
// thr = round(p 2^32). The Shared-Sample estimator (Remark of Section 4) uses
// counter word 2 = 0 for every stratum, i.e. the same R suffixes under every
// prefix. A work item is 1024 consecutive samples of one stratum: one warp
// runs it in the Partitioned kernel (k_mc_warp), one block in the
// Shared-Sample kernel (k_mc_shared, whose strata table, written once per job by
// k_mc_shared_tab, sits in shared memory).
// Per-item (count, mean, M2) go to scratch and are combined per stratum
// (Chan et al.'s pairwise update) and then across strata in FP64 (eq. mc12
// and its variance). A shard runs the strata m = shard + j n_shards only.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bt_internal.h"
#include "mc_internal.h"

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplications whose high halves are xored with the other words and the
// round key; the key advances by the Weyl constants each round.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // high and low halves of the two 32x32 products as separate 32-bit multiplies (measured
        // slightly faster than one 64-bit wide multiply each, and 8 registers fewer)
        const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

extern "C" __global__ void k_philox_selftest(const uint4 *ctr, const uint2 *key, uint4 *out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], key[i]);
}

// Prefix (stratum) state in FP64: tau, beta, C of the affine form
// payoff = beta * max(+-(tau + f), 0) + C, as in the exhaustive kernels.
struct mc_pref {
    double tau, beta, C, prob;
};

__device__ static mc_pref stratum_state(const bt_mc_job &J, uint64_t m) {
    const int mb = J.mb, N = J.N, L = N - mb;
    const double u = J.u, d = J.d, lnu = log(u);
    int lvl = 0, mx = -BT_LVL_NONE, mn = BT_LVL_NONE, D = 0, k = 0;
    double R = 0.0;  // Sigma_P / S_P as sum_t u^{l_t - l_P}
    for (int t = 1; t <= mb; ++t) {
        const int up = (int)((m >> (mb - t)) & 1u);
        k += up;
        lvl += up ? 1 : -1;
        R = R * (up ? d : u) + 1.0;
        mx = lvl > mx ? lvl : mx;
        mn = lvl < mn ? lvl : mn;
        D += lvl;
    }
    mc_pref s;
    s.prob = J.prob_k[k];
    const double SP = J.S0 * exp((double)lvl * lnu);
    s.C = 0.0;
    switch (J.field) {
    case BT_F_ARITH:
        s.tau = R - (double)N * J.K / SP;
        s.beta = SP / (double)N;
        break;
    case BT_F_EURO:
        s.tau = -J.K / SP;
        s.beta = SP;
        break;
    case BT_F_GEO: {
        const double g = J.S0 * exp((double)(D + L * lvl) * lnu / (double)N);
        s.tau = -J.K / g;
        s.beta = g;
        break;
    }
    case BT_F_LOOKMAX:
        if (mb > 0) {
            const double M = J.S0 * exp((double)mx * lnu);
            s.tau = -fmax(M, J.K) / SP;
            s.C = fmax(M - J.K, 0.0);
        } else {
            s.tau = -J.K / SP;
        }
        s.beta = SP;
        break;
    default:
        if (mb > 0) {
            const double M = J.S0 * exp((double)mn * lnu);
            s.tau = -fmin(M, J.K) / SP;
            s.C = fmax(J.K - M, 0.0);
        } else {
            s.tau = -J.K / SP;
        }
        s.beta = SP;
        break;
    }
    return s;
}

// Suffix state while walking: relative price and partial sum (arithmetic),
// or integer level, extreme level and level sum (the other payoffs).
template <int FIELD>
struct walker {
    float rel = 1.0f, f = 0.0f;
    int lvl = 0, ext = FIELD == BT_F_LOOKMAX ? -BT_LVL_NONE : BT_LVL_NONE, D = 0;
    __device__ __forceinline__ void step(bool up, float uf, float df) {
        if (FIELD == BT_F_ARITH) {
            rel *= up ? uf : df;
            f += rel;
        } else {
            step_level(up);
        }
    }
    // The arithmetic step from the Philox word itself: up iff word < thr. The factor is applied by
    // two predicated multiplies (FMA pipe) instead of a select (ALU pipe, the busier one here) and
    // one multiply; the same IEEE product either way (BT_MC_SELECT_MUL builds the select form).
    __device__ __forceinline__ void step_word(unsigned word, unsigned thr, float uf, float df) {
#ifndef BT_MC_SELECT_MUL
        if (FIELD == BT_F_ARITH) {
            asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p mul.rn.f32 %0, %0, %3;\n\t"
                "@!p mul.rn.f32 %0, %0, %4;\n\t}"
                : "+f"(rel)
                : "r"(word), "r"(thr), "f"(uf), "f"(df));
            f += rel;
            return;
        }
#endif
        step(word < thr, uf, df);
    }
    __device__ __forceinline__ void step_level(bool up) {
        lvl += up ? 1 : -1;
        if (FIELD == BT_F_GEO) D += lvl;
        if (FIELD == BT_F_LOOKMAX) ext = lvl > ext ? lvl : ext;
        if (FIELD == BT_F_LOOKMIN) ext = lvl < ext ? lvl : ext;
    }
    // The per-suffix number f (see exact.cu): arithmetic sum_j u^{l'_j},
    // geometric u^{sum_j l'_j / N}, European u^{l'_L}, lookback u^{max/min l'_j};
    // an empty suffix (L = 0) gives the value that leaves only the prefix.
    __device__ __forceinline__ float value(const bt_mc_job &J, int L) const {
        switch (FIELD) {
        case BT_F_ARITH: return f;
        case BT_F_GEO: return expf((float)D * J.lnu_f / (float)J.N);
        case BT_F_EURO: return expf((float)lvl * J.lnu_f);
        case BT_F_LOOKMAX: return L > 0 ? expf((float)ext * J.lnu_f) : 0.0f;
        default: return L > 0 ? expf((float)ext * J.lnu_f) : 3.0e38f;
        }
    }
};

// Simulates the suffixes of W samples together (W independent Philox streams
// per thread, for instruction-level parallelism).
template <int FIELD, int W>
__device__ __forceinline__ void simulate_w(const bt_mc_job &J, const unsigned (&idx)[W], unsigned c2, float (&f)[W],
                                           uint2 key) {
    const int L = J.N - J.mb;
    walker<FIELD> A[W];
    const int L4 = L & ~3;
    int j0 = 0;
    for (; j0 < L4; j0 += 4) {  // whole blocks of four steps, no per-step bound test
        uint4 r[W];
#pragma unroll
        for (int w = 0; w < W; ++w) r[w] = philox4x32_10(make_uint4((unsigned)(j0 >> 2), idx[w], c2, J.stream), key);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            A[w].step_word(r[w].x, J.thr, J.uf, J.df);
            A[w].step_word(r[w].y, J.thr, J.uf, J.df);
            A[w].step_word(r[w].z, J.thr, J.uf, J.df);
            A[w].step_word(r[w].w, J.thr, J.uf, J.df);
        }
    }
    if (j0 < L) {  // the last one to three steps: words 0..L-j0-1 of the final block
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint4 r = philox4x32_10(make_uint4((unsigned)(j0 >> 2), idx[w], c2, J.stream), key);
            const unsigned wd[3] = {r.x, r.y, r.z};
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (j0 + q < L) A[w].step(wd[q] < J.thr, J.uf, J.df);
        }
    }
#pragma unroll
    for (int w = 0; w < W; ++w) f[w] = A[w].value(J, L);
}

#ifndef BT_MC_WALKERS
#define BT_MC_WALKERS 8   // samples per thread at once in the Partitioned kernel (measured: 2 < 4 < 8)
#endif
#ifndef BT_MC_WARP_THREADS
#define BT_MC_WARP_THREADS 256   // block size of the Partitioned kernel (its warps are independent)
#endif
#ifndef BT_MC_MIN_BLOCKS
#define BT_MC_MIN_BLOCKS 2   // resident blocks per SM the Partitioned kernel is compiled for
#endif

__device__ __forceinline__ float payoff_of(const bt_mc_job &J, float tau, float beta, float C, float f) {
    const float y = tau + f;
    const float z = J.sign > 0 ? fmaxf(y, 0.0f) : fmaxf(-y, 0.0f);
    return fmaf(beta, z, C);
}

// Chan et al. combination of (n, mean, M2) summaries.
__device__ __forceinline__ void chan(float &n, float &mean, float &M2, float nb, float meanb, float M2b) {
    const float nn = n + nb;
    if (nn == 0.0f) return;
    const float delta = meanb - mean;
    mean = mean + delta * (nb / nn);
    M2 = M2 + M2b + delta * delta * (n * nb / nn);
    n = nn;
}

// The Shared-Sample estimator (the Remark of Section 4, eq. mc16): every suffix sample i is
// scored under all 2^m prefixes, h_i = sum_m P(D_m) V(z_m, y_i). With
// V = beta_m max(sign (tau_m + f_i), 0) + C_m, the C part is the per-job constant
// s_pc = sum_m P(D_m) C_m and each (prefix, sample) pair costs a clamped add and a multiply-add.
// The block holds the job's table as (t_m, t_m, w_m, w_m) with t_m = sign tau_m 2^-k and
// w_m = P(D_m) beta_m 2^k, where 2^k >= 2 max_{m,i} sign (tau_m + f_i) (the largest sign tau_m
// plus a bound of sign f), k >= 0: then t_m + sign f_i 2^-k < 1 and the saturating add
// sat(t_m + sign f_i 2^-k) is max(sign (tau_m + f_i), 0) 2^-k exactly (the scale is a power of
// 2), so the clamp runs on the FMA pipe instead of the ALU pipe, and w_m sat(.) is the unscaled
// term, the same FP32 number as without the scale. (scale_k = -1: an unscaled table for bounds
// beyond 2^60, clamped with max(., 0).) Two samples share each
// paired multiply-add (__ffma2_rn). The sum over prefixes runs in blocks of 64 (two-level
// summation: FP32 error under 64 + 2^mb / 64 ulps). A work item is BT_MC_ITEM = 4 x BT_THREADS
// samples: four per thread, walked together. The item's (count, mean, M2) is combined over its
// warps in FP32 by warp 0 and stored in FP64.
template <int FIELD>
__device__ void mc_shared_item(const bt_mc_args &a, const bt_mc_job &J, int64_t item, const float4 *s_tab,
                               float s_pc, int scale_k, float3 *red) {
    static_assert(BT_MC_ITEM == 4 * BT_THREADS, "four samples per thread and item");
    const int64_t i0 = item * BT_MC_ITEM + threadIdx.x;
    unsigned idx[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) idx[w] = (unsigned)(i0 + (int64_t)w * BT_THREADS);
    float f[4];
    simulate_w<FIELD, 4>(J, idx, 0u, f, make_uint2(a.key_lo, a.key_hi));
    const float down = scale_k >= 0 ? scalbnf(1.0f, -scale_k) : 1.0f;
    const float sg = J.sign > 0 ? down : -down;   // sign 2^-k
    const float fa = sg * f[0], fb = sg * f[1], fc = sg * f[2], fd = sg * f[3];
    float2 v01 = make_float2(0.0f, 0.0f), v23 = make_float2(0.0f, 0.0f);
    const int M = 1 << J.mb;
    for (int m0 = 0; m0 < M; m0 += 64) {
        const int m1 = min(m0 + 64, M);
        float2 a01 = make_float2(0.0f, 0.0f), a23 = make_float2(0.0f, 0.0f);
        if (scale_k >= 0) {
#pragma unroll 8
            for (int m = m0; m < m1; ++m) {
                const float4 P = s_tab[m];
                const float2 WW = make_float2(P.z, P.w);
                a01 = __ffma2_rn(WW, make_float2(__saturatef(__fadd_rn(P.x, fa)), __saturatef(__fadd_rn(P.y, fb))),
                                 a01);
                a23 = __ffma2_rn(WW, make_float2(__saturatef(__fadd_rn(P.x, fc)), __saturatef(__fadd_rn(P.y, fd))),
                                 a23);
            }
        } else {   // unscaled table (suffix quantities beyond 2^60): the clamp as max(., 0)
#pragma unroll 8
            for (int m = m0; m < m1; ++m) {
                const float4 P = s_tab[m];
                const float2 WW = make_float2(P.z, P.w);
                a01 = __ffma2_rn(WW, make_float2(fmaxf(__fadd_rn(P.x, fa), 0.0f), fmaxf(__fadd_rn(P.y, fb), 0.0f)), a01);
                a23 = __ffma2_rn(WW, make_float2(fmaxf(__fadd_rn(P.x, fc), 0.0f), fmaxf(__fadd_rn(P.y, fd), 0.0f)), a23);
            }
        }
        v01 = __fadd2_rn(v01, a01);
        v23 = __fadd2_rn(v23, a23);
    }
    const float v[4] = {v01.x + s_pc, v01.y + s_pc, v23.x + s_pc, v23.y + s_pc};
    float n = 0.0f, mean = 0.0f, M2 = 0.0f;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        if (i0 + (int64_t)w * BT_THREADS >= J.R) break;
        n += 1.0f;  // Welford update
        const float delta = v[w] - mean;
        mean += delta / n;
        M2 += delta * (v[w] - mean);
    }
    // warp, then block combination (fixed shape)
    for (int o = 16; o > 0; o >>= 1) {
        const float nb = __shfl_down_sync(0xffffffffu, n, o);
        const float mb_ = __shfl_down_sync(0xffffffffu, mean, o);
        const float M2b = __shfl_down_sync(0xffffffffu, M2, o);
        chan(n, mean, M2, nb, mb_, M2b);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_float3(n, mean, M2);
    __syncthreads();
    if (threadIdx.x < 32) {
        static_assert(BT_THREADS / 32 <= 32, "one warp combines the block's warps");
        const float3 r = threadIdx.x < BT_THREADS / 32 ? red[threadIdx.x] : make_float3(0.0f, 0.0f, 0.0f);
        n = r.x, mean = r.y, M2 = r.z;
        for (int o = BT_THREADS / 64; o > 0; o >>= 1) {
            const float nb = __shfl_down_sync(0xffffffffu, n, o);
            const float mb_ = __shfl_down_sync(0xffffffffu, mean, o);
            const float M2b = __shfl_down_sync(0xffffffffu, M2, o);
            chan(n, mean, M2, nb, mb_, M2b);
        }
        if (threadIdx.x == 0) a.item_stats[J.item_begin + item] = make_double4(n, mean, M2, 0.0);
    }
}

// Shared-Sample strata table of every job (one thread per stratum, BT_MC_TAB_BLOCKS blocks per
// job): entry m = (sign tau_m, sign tau_m, P(D_m) beta_m, P(D_m) beta_m) in FP32, and each
// block's FP64 partial sum of P(D_m) C_m. The FP64 strata states are computed once per job here,
// not once per block of the sampling kernel.
__global__ void __launch_bounds__(BT_MC_TAB_THREADS) k_mc_shared_tab(bt_mc_args a) {
    __shared__ double s_w[BT_MC_TAB_THREADS / 32];
    const int job = blockIdx.x / BT_MC_TAB_BLOCKS, blk = blockIdx.x % BT_MC_TAB_BLOCKS;
    const bt_mc_job &J = a.jobs[job];
    const int m = blk * BT_MC_TAB_THREADS + threadIdx.x;
    double pc = 0.0;
    if (m < (1 << J.mb)) {
        const mc_pref P = stratum_state(J, (uint64_t)m);
        const float t = (float)(J.sign > 0 ? P.tau : -P.tau), w = (float)(P.prob * P.beta);
        a.shared_tab[(size_t)job * BT_MC_TAB_ENTRIES + m] = make_float4(t, t, w, w);
        pc = P.prob * P.C;
    }
    for (int o = 16; o > 0; o >>= 1) pc += __shfl_down_sync(0xffffffffu, pc, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = pc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < BT_MC_TAB_THREADS / 32; ++w) t += s_w[w];
        a.shared_pc[(size_t)job * BT_MC_TAB_BLOCKS + blk] = t;
    }
}

// Claims the next work item for the block: (item, job), item -1 once all are taken.
__device__ __forceinline__ void mc_claim(const bt_mc_args &a, int64_t *item, int *job) {
    const unsigned long long i = atomicAdd(a.counter, 1ull);
    if (i >= (unsigned long long)a.n_items) {
        *item = -1;
        return;
    }
    int lo = 0, hi = a.n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.jobs[mid].item_begin <= (int64_t)i) lo = mid;
        else hi = mid - 1;
    }
    *item = (int64_t)i;
    *job = lo;
}

// Shared-Sample sampling kernel: blocks take work items (BT_MC_ITEM samples of one job) from a
// global counter; a block loads a job's strata table into shared memory when it moves to that job.
// Thread 0 claims item k + 1 while the block runs item k; the claim and the warp statistics are
// double-buffered by the parity of k, so an item costs one block barrier (inside the item):
// slot k & 1 is read before that barrier of item k and written again only after it, in item k + 1.
__global__ void __launch_bounds__(BT_THREADS, 2) k_mc_shared(bt_mc_args a) {
    __shared__ float4 s_tab[BT_MC_TAB_ENTRIES];
    __shared__ float s_pc;
    __shared__ float s_max[BT_THREADS / 32];
    __shared__ int s_k;
    __shared__ float3 red[2][BT_THREADS / 32];
    __shared__ int64_t s_item[2];
    __shared__ int s_job[2];
    __shared__ bt_mc_job sJ;
    if (threadIdx.x == 0) mc_claim(a, &s_item[0], &s_job[0]);
    __syncthreads();
    int cur_job = -1;
    for (int k = 0;; ++k) {
        const int64_t it = s_item[k & 1];
        const int jb = s_job[k & 1];
        if (it < 0) break;
        if (threadIdx.x == 0) mc_claim(a, &s_item[(k + 1) & 1], &s_job[(k + 1) & 1]);
        if (jb != cur_job) {
            // every thread is past the barrier of item k - 1: the old table is no longer read
            if (threadIdx.x == 0) {
                sJ = a.jobs[jb];
                double t = 0.0;
                for (int b = 0; b < BT_MC_TAB_BLOCKS; ++b) t += a.shared_pc[(size_t)jb * BT_MC_TAB_BLOCKS + b];
                s_pc = (float)t;
            }
            const int M = 1 << a.jobs[jb].mb;
            const float4 *tab = a.shared_tab + (size_t)jb * BT_MC_TAB_ENTRIES;
            float tmax = -3.0e38f;
            for (int m = threadIdx.x; m < M; m += BT_THREADS) {
                s_tab[m] = tab[m];
                tmax = fmaxf(tmax, tab[m].x);
            }
            // the pair loop's scale: 2^k >= 2 (max_m t_m + bound of sign f), k >= 0; beyond 2^60
            // (k = -1) the table stays unscaled and the loop clamps with max(., 0)
            for (int o = 16; o > 0; o >>= 1) tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
            if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = tmax;
            __syncthreads();
            if (threadIdx.x == 0) {
                float t = s_max[0];
                for (int w = 1; w < BT_THREADS / 32; ++w) t = fmaxf(t, s_max[w]);
                const double B = (double)t + a.jobs[jb].fbound;
                s_k = B < 0.5 ? 0 : B < 0x1p60 ? ilogb(B) + 2 : -1;
            }
            __syncthreads();
            if (s_k > 0) {
                const float down = scalbnf(1.0f, -s_k), up = scalbnf(1.0f, s_k);
                for (int m = threadIdx.x; m < M; m += BT_THREADS) {
                    const float4 e = s_tab[m];
                    s_tab[m] = make_float4(e.x * down, e.y * down, e.z * up, e.w * up);
                }
            }
            __syncthreads();
            cur_job = jb;
        }
        const bt_mc_job &J = sJ;
        const int64_t item = it - J.item_begin;
        float3 *rk = red[k & 1];
        const int sk = s_k;
        switch (J.field) {
        case BT_F_ARITH: mc_shared_item<BT_F_ARITH>(a, J, item, s_tab, s_pc, sk, rk); break;
        case BT_F_GEO: mc_shared_item<BT_F_GEO>(a, J, item, s_tab, s_pc, sk, rk); break;
        case BT_F_EURO: mc_shared_item<BT_F_EURO>(a, J, item, s_tab, s_pc, sk, rk); break;
        case BT_F_LOOKMAX: mc_shared_item<BT_F_LOOKMAX>(a, J, item, s_tab, s_pc, sk, rk); break;
        default: mc_shared_item<BT_F_LOOKMIN>(a, J, item, s_tab, s_pc, sk, rk); break;
        }
    }
}

// The Partitioned estimator, one work item per warp: a warp takes items from
// the shared counter and runs them to the end on its own -- 32 lanes x 32
// samples of one stratum, a shuffle-tree Welford combination, one FP64
// record per item -- so no block-wide barrier ever holds the other warps.
// Same draws, same item records and the same per-stratum combination
// (k_mc_strata) as the block kernel.
template <int FIELD>
__device__ __forceinline__ void mc_warp_item(const bt_mc_args &a, const bt_mc_job &J, int64_t item_local,
                                             float tau, float beta, float C, int64_t m) {
    const int lane = threadIdx.x & 31;
    const int64_t chunks = (J.R + BT_MC_ITEM - 1) / BT_MC_ITEM;
    const int64_t i0 = (item_local % chunks) * BT_MC_ITEM;
    float n = 0.0f, mean = 0.0f, M2 = 0.0f;
    constexpr int W = BT_MC_WALKERS;
    static_assert((BT_MC_ITEM / 32) % W == 0, "walkers must divide a lane's samples per item");
#pragma unroll 1
    for (int k = 0; k < BT_MC_ITEM / 32; k += W) {
        const int64_t ia = i0 + lane + (int64_t)k * 32;
        if (ia >= J.R) break;
        unsigned idx[W];
#pragma unroll
        for (int w = 0; w < W; ++w) idx[w] = (unsigned)(ia + 32 * w);
        float fw[W];
        simulate_w<FIELD, W>(J, idx, (unsigned)m, fw, make_uint2(a.key_lo, a.key_hi));
#pragma unroll
        for (int h = 0; h < W; ++h) {
            if (h > 0 && ia + 32 * h >= J.R) break;
            const float v = payoff_of(J, tau, beta, C, fw[h]);
            n += 1.0f;
            const float delta = v - mean;
            mean += delta / n;
            M2 += delta * (v - mean);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float nb = __shfl_down_sync(0xffffffffu, n, o);
        const float mb_ = __shfl_down_sync(0xffffffffu, mean, o);
        const float M2b = __shfl_down_sync(0xffffffffu, M2, o);
        chan(n, mean, M2, nb, mb_, M2b);
    }
    if (lane == 0) a.item_stats[J.item_begin + item_local] = make_double4(n, mean, M2, (double)m);
}

__global__ void __launch_bounds__(BT_MC_WARP_THREADS, BT_MC_MIN_BLOCKS) k_mc_warp(bt_mc_args a) {
    const int lane = threadIdx.x & 31;
    int cur_job = -1;
    int64_t cur_stratum = -1;
    float tau = 0.0f, beta = 0.0f, C = 0.0f;
    for (;;) {
        unsigned long long i = 0;
        int j = 0;
        if (lane == 0) {
            i = atomicAdd(a.counter, 1ull);
            if (i < (unsigned long long)a.n_items) {
                int lo = 0, hi = a.n_jobs - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (a.jobs[mid].item_begin <= (int64_t)i) lo = mid;
                    else hi = mid - 1;
                }
                j = lo;
            }
        }
        i = __shfl_sync(0xffffffffu, i, 0);
        j = __shfl_sync(0xffffffffu, j, 0);
        if (i >= (unsigned long long)a.n_items) break;
        const bt_mc_job J = a.jobs[j];
        const int64_t item_local = (int64_t)i - J.item_begin;
        const int64_t chunks = (J.R + BT_MC_ITEM - 1) / BT_MC_ITEM;
        const int64_t m = J.shard + (item_local / chunks) * J.n_shards;  // global stratum index
        if (j != cur_job || m != cur_stratum) {
            if (lane == 0) {
                const mc_pref st = stratum_state(J, (uint64_t)m);
                tau = (float)st.tau;
                beta = (float)st.beta;
                C = (float)st.C;
            }
            tau = __shfl_sync(0xffffffffu, tau, 0);
            beta = __shfl_sync(0xffffffffu, beta, 0);
            C = __shfl_sync(0xffffffffu, C, 0);
            cur_job = j;
            cur_stratum = m;
        }
        switch (J.field) {
        case BT_F_ARITH: mc_warp_item<BT_F_ARITH>(a, J, item_local, tau, beta, C, m); break;
        case BT_F_GEO: mc_warp_item<BT_F_GEO>(a, J, item_local, tau, beta, C, m); break;
        case BT_F_EURO: mc_warp_item<BT_F_EURO>(a, J, item_local, tau, beta, C, m); break;
        case BT_F_LOOKMAX: mc_warp_item<BT_F_LOOKMAX>(a, J, item_local, tau, beta, C, m); break;
        default: mc_warp_item<BT_F_LOOKMIN>(a, J, item_local, tau, beta, C, m); break;
        }
    }
}

// Combination, first half: per stratum, its work items in two passes without a division per item
// (FP64 division is slow on this part): N = sum n_i and S = sum n_i mean_i give mean = S / N, then
// M2 = sum M2_i + n_i (mean_i - mean)^2, the exact decomposition of the sum of squares about the
// stratum mean. One thread per stratum for up to 32 work items, one warp for up to
// BT_MC_STRATA_BLOCK, one block above (the choice depends only on R, so a stratum's result does not
// depend on the other strata of the call). Fixed lane order, fixed reduction trees. Writes per stratum
// (mean, P(D_m), P(D_m)^2 s_m^2 / n_m, P(D_m) M2_m / n_m) with s_m^2 = M2_m / (n_m - 1), the
// terms of eq. mc12, its variance and eq. mc14, and the per-stratum statistics when asked.
__device__ __forceinline__ double warp_sum64(double x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
enum { MC_BY_THREAD, MC_BY_WARP, MC_BY_BLOCK };
template <int BY>
__device__ __forceinline__ double group_sum64(double x, double *sh) {
    if (BY == MC_BY_THREAD) return x;
    x = warp_sum64(x);
    if (BY == MC_BY_WARP) return x;
    __syncthreads();  // sh is free (its last readers are past this barrier)
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < BT_THREADS / 32; ++w) t += sh[w];
    return t;
}
template <int BY>
__global__ void k_mc_strata(const bt_mc_job *jobs, int n_jobs, const double4 *item_stats, int64_t n_strata,
                            double4 *strata_nmq, double *strata /* [n_strata][3] or null */) {
    __shared__ double sh[BT_THREADS / 32];
    const int64_t g = BY == MC_BY_BLOCK  ? (int64_t)blockIdx.x
                      : BY == MC_BY_WARP ? (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)
                                         : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = BY == MC_BY_BLOCK ? threadIdx.x : BY == MC_BY_WARP ? (threadIdx.x & 31) : 0;
    const int width = BY == MC_BY_BLOCK ? BT_THREADS : BY == MC_BY_WARP ? 32 : 1;
    if (g >= n_strata) return;  // uniform over the group that combines one stratum
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].strata_off <= g) lo = mid;
        else hi = mid - 1;
    }
    const bt_mc_job &J = jobs[lo];
    const int64_t m = g - J.strata_off;                // stratum of this run
    const int64_t mg = J.shard + m * J.n_shards;       // its global index
    const int64_t chunks = (J.R + BT_MC_ITEM - 1) / BT_MC_ITEM;
    const double4 *it = item_stats + J.item_begin + m * chunks;
    double n = 0.0, S = 0.0;
#pragma unroll 4
    for (int64_t c = lane; c < chunks; c += width) {
        const double4 s = it[c];
        n += s.x;
        S = fma(s.x, s.y, S);
    }
    n = group_sum64<BY>(n, sh);
    S = group_sum64<BY>(S, sh);
    const double mu = n > 0.0 ? S / n : 0.0;
    double Q = 0.0;
#pragma unroll 4
    for (int64_t c = lane; c < chunks; c += width) {
        const double4 s = it[c];
        const double d = s.y - mu;
        Q += s.z;
        Q = fma(s.x * d, d, Q);
    }
    Q = group_sum64<BY>(Q, sh);
    if (lane == 0) {
        const double prob = J.shared ? 1.0 : J.prob_k[__popcll((unsigned long long)mg)];
        const double s2 = n > 1.0 ? Q / (n - 1.0) : 0.0;
        strata_nmq[g] = make_double4(mu, prob, n > 0.0 ? prob * prob * s2 / n : 0.0, n > 0.0 ? prob * Q / n : 0.0);
        if (strata) {
            strata[3 * g] = mu;
            strata[3 * g + 1] = s2;
            strata[3 * g + 2] = prob;
        }
    }
}

// Combination, second half: across strata, eq. mc12 (theta = sum_m P(D_m) mean_m, Neumaier-
// compensated), Var = sum_m P(D_m)^2 s_m^2 / n_m, and the variance of one plain draw by the law
// of total variance (eq. mc14): sum_m P(D_m) M2_m / n_m + sum_m P(D_m) (mean_m - theta)^2. The
// last sum is taken about c = mean_0 in one pass, from A = sum P (mean - c)^2, B = sum P (mean - c)
// and P = sum P(D_m): sum P (mean - theta)^2 = A - 2 (theta - c) B + (theta - c)^2 P.
// BT_MC_FIN_BLOCKS blocks per job each take a fixed contiguous range of its strata; one warp per
// job then adds the blocks' partial sums in block order.
__global__ void k_mc_fin_part(const bt_mc_job *jobs, int n_jobs, const double4 *strata_nmq, double *partials) {
    const int j = blockIdx.x / BT_MC_FIN_BLOCKS, b = blockIdx.x % BT_MC_FIN_BLOCKS;
    if (j >= n_jobs) return;
    const bt_mc_job &J = jobs[j];
    const int64_t M = J.M, m0 = M * b / BT_MC_FIN_BLOCKS, m1 = M * (b + 1) / BT_MC_FIN_BLOCKS;
    const double c = strata_nmq[J.strata_off].x;
    double th = 0.0, thc = 0.0, var = 0.0, ew = 0.0, A = 0.0, B = 0.0, P = 0.0;
    for (int64_t m = m0 + threadIdx.x; m < m1; m += BT_THREADS) {
        const double4 s = strata_nmq[J.strata_off + m];
        const double mu = s.x, prob = s.y;
        const double x = prob * mu;
        const double t = th + x;
        thc += fabs(th) >= fabs(x) ? (th - t) + x : (x - t) + th;
        th = t;
        var += s.z;
        ew += s.w;
        const double d = mu - c;
        A = fma(prob * d, d, A);
        B = fma(prob, d, B);
        P += prob;
    }
    __shared__ double sh[6][BT_THREADS];
    const double v[6] = {th + thc, var, ew, A, B, P};
    for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int w = BT_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 6) partials[((size_t)j * BT_MC_FIN_BLOCKS + b) * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_mc_finalize(const bt_mc_job *jobs, int n_jobs, const double4 *strata_nmq, const double *partials,
                              bt_result *out) {
    static_assert(BT_MC_FIN_BLOCKS <= 32, "one lane per partial");
    const int j = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= n_jobs) return;
    const bt_mc_job &J = jobs[j];
    double v[6];
    for (int q = 0; q < 6; ++q) {
        const double x = lane < BT_MC_FIN_BLOCKS ? partials[((size_t)j * BT_MC_FIN_BLOCKS + lane) * 8 + q] : 0.0;
        v[q] = warp_sum64(x);
    }
    if (lane == 0) {
        const double theta = v[0], c = strata_nmq[J.strata_off].x, e = theta - c;
        const double vb = v[3] - 2.0 * e * v[4] + e * e * v[5];
        bt_result r;
        r.value = J.disc * theta;
        r.stderr_mc = J.disc * sqrt(v[1]);
        // eq. mc14 needs the mean over all strata: only a run over all of them has it
        r.var_plain = J.shared || J.n_shards > 1 ? 0.0 : v[2] + fmax(vb, 0.0);
        r.err_est = 0.0;
        r.paths = (int64_t)J.M * J.R;
        out[J.out] = r;
    }
}

extern "C" int bt_launch_mc(const bt_mc_args *a, int shared, int grid, void *stream) {
    if (a->n_items <= 0) return 0;
    if (shared) {
        k_mc_shared_tab<<<(unsigned)a->n_jobs * BT_MC_TAB_BLOCKS, BT_MC_TAB_THREADS, 0, (cudaStream_t)stream>>>(*a);
        if ((int64_t)grid > a->n_items) grid = (int)a->n_items;
        k_mc_shared<<<grid, BT_THREADS, 0, (cudaStream_t)stream>>>(*a);
    } else {
        const int64_t warps = (int64_t)grid * (BT_MC_WARP_THREADS / 32);
        if (warps > a->n_items)
            grid = (int)((a->n_items + BT_MC_WARP_THREADS / 32 - 1) / (BT_MC_WARP_THREADS / 32));
        k_mc_warp<<<grid, BT_MC_WARP_THREADS, 0, (cudaStream_t)stream>>>(*a);
    }
    return (int)cudaGetLastError();
}

extern "C" int bt_launch_mc_finalize(const bt_mc_job *jobs, int n_jobs, int64_t chunks, const double4 *item_stats,
                                     int64_t n_strata, double4 *strata_nmq, double *partials, bt_result *out,
                                     double *strata, void *stream) {
    if (n_jobs <= 0) return 0;
    cudaStream_t st = (cudaStream_t)stream;
    const int wpb = BT_THREADS / 32;
    if (chunks > BT_MC_STRATA_BLOCK)
        k_mc_strata<MC_BY_BLOCK><<<(unsigned)n_strata, BT_THREADS, 0, st>>>(jobs, n_jobs, item_stats, n_strata,
                                                                          strata_nmq, strata);
    else if (chunks > 32)
        k_mc_strata<MC_BY_WARP><<<(unsigned)((n_strata + wpb - 1) / wpb), BT_THREADS, 0, st>>>(
            jobs, n_jobs, item_stats, n_strata, strata_nmq, strata);
    else
        k_mc_strata<MC_BY_THREAD><<<(unsigned)((n_strata + BT_THREADS - 1) / BT_THREADS), BT_THREADS, 0, st>>>(
            jobs, n_jobs, item_stats, n_strata, strata_nmq, strata);
    k_mc_fin_part<<<(unsigned)n_jobs * BT_MC_FIN_BLOCKS, BT_THREADS, 0, st>>>(jobs, n_jobs, strata_nmq, partials);
    k_mc_finalize<<<(unsigned)((n_jobs + wpb - 1) / wpb), BT_THREADS, 0, st>>>(jobs, n_jobs, strata_nmq, partials, out);
    return (int)cudaGetLastError();
}

extern "C" int bt_launch_philox_selftest(const uint4 *ctr, const uint2 *key, uint4 *out, int n, void *stream) {
    k_philox_selftest<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(ctr, key, out, n);
    return (int)cudaGetLastError();
}

extern "C" int bt_mc_grid_size(int device, int shared) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (shared) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mc_shared, BT_THREADS, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mc_warp, BT_MC_WARP_THREADS, 0);
    if (per < 1) per = 1;
    return sms * per;
}
