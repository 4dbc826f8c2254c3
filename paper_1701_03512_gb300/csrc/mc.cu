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
// Shared-Sample kernel (k_mc, whose strata states sit in shared memory).
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
    const double u = J.u, d = J.d, lnu = log(u), p = J.p;
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
    s.prob = pow(p, (double)k) * pow(1.0 - p, (double)(mb - k));
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
            lvl += up ? 1 : -1;
            if (FIELD == BT_F_GEO) D += lvl;
            if (FIELD == BT_F_LOOKMAX) ext = lvl > ext ? lvl : ext;
            if (FIELD == BT_F_LOOKMIN) ext = lvl < ext ? lvl : ext;
        }
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
            A[w].step(r[w].x < J.thr, J.uf, J.df);
            A[w].step(r[w].y < J.thr, J.uf, J.df);
            A[w].step(r[w].z < J.thr, J.uf, J.df);
            A[w].step(r[w].w < J.thr, J.uf, J.df);
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
__device__ __forceinline__ void chan64(double &n, double &mean, double &M2, double nb, double meanb, double M2b) {
    const double nn = n + nb;
    if (nn == 0.0) return;
    const double delta = meanb - mean;
    mean = mean + delta * (nb / nn);
    M2 = M2 + M2b + delta * delta * (n * nb / nn);
    n = nn;
}

template <int FIELD, bool SHARED>
__device__ void mc_item(const bt_mc_args &a, const bt_mc_job &J, int64_t item_local, const mc_pref *s_str,
                        float3 *red) {
    // item -> (stratum, first sample); shared mode has one "stratum" index 0
    const int64_t chunks = (J.R + BT_MC_ITEM - 1) / BT_MC_ITEM;
    const int64_t m = J.shard + (item_local / chunks) * J.n_shards;  // global stratum index
    const int64_t i0 = (item_local % chunks) * BT_MC_ITEM;
    float n = 0.0f, mean = 0.0f, M2 = 0.0f;
    float tau = 0.0f, beta = 0.0f, C = 0.0f;
    if (!SHARED) {
        tau = (float)s_str[0].tau;
        beta = (float)s_str[0].beta;
        C = (float)s_str[0].C;
    }
#pragma unroll 1
    for (int k = 0; k < BT_MC_ITEM / BT_THREADS; k += 2) {
        const int64_t ia = i0 + threadIdx.x + (int64_t)k * BT_THREADS;
        const int64_t ib = ia + BT_THREADS;
        if (ia >= J.R) break;
        const unsigned idx[2] = {(unsigned)ia, (unsigned)ib};
        float f2[2];
        simulate_w<FIELD, 2>(J, idx, SHARED ? 0u : (unsigned)m, f2, make_uint2(a.key_lo, a.key_hi));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && ib >= J.R) break;
            float v;
            if (!SHARED) {
                v = payoff_of(J, tau, beta, C, f2[h]);
            } else {
                // h_i = sum_m P(D_m) V(z_m, y_i): the same suffix under every prefix (eq. mc16)
                float acc = 0.0f, accc = 0.0f;
                for (int s = 0; s < (1 << J.mb); ++s) {
                    const mc_pref P = s_str[s];
                    const float term = (float)P.prob * payoff_of(J, (float)P.tau, (float)P.beta, (float)P.C, f2[h]);
                    const float t = acc + term;  // Kahan-compensated sum over strata
                    accc += (acc - t) + term;
                    acc = t;
                }
                v = acc + accc;
            }
            // Welford update
            n += 1.0f;
            const float delta = v - mean;
            mean += delta / n;
            M2 += delta * (v - mean);
        }
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
    if (threadIdx.x == 0) {
        double N_ = 0.0, MU = 0.0, Q = 0.0;
        for (int w = 0; w < BT_THREADS / 32; ++w) chan64(N_, MU, Q, red[w].x, red[w].y, red[w].z);
        a.item_stats[J.item_begin + item_local] = make_double4(N_, MU, Q, (double)m);
    }
}

__global__ void __launch_bounds__(BT_THREADS, 2) k_mc(bt_mc_args a) {
    __shared__ mc_pref s_str[1 << BT_MC_SHARED_MAX_BITS];
    __shared__ float3 red[BT_THREADS / 32];
    __shared__ int s_job;
    __shared__ int64_t s_item;
    __shared__ bt_mc_job sJ;
    int cur_job = -1;
    int64_t cur_stratum = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned long long i = atomicAdd(a.counter, 1ull);
            s_item = i < (unsigned long long)a.n_items ? (int64_t)i : -1;
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
        if (s_item < 0) break;
        if (s_job != cur_job) {
            if (threadIdx.x == 0) sJ = a.jobs[s_job];
            __syncthreads();
        }
        const bt_mc_job &J = sJ;
        const int64_t item_local = s_item - J.item_begin;
        if (J.shared) {
            if (s_job != cur_job) {
                for (int s = threadIdx.x; s < (1 << J.mb); s += BT_THREADS) s_str[s] = stratum_state(J, (uint64_t)s);
                __syncthreads();
            }
        } else {
            const int64_t chunks = (J.R + BT_MC_ITEM - 1) / BT_MC_ITEM;
            const int64_t m = J.shard + (item_local / chunks) * J.n_shards;
            if (s_job != cur_job || m != cur_stratum) {
                __syncthreads();
                if (threadIdx.x == 0) s_str[0] = stratum_state(J, (uint64_t)m);
                __syncthreads();
                cur_stratum = m;
            }
        }
        cur_job = s_job;
        switch (J.field * 2 + (J.shared ? 1 : 0)) {
        case BT_F_ARITH * 2: mc_item<BT_F_ARITH, false>(a, J, item_local, s_str, red); break;
        case BT_F_ARITH * 2 + 1: mc_item<BT_F_ARITH, true>(a, J, item_local, s_str, red); break;
        case BT_F_GEO * 2: mc_item<BT_F_GEO, false>(a, J, item_local, s_str, red); break;
        case BT_F_GEO * 2 + 1: mc_item<BT_F_GEO, true>(a, J, item_local, s_str, red); break;
        case BT_F_EURO * 2: mc_item<BT_F_EURO, false>(a, J, item_local, s_str, red); break;
        case BT_F_EURO * 2 + 1: mc_item<BT_F_EURO, true>(a, J, item_local, s_str, red); break;
        case BT_F_LOOKMAX * 2: mc_item<BT_F_LOOKMAX, false>(a, J, item_local, s_str, red); break;
        case BT_F_LOOKMAX * 2 + 1: mc_item<BT_F_LOOKMAX, true>(a, J, item_local, s_str, red); break;
        case BT_F_LOOKMIN * 2: mc_item<BT_F_LOOKMIN, false>(a, J, item_local, s_str, red); break;
        default: mc_item<BT_F_LOOKMIN, true>(a, J, item_local, s_str, red); break;
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

// Combination, first half: one warp per stratum combines the stratum's work items
// (Chan et al.'s update, fixed lane order and a fixed shuffle tree).
__global__ void k_mc_strata(const bt_mc_job *jobs, int n_jobs, const double4 *item_stats, int64_t n_strata,
                            double4 *strata_nmq /* per stratum (n, mean, M2, prob) */) {
    const int64_t g = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= n_strata) return;
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
    double n = 0.0, mu = 0.0, Q = 0.0;
    for (int64_t c = lane; c < chunks; c += 32) {
        const double4 s = item_stats[J.item_begin + m * chunks + c];
        chan64(n, mu, Q, s.x, s.y, s.z);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double nb = __shfl_down_sync(0xffffffffu, n, o);
        const double mb_ = __shfl_down_sync(0xffffffffu, mu, o);
        const double Qb = __shfl_down_sync(0xffffffffu, Q, o);
        chan64(n, mu, Q, nb, mb_, Qb);
    }
    if (lane == 0) strata_nmq[g] = make_double4(n, mu, Q, J.shared ? 1.0 : stratum_state(J, (uint64_t)mg).prob);
}

// Combination, second half: across strata, eq. mc12 and Var = sum_m P(D_m)^2 s_m^2 / R_m
// (unbiased s_m^2); also the variance of one draw by the law of total variance
// (eq. mc14), for plain-MC comparisons. One block per option.
__global__ void k_mc_finalize(const bt_mc_job *jobs, int n_jobs, const double4 *strata_nmq, bt_result *out,
                              double *strata /* [sum over jobs of 2^mb][3] or null */) {
    const int j = blockIdx.x;
    if (j >= n_jobs) return;
    const bt_mc_job J = jobs[j];
    __shared__ double sh[3][BT_THREADS];
    const int64_t M = J.M;
    double th = 0.0, thc = 0.0, var = 0.0, ew = 0.0;
    for (int64_t m = threadIdx.x; m < M; m += BT_THREADS) {
        const double4 s = strata_nmq[J.strata_off + m];
        const double n = s.x, mu = s.y, Q = s.z, prob = s.w;
        const double s2 = n > 1.0 ? Q / (n - 1.0) : 0.0;
        const double x = prob * mu;
        const double t = th + x;
        thc += fabs(th) >= fabs(x) ? (th - t) + x : (x - t) + th;
        th = t;
        var += prob * prob * s2 / n;
        ew += prob * (n > 0.0 ? Q / n : 0.0);  // sum_m P_m Var[V|D_m] (population form)
        if (strata) {
            double *o = strata + 3 * (J.strata_off + m);
            o[0] = mu;
            o[1] = s2;
            o[2] = prob;
        }
    }
    sh[0][threadIdx.x] = th + thc;
    sh[1][threadIdx.x] = var;
    sh[2][threadIdx.x] = ew;
    __syncthreads();
    for (int w = BT_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    const double theta = sh[0][0], var_tot = sh[1][0], ew_tot = sh[2][0];
    __syncthreads();
    // Var_D E[V|D] = sum_m P_m (mu_m - theta)^2
    double vb = 0.0;
    for (int64_t m = threadIdx.x; m < M; m += BT_THREADS) {
        const double4 s = strata_nmq[J.strata_off + m];
        vb += s.w * (s.y - theta) * (s.y - theta);
    }
    sh[0][threadIdx.x] = vb;
    __syncthreads();
    for (int w = BT_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bt_result r;
        r.value = J.disc * theta;
        r.stderr_mc = J.disc * sqrt(var_tot);
        // eq. mc14 needs the mean over all strata: only a run over all of them has it
        r.var_plain = J.shared || J.n_shards > 1 ? 0.0 : ew_tot + sh[0][0];
        r.err_est = 0.0;
        r.paths = (int64_t)M * J.R;
        out[J.out] = r;
    }
}

extern "C" int bt_launch_mc(const bt_mc_args *a, int shared, int grid, void *stream) {
    if (a->n_items <= 0) return 0;
    if (shared) {
        if ((int64_t)grid > a->n_items) grid = (int)a->n_items;
        k_mc<<<grid, BT_THREADS, 0, (cudaStream_t)stream>>>(*a);
    } else {
        const int64_t warps = (int64_t)grid * (BT_MC_WARP_THREADS / 32);
        if (warps > a->n_items)
            grid = (int)((a->n_items + BT_MC_WARP_THREADS / 32 - 1) / (BT_MC_WARP_THREADS / 32));
        k_mc_warp<<<grid, BT_MC_WARP_THREADS, 0, (cudaStream_t)stream>>>(*a);
    }
    return (int)cudaGetLastError();
}

extern "C" int bt_launch_mc_finalize(const bt_mc_job *jobs, int n_jobs, const double4 *item_stats,
                                     int64_t n_strata, double4 *strata_nmq, bt_result *out, double *strata,
                                     void *stream) {
    if (n_jobs <= 0) return 0;
    const int wpb = BT_THREADS / 32;
    k_mc_strata<<<(unsigned)((n_strata + wpb - 1) / wpb), BT_THREADS, 0, (cudaStream_t)stream>>>(
        jobs, n_jobs, item_stats, n_strata, strata_nmq);
    k_mc_finalize<<<n_jobs, BT_THREADS, 0, (cudaStream_t)stream>>>(jobs, n_jobs, strata_nmq, out, strata);
    return (int)cudaGetLastError();
}

extern "C" int bt_launch_philox_selftest(const uint4 *ctr, const uint2 *key, uint4 *out, int n, void *stream) {
    k_philox_selftest<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(ctr, key, out, n);
    return (int)cudaGetLastError();
}

extern "C" int bt_mc_grid_size(int device, int shared) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (shared) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mc, BT_THREADS, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mc_warp, BT_MC_WARP_THREADS, 0);
    if (per < 1) per = 1;
    return sms * per;
}
