// Internal layout of the Monte Carlo kernels (mc.cu) and their host runtime.
#pragma once
#include <stdint.h>

#include "bt_internal.h"

#define BT_MC_ITEM 1024            // samples per work item (256 threads x 4)
#define BT_MC_SHARED_MAX_BITS 10   // Shared-Sample strata live in shared memory
#define BT_MC_TAB_ENTRIES (1 << BT_MC_SHARED_MAX_BITS)         // one table entry per stratum
#define BT_MC_TAB_THREADS 64                                    // threads per block of the table kernel
#define BT_MC_TAB_BLOCKS (BT_MC_TAB_ENTRIES / BT_MC_TAB_THREADS)
#define BT_MC_MAX_N 4096
#define BT_MC_MAX_BITS 24
#define BT_MC_FIN_BLOCKS 32        // blocks per job of the across-strata combination
#define BT_MC_STRATA_BLOCK 256     // work items per stratum above which a block (not a warp) combines them

struct bt_mc_job {
    int32_t N, mb;                 // tree depth, strata bits (prefix length)
    int64_t R;                     // samples per stratum (Shared-Sample: per prefix set)
    int32_t field, sign;           // suffix quantity (bt_field) and +1 call / -1 put
    int32_t shared;                // 1: Shared-Sample estimator
    uint32_t stream;               // Philox counter word 3 (the option's index in the call)
    uint32_t key_lo, key_hi;       // Philox key (the seed)
    uint32_t thr;                  // up iff the 32-bit word < thr = round(p 2^32)
    int32_t out;                   // result slot
    double u, d, p, S0, K, disc;
    double fbound;                 // Shared-Sample: an upper bound of the suffix quantity f of a call
                                   // (sign +1; 0 for a put), sizing the pair loop's power-of-2 scale
    float uf, df, lnu_f;
    int32_t pad;
    int32_t shard, n_shards;       // this run covers strata m = shard + j * n_shards
    int64_t M;                     // strata in this run (1 for Shared-Sample)
    int64_t item_begin, n_items, strata_off;
    double prob_k[BT_MC_MAX_BITS + 1];  // P(D_m) of a stratum with k up moves: p^k (1 - p)^(mb - k)
};

struct bt_mc_args {
    const bt_mc_job *jobs;
    int32_t n_jobs;
    int32_t pad;
    uint32_t key_lo, key_hi;       // the Philox key (the seed), the same for every job of a launch: as a
                                   // kernel argument it is warp-uniform, and so are its round keys
    int64_t n_items;
    double4 *item_stats;           // per item: (count, mean, M2, stratum)
    unsigned long long *counter;
    // Shared-Sample only: per job, the strata table the payoff loop reads (per stratum m,
    // (sign tau_m, sign tau_m, P(D_m) beta_m, P(D_m) beta_m)) and BT_MC_TAB_BLOCKS partial sums
    // of P(D_m) C_m in FP64
    float4 *shared_tab;            // [n_jobs][BT_MC_TAB_ENTRIES]
    double *shared_pc;             // [n_jobs][BT_MC_TAB_BLOCKS]
};

#ifdef __cplusplus
extern "C" {
#endif
int bt_launch_mc(const bt_mc_args *a, int shared, int grid, void *stream);
int bt_launch_mc_finalize(const bt_mc_job *jobs, int n_jobs, int64_t chunks, const double4 *item_stats,
                          int64_t n_strata, double4 *strata_nmq, double *partials, bt_result *out, double *strata,
                          void *stream);
int bt_launch_philox_selftest(const uint4 *ctr, const uint2 *key, uint4 *out, int n, void *stream);
int bt_mc_grid_size(int device, int shared);
#ifdef __cplusplus
}
#endif
