// Internal layout shared by the host runtime and the CUDA kernels of libbtree.
// Not part of the public ABI (that is include/btree.h).
#pragma once
#include <stdint.h>

#include "../../include/btree.h"

#define BT_MAX_N_EXACT 40
#define BT_MAX_L 13            // suffix steps held in a shared-memory table (lattice passes)
#define BT_STEPS_MAX_L 12      // b^L <= 2^12 suffixes for trees given move by move, FP64 pass (16-byte entries)
#define BT_STEPS32_MAX_L 13    // b^L <= 2^13 for the FP32 pass (12 bytes a suffix: three float arrays)
#define BT_ARITH_CLS_MAX_N 27  // FP32 arithmetic-Asian jobs up to this depth sum each suffix as a class
// The FP32 passes that round every path once average those roundings over
// the tree's effective number of paths, n_eff = 1 / sum_x p(x)^2 (2^N for a
// balanced binomial tree, (p^2 + (1-p)^2)^-N for the lattice, prod_t 1 /
// sum_k q_tk^2 for a tree given move by move). They are used only where
// log2(n_eff) reaches this bound; other trees take a pass that rounds no
// single path (the pair-sum class pass of the lattice, or FP64 for trees
// given move by move).
#ifndef BT_PER_PATH_MIN_NEFF_LOG2
#define BT_PER_PATH_MIN_NEFF_LOG2 27.0
#endif
#define BT_ARITH_CLS_MAX_L 12  // ... with at most 2^12 classes of 16 bytes in shared memory
#define BT_LOW_BITS 10         // a work item covers 2^10 consecutive prefixes
#define BT_MIN_ITEM_BITS 5     // the split keeps >= 2^5 work items per option where it can
#ifndef BT_MIN_ITEM_BITS_FP64
#define BT_MIN_ITEM_BITS_FP64 7  // the FP64 pass keeps >= 2^7 (below N = 30: the FP64 pipe is slow, one
#endif                           // option should reach most SMs; measured best of 5, 7, 8, 9)
#define BT_THREADS 256         // threads per block of the path-sum kernels
#define BT_PT 4                // prefixes per thread (FP32 kernel): 256 * 4 = 2^10
#define BT_PT64 4              // prefixes per thread (FP64 kernel)
#define BT_UNROLL 8            // suffix groups are padded to a multiple of this
#define BT_SUF_MAX ((1 << BT_MAX_L) + (BT_MAX_L + 1) * (BT_UNROLL - 1))
#define BT_SUF_MAX_EVEN ((BT_SUF_MAX + 1) & ~1)   // float2 count keeping what follows 16-byte aligned
#define BT_LVL_NONE 30000      // sentinel level: "no price in this block"
#ifndef BT_CLS_UNROLL
#define BT_CLS_UNROLL 2        // class groups are padded to a multiple of this (measured: 2 beats 1 and 4)
#endif
#define BT_KEY_SPAN (BT_MAX_L * (BT_MAX_L + 1) / 2)   // |class key| <= this (level sum of the suffix)

// What the suffix table of a job holds (one field per job).
enum bt_field {
    BT_F_ARITH = 0,   // f_s = sum_{j=1}^{L} u^{l'_j}         (relative partial sum)
    BT_F_GEO = 1,     // f_s = u^{D_s/N}, D_s = sum_j l'_j    (relative geometric factor)
    BT_F_EURO = 2,    // f_s = u^{l'_L}                       (relative end price)
    BT_F_LOOKMAX = 3, // f_s = u^{max_j l'_j}                 (relative running max)
    BT_F_LOOKMIN = 4  // f_s = u^{min_j l'_j}                 (relative running min)
};
enum bt_mode { BT_MODE_CALL = 1, BT_MODE_PUT = 2, BT_MODE_BOTH = 3 };

// One pass over the 2^N paths of one option (possibly two payoffs).
struct bt_job {
    int32_t opt;              // option index (numeric inputs)
    int32_t out_call, out_put;// result slots of the call / put payoff, -1 if none
    int32_t N, L, P, H, M;    // N = P + L, P = H + M
    int32_t field, mode;
    int32_t suf_len;          // padded suffix table length
    int32_t goff[BT_MAX_L + 2];
    int32_t geo_imin, geo_len;
    int32_t n_items;          // ceil(2^P / 2^BT_LOW_BITS)
    int32_t cls;              // 1: suffix table of recombined classes (goff in class units)
    int64_t item_begin;       // first work item of this job in the launch's numbering
    int64_t item_offset;      // job-local index of that first item (0 unless a launch covers part of a job)
    int64_t part_off;         // index of the job's item 0 in the partials array
    int64_t prm_off;          // index of the job's parameters in the parameter array
    int64_t off_suf;          // element offset in the suffix arena
    int64_t off_ph, off_pm;   // entry offsets in the prefix-table arena
    int64_t off_pow, off_geo; // entry offsets in the power-table arena
    // trees given move by move (steps.cu): branches per node and the number of
    // prefixes, middle-block prefixes and suffixes (b^P, b^M, b^L)
    int32_t branches, pad2;
    int64_t n_prefix, n_mid, n_suffix;
};

struct bt_pentry {            // one entry of a two-level prefix table
    double R64;               // backward-relative partial sum sum_t u^{l_t - l_end}
    float R_hi, R_lo;
    int16_t lvl, mx, mn, D;   // end level, max level, min level, level sum
    float Q;                  // level-weighted backward sum sum_t l_t u^{l_t - l_end}
    int32_t pad;
};

struct bt_spentry {           // one entry of a time-varying two-level prefix table (steps.cu)
    double rho, irho, R, mx, mn, e, ie, w;              // FP64
    float2 rho2, irho2, R2, mx2, mn2, e2, ie2, w2;      // the same as FP32 pairs
};

struct bt_pow {               // u^e for some exponent e, in FP64 and as an FP32 pair
    double v;
    float hi, lo;
};

// Numeric parameters of a job, computed on the device from the option.
struct bt_jparams {
    double u, d, p, disc, lnu;
    double S0, K;
    double NKoS0, KoS0, S0oN;
    double fmin, fmax;
    double W[BT_MAX_L + 1];          // suffix-group weights p^k (1-p)^{L-k}
    double wl[BT_LOW_BITS + 1];      // p^c (1-p)^{Plo-c}, Plo = min(P, BT_LOW_BITS)
    double wh[BT_MAX_N_EXACT + 1];   // p^c (1-p)^{Phi-c}, Phi = P - Plo
    float2 W2[BT_MAX_L + 1];         // FP32 pairs of the above
    float2 wl2[BT_LOW_BITS + 1];
    float2 NKoS0_2, KoS0_2, S0oN_2, S0_2, K_2;
    float fmin_f, fmax_f;
    int32_t gexp;                    // FP32 split grid of f: f_hi is a multiple of 2^gexp
    int32_t ok;                      // 0 if the device found p outside (0,1)
};

struct bt_exact_args {
    const bt_option *opts;
    const bt_job *jobs;
    const bt_jparams *prm;
    int32_t n_jobs;
    int32_t shard, n_shards;
    int32_t pad;
    int64_t n_run_items;      // items executed by this launch
    const float2 *suf32;
    const double *suf64;
    const bt_pentry *ph;
    const bt_pentry *pm;
    const bt_pow *pw;
    double2 *partials;        // per global work item: (call slot, put slot)
    unsigned long long *counter;
    const float *sufd;        // derivative pass: df_s/du table
    double4 *partials4;       // derivative pass: per item (V, sum w pay k, dV/du part, ITM weight)
};

#ifdef __cplusplus
extern "C" {
#endif
// Kernel launchers (exact.cu). Each returns a cudaError_t as int.
int bt_launch_params(const bt_option *d_opts, const bt_job *d_jobs, bt_jparams *d_prm, int n_jobs,
                     void *stream);
int bt_launch_tables(const bt_job *d_jobs, const bt_jparams *d_prm, int n_jobs, int max_len, int prec,
                     float2 *suf32, double *suf64, bt_pentry *ph, bt_pentry *pm, bt_pow *pw, void *stream);
// As bt_launch_tables, also writing the suffix derivative table df_s/du (FP32,
// same positions as the suffix table, 0 in the padding).
int bt_launch_tables_d(const bt_job *d_jobs, const bt_jparams *d_prm, int n_jobs, int max_len, float2 *suf32,
                       float *sufd, bt_pentry *ph, bt_pentry *pm, bt_pow *pw, void *stream);
int bt_launch_exact(const bt_exact_args *a, int prec, int grid, void *stream);
int bt_launch_finalize(const bt_job *d_jobs, const bt_jparams *d_prm, int n_jobs, const double2 *partials,
                       int shard, int n_shards, int prec, bt_result *d_out, void *stream);
int bt_exact_grid_size(int prec, int device);
int bt_launch_steps_params(const bt_option *d_opts, const bt_job *d_jobs, const double *d_steps, bt_jparams *d_prm,
                           int n_jobs, void *stream);
int bt_launch_steps_tables(const bt_job *d_jobs, const bt_jparams *d_prm, const double *d_steps, int n_jobs,
                           int max_len, int prec, float4 *suf32, double2 *suf64, bt_spentry *tab, void *stream);
int bt_launch_steps(const bt_exact_args *a, const bt_spentry *tab, int prec, int device, void *stream);
int bt_launch_greeks(const bt_exact_args *a, int grid, void *stream);
int bt_launch_greeks_finalize(const bt_job *d_jobs, int n_jobs, const double4 *partials, double4 *sums,
                              void *stream);
#ifdef __cplusplus
}
#endif
