// Host-side declarations shared by the runtime's translation units.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <vector>

#include "bt_internal.h"

#include <mutex>

struct bt_ctx {
    int device;
    size_t budget;
    std::atomic<size_t> used;
    cudaStream_t stream;
    int n_sm;
    int grid32, grid64;
    // scratch reused by bt_price_exact (grown on demand, freed with the context)
    std::mutex cache_mu;
    void *cache;
    size_t cache_bytes;
};

bt_status bt_fail(bt_status s, const char *fmt, ...);
bt_status bt_cuda_fail(int err, const char *what);
bt_status ctx_alloc(bt_ctx *c, size_t bytes, void **p);
void ctx_free(bt_ctx *c, void *p, size_t bytes);
cudaStream_t ctx_stream(bt_ctx *c, void *s);
bt_status ctx_scratch(bt_ctx *c, size_t bytes, void **p);
bt_status host_tree(const bt_option *o, double *u, double *d, double *p);
bt_status validate_option(const bt_option *o, int idx, int max_n);
int exact_split_L(int N);
int exact_split_L_fp64(int N);
void payoff_field(int payoff, int *field, int *mode);
// true if the tree has fewer than 2^BT_PER_PATH_MIN_NEFF_LOG2 effective
// paths (the per-path FP32 pass then does not meet 1e-9; the option takes a
// pass that rounds no single path). Needs a validated option.
bool tree_skewed(const bt_option &o);
void fill_job_shape(bt_job &J, int N, int field, int mode, int prec, bool skewed);
bt_status plan_jobs(const bt_option *opts, int n, int prec, std::vector<bt_job> &jobs, int64_t *n_items,
                    int64_t *payoff_paths, int64_t *path_evals, int max_n);
void plan_one_job(const bt_option *opts, int n, int i, bt_job *J, int *step, int prec);
