// Allocation-free variant of the exhaustive pricing call.
//
// For callers that must not allocate device memory while they run: an
// application that has handed the device to its own allocator, or a latency-
// sensitive loop that cannot afford cudaMalloc/cudaFree (cudaFree synchronises
// the whole device). Every intermediate buffer of the pass lives in one
// file-scope device array of fixed size; the call allocates nothing on the
// device or the host heap.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "bt_internal.h"
#include "host_common.h"

#define BT_NOALLOC_MAX_DEVICES 64

// The scratch array. Every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[BT_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;                               // serialises calls (one array per device)
void *g_scratch_ptr[BT_NOALLOC_MAX_DEVICES];            // device address of the array, per device
int g_grid32[BT_NOALLOC_MAX_DEVICES], g_grid64[BT_NOALLOC_MAX_DEVICES];

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Waits for the call's stream when the call returns early after enqueuing
// work, so that the lock (released after this guard) is never given to a
// later call while this call's kernels may still use the shared array.
struct drain_on_exit {
    cudaStream_t st;
    bool armed = false;
    ~drain_on_exit() {
        if (armed) cudaStreamSynchronize(st);
    }
};
}  // namespace

extern "C" bt_status bt_price_exact_noalloc(const bt_option *opts, int32_t n, bt_precision prec, bt_result *out,
                                            void *stream) {
    if (!opts || !out || n < 1) return bt_fail(BT_EINVAL, "bt_price_exact_noalloc: bad arguments");
    if (n > BT_NOALLOC_MAX_OPTIONS)
        return bt_fail(BT_EUNSUPPORTED, "bt_price_exact_noalloc: %d options exceed the limit of %d", n,
                       BT_NOALLOC_MAX_OPTIONS);
    if (prec != BT_PREC_FP64 && prec != BT_PREC_FP32_COMP) return bt_fail(BT_EINVAL, "bad precision %d", (int)prec);

    // Plan on the stack (same split and pairing as bt_price_exact).
    bt_job jobs[BT_NOALLOC_MAX_OPTIONS];
    int nj = 0;
    int64_t items = 0, suf = 0, ph = 0, pm = 0, pw = 0;
    int max_len = 0;
    for (int i = 0; i < n; ++i) {
        bt_status s = validate_option(&opts[i], i, BT_MAX_N_EXACT);
        if (s != BT_OK) return s;
        if (prec == BT_PREC_FP32_COMP) {
            double u, d, p;
            host_tree(&opts[i], &u, &d, &p);
            if (p < 0.004 || 1.0 - p < 0.004)
                return bt_fail(BT_EUNSUPPORTED, "option %d: p = %.6g; FP32_COMP needs min(p,1-p) >= 0.004", i, p);
        }
    }
    for (int i = 0; i < n;) {
        bt_job &J = jobs[nj];
        memset(&J, 0, sizeof(J));
        int step = 1;
        plan_one_job(opts, n, i, &J, &step, prec);
        J.item_begin = items;
        J.item_offset = 0;
        J.part_off = items;
        J.prm_off = nj;
        J.off_suf = suf;
        J.off_ph = ph;
        J.off_pm = pm;
        J.off_pow = pw;
        J.off_geo = pw + 2 * J.N + 3;
        items += J.n_items;
        suf += J.suf_len;
        ph += 1ll << J.H;
        pm += 1ll << J.M;
        pw += 2 * J.N + 3 + J.geo_len;
        int64_t len = (1ll << J.L) + J.suf_len + (1ll << J.H) + (1ll << J.M) + 2 * J.N + 3 + J.geo_len;
        if (len > max_len) max_len = (int)len;
        ++nj;
        i += step;
    }

    // Carve the array.
    size_t off = 0;
    const size_t o_opts = off; off = up256(off + sizeof(bt_option) * n);
    const size_t o_jobs = off; off = up256(off + sizeof(bt_job) * nj);
    const size_t o_prm = off; off = up256(off + sizeof(bt_jparams) * nj);
    const size_t o_suf = off; off = up256(off + (prec == BT_PREC_FP64 ? sizeof(double) : sizeof(float2)) * suf);
    const size_t o_ph = off; off = up256(off + sizeof(bt_pentry) * ph);
    const size_t o_pm = off; off = up256(off + sizeof(bt_pentry) * pm);
    const size_t o_pw = off; off = up256(off + sizeof(bt_pow) * pw);
    const size_t o_part = off; off = up256(off + sizeof(double2) * items);
    const size_t o_out = off; off = up256(off + sizeof(bt_result) * n);
    const size_t o_cnt = off; off = up256(off + sizeof(unsigned long long));
    if (off > (size_t)BT_NOALLOC_SCRATCH_BYTES)
        return bt_fail(BT_EUNSUPPORTED,
                       "bt_price_exact_noalloc: this batch needs %zu bytes of scratch; the fixed array holds %zu "
                       "(use bt_price_exact, or fewer or smaller options)",
                       off, (size_t)BT_NOALLOC_SCRATCH_BYTES);

    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bt_cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= BT_NOALLOC_MAX_DEVICES) return bt_fail(BT_EUNSUPPORTED, "device %d out of range", dev);
    if (!g_scratch_ptr[dev]) {
        // One-time set-up on this device (the device is current): the host
        // symbol is only a stand-in, so ask the runtime for the device address.
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return bt_cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        const int g32 = bt_exact_grid_size(BT_PREC_FP32_COMP, dev);
        if (g32 < 0) return bt_cuda_fail(-g32, "kernel attributes (FP32 pass)");
        const int g64 = bt_exact_grid_size(BT_PREC_FP64, dev);
        if (g64 < 0) return bt_cuda_fail(-g64, "kernel attributes (FP64 pass)");
        g_grid32[dev] = g32;
        g_grid64[dev] = g64;
        g_scratch_ptr[dev] = p;
    }
    char *base = (char *)g_scratch_ptr[dev];
    bt_option *d_opts = (bt_option *)(base + o_opts);
    bt_job *d_jobs = (bt_job *)(base + o_jobs);
    bt_jparams *d_prm = (bt_jparams *)(base + o_prm);
    float2 *d_suf32 = prec == BT_PREC_FP64 ? nullptr : (float2 *)(base + o_suf);
    double *d_suf64 = prec == BT_PREC_FP64 ? (double *)(base + o_suf) : nullptr;
    bt_pentry *d_ph = (bt_pentry *)(base + o_ph);
    bt_pentry *d_pm = (bt_pentry *)(base + o_pm);
    bt_pow *d_pw = (bt_pow *)(base + o_pw);
    double2 *d_part = (double2 *)(base + o_part);
    bt_result *d_out = (bt_result *)(base + o_out);
    unsigned long long *d_cnt = (unsigned long long *)(base + o_cnt);

    cudaStream_t st = (cudaStream_t)stream;
    drain_on_exit drain{st};
    drain.armed = true;   // from the first copy on, every return waits for the stream
    e = cudaMemcpyAsync(d_opts, opts, sizeof(bt_option) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_jobs, jobs, sizeof(bt_job) * nj, cudaMemcpyHostToDevice, st);
    // The array keeps the previous call's contents: clear what must start at zero.
    if (e == cudaSuccess) e = cudaMemsetAsync(d_part, 0, sizeof(double2) * items, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return bt_cuda_fail(e, "bt_price_exact_noalloc: copies");
    int le = bt_launch_params(d_opts, d_jobs, d_prm, nj, st);
    if (le) return bt_cuda_fail(le, "params kernel");
    le = bt_launch_tables(d_jobs, d_prm, nj, max_len, prec, d_suf32, d_suf64, d_ph, d_pm, d_pw, st);
    if (le) return bt_cuda_fail(le, "tables kernel");
    bt_exact_args a;
    memset(&a, 0, sizeof(a));
    a.opts = d_opts;
    a.jobs = d_jobs;
    a.prm = d_prm;
    a.n_jobs = nj;
    a.shard = 0;
    a.n_shards = 1;
    a.n_run_items = items;
    a.suf32 = d_suf32;
    a.suf64 = d_suf64;
    a.ph = d_ph;
    a.pm = d_pm;
    a.pw = d_pw;
    a.partials = d_part;
    a.counter = d_cnt;
    le = bt_launch_exact(&a, prec, prec == BT_PREC_FP64 ? g_grid64[dev] : g_grid32[dev], st);
    if (le) return bt_cuda_fail(le, "path-sum kernel");
    le = bt_launch_finalize(d_jobs, d_prm, nj, d_part, 0, 1, prec, d_out, st);
    if (le) return bt_cuda_fail(le, "finalize kernel");
    e = cudaMemcpyAsync(out, d_out, sizeof(bt_result) * n, cudaMemcpyDeviceToHost, st);
    // Return only after this call's GPU work is done, so no later call can
    // overwrite the array while it is in use.
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bt_cuda_fail(e, "bt_price_exact_noalloc");
    drain.armed = false;   // drained above
    return BT_OK;
}
