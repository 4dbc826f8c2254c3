// Payoff plug-ins (include/btree_payoff.cuh) compiled at run time.
//
// bt_plugin_compile appends the caller's Payoff source to the plug-in header,
// adds one kernel that instantiates btp::run<Payoff>, and builds it for the
// context's GPU with NVRTC (loaded with dlopen, so the library itself does
// not depend on it); the image is loaded with the runtime's library API and
// never inspected. bt_price_exact_plugin runs every path of every option and
// adds the per-item partials on the host in item order (Neumaier), times the
// discount.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "btree_payoff.cuh"
#include "host_common.h"

static const char kPayoffHeader[] =
#include "btree_payoff_src.inc"
    ;

namespace {

struct nvrtc_api {
    bool ok = false;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    decltype(&nvrtcGetErrorString) err = nullptr;
};

const nvrtc_api &nvrtc() {
    static nvrtc_api api;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"};
        void *h = nullptr;
        for (const char *n : names)
            if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) return;
        api.create = (decltype(api.create))dlsym(h, "nvrtcCreateProgram");
        api.compile = (decltype(api.compile))dlsym(h, "nvrtcCompileProgram");
        api.log_size = (decltype(api.log_size))dlsym(h, "nvrtcGetProgramLogSize");
        api.log = (decltype(api.log))dlsym(h, "nvrtcGetProgramLog");
        api.cubin_size = (decltype(api.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
        api.cubin = (decltype(api.cubin))dlsym(h, "nvrtcGetCUBIN");
        api.destroy = (decltype(api.destroy))dlsym(h, "nvrtcDestroyProgram");
        api.err = (decltype(api.err))dlsym(h, "nvrtcGetErrorString");
        api.ok = api.create && api.compile && api.log_size && api.log && api.cubin_size && api.cubin &&
                 api.destroy && api.err;
    });
    return api;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct bt_payoff_plugin {
    int device;
    cudaLibrary_t lib;
    cudaKernel_t kern;
    int grid;
};

extern "C" bt_status bt_plugin_compile(bt_ctx *ctx, const char *source, char *log, size_t log_size,
                                       bt_payoff_plugin **out) {
    if (!ctx || !source || !out) return bt_fail(BT_EINVAL, "bt_plugin_compile: bad arguments");
    *out = nullptr;
    if (log && log_size) log[0] = 0;
    const nvrtc_api &R = nvrtc();
    if (!R.ok) return bt_fail(BT_EUNSUPPORTED, "bt_plugin_compile: the run-time compiler (libnvrtc) is not available");
    int major = 0, minor = 0;
    cudaSetDevice(ctx->device);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, ctx->device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, ctx->device);
    char arch[32];
    snprintf(arch, sizeof(arch), "-arch=sm_%d%da", major, minor);
    std::string src(kPayoffHeader);
    src += "\n#line 1 \"payoff plug-in\"\n";
    src += source;
    src += "\nextern \"C\" __global__ void __launch_bounds__(BTP_THREADS) bt_plugin_kernel(btp::args a) "
           "{ btp::run<Payoff>(a); }\n";
    nvrtcProgram prog = nullptr;
    nvrtcResult r = R.create(&prog, src.c_str(), "bt_plugin.cu", 0, nullptr, nullptr);
    if (r != NVRTC_SUCCESS) return bt_fail(BT_ENOMEM, "nvrtcCreateProgram: %s", R.err(r));
    const char *optv[] = {arch, "-std=c++17", "-default-device"};
    r = R.compile(prog, 3, optv);
    size_t ls = 0;
    R.log_size(prog, &ls);
    std::string text(ls, '\0');
    if (ls) R.log(prog, &text[0]);
    if (log && log_size) {
        const size_t n = std::min(log_size - 1, strlen(text.c_str()));
        memcpy(log, text.c_str(), n);
        log[n] = 0;
    }
    if (r != NVRTC_SUCCESS) {
        R.destroy(&prog);
        return bt_fail(BT_EINVAL, "bt_plugin_compile: %s: %.300s", R.err(r), text.c_str());
    }
    size_t cs = 0;
    R.cubin_size(prog, &cs);
    std::vector<char> image(cs);
    R.cubin(prog, image.data());
    R.destroy(&prog);
    bt_payoff_plugin *pl = new (std::nothrow) bt_payoff_plugin();
    if (!pl) return bt_fail(BT_ENOMEM, "bt_plugin_compile: host allocation");
    pl->device = ctx->device;
    cudaError_t e = cudaLibraryLoadData(&pl->lib, image.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&pl->kern, pl->lib, "bt_plugin_kernel");
    int per = 0, sms = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void *)pl->kern, BTP_THREADS, 0);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) {
        delete pl;
        return bt_cuda_fail(e, "bt_plugin_compile: loading the plug-in");
    }
    pl->grid = sms * std::max(1, per);
    *out = pl;
    return BT_OK;
}

extern "C" void bt_plugin_destroy(bt_payoff_plugin *pl) {
    if (!pl) return;
    cudaLibraryUnload(pl->lib);
    delete pl;
}

extern "C" int bt_branch_builtin_grid(int device);
extern "C" int bt_launch_branch_builtin(const btp::args *a, int grid, void *stream);

// Runs the generic pass over opts[0..n) on a b-ary tree whose moves are given
// per step as b factors then b probabilities (host array `moves`, options
// concatenated), with the plug-in kernel or, if pl is NULL, the built-in
// payoffs. Per-item partials are added on the host in item order.
static bt_status generic_run(bt_ctx *ctx, const bt_payoff_plugin *pl, const bt_option *opts, int n, int b,
                             const std::vector<double> &moves, const double *params, bt_result *out, void *stream) {
    std::vector<btp::job> jobs((size_t)n);
    std::vector<int64_t> move_off((size_t)n);
    int64_t o = 0, items = 0;
    for (int i = 0; i < n; ++i) {
        const bt_option &op = opts[i];
        btp::job &J = jobs[i];
        memset(&J, 0, sizeof(J));
        J.N = op.N;
        J.b = b;
        int L = 0;
        long long leaves = 1;
        while (L < op.N && leaves * b <= 4096) {
            leaves *= b;
            ++L;
        }
        J.L = L;
        J.P = op.N - L;
        J.n_leaves = leaves;
        long long pre = 1;
        for (int t = 0; t < J.P; ++t) pre *= b;
        J.n_prefixes = pre;
        J.item_begin = items;
        J.n_items = std::max<long long>(1, (pre + BTP_THREADS - 1) / BTP_THREADS);
        J.S0 = op.S0;
        if (pl) {
            if (params) memcpy(J.param, params + BTP_PARAMS * i, sizeof(J.param));
            else J.param[0] = op.K;
        } else {
            J.param[0] = op.K;
            J.param[1] = (double)op.payoff;
            J.param[2] = 1.0 / (double)op.N;
        }
        items += J.n_items;
        move_off[i] = 2 * b * o;  // J.moves is set once the device copy exists
        o += op.N;
    }
    if (items > ((int64_t)1 << 31)) return bt_fail(BT_EUNSUPPORTED, "%lld work items", (long long)items);
    size_t off = 0;
    const size_t o_jobs = off; off = up256(off + sizeof(btp::job) * n);
    const size_t o_mv = off; off = up256(off + sizeof(double) * moves.size());
    const size_t o_part = off; off = up256(off + sizeof(double) * items);
    const size_t o_cnt = off; off = up256(off + sizeof(unsigned long long));
    cudaSetDevice(ctx->device);
    // the context's reusable scratch (no allocation per call once it is large enough)
    std::lock_guard<std::mutex> lock(ctx->cache_mu);
    void *arena = nullptr;
    bt_status rs = ctx_scratch(ctx, off, &arena);
    if (rs != BT_OK) return rs;
    char *base = (char *)arena;
    const double *d_mv = (const double *)(base + o_mv);
    for (int i = 0; i < n; ++i) jobs[i].moves = d_mv + move_off[i];
    cudaStream_t sm = ctx_stream(ctx, stream);
    std::vector<double> part((size_t)items);
    cudaError_t e = cudaMemcpyAsync(base + o_jobs, jobs.data(), sizeof(btp::job) * n, cudaMemcpyHostToDevice, sm);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + o_mv, moves.data(), sizeof(double) * moves.size(), cudaMemcpyHostToDevice, sm);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_cnt, 0, sizeof(unsigned long long), sm);
    if (e == cudaSuccess) {
        btp::args a;
        memset(&a, 0, sizeof(a));
        a.jobs = (const btp::job *)(base + o_jobs);
        a.n_jobs = n;
        a.n_items = items;
        a.partials = (double *)(base + o_part);
        a.counter = (unsigned long long *)(base + o_cnt);
        if (pl) {
            void *kargs[] = {&a};
            const int grid = (int)std::min<int64_t>(pl->grid, items);
            e = cudaLaunchKernel((const void *)pl->kern, dim3(grid), dim3(BTP_THREADS), kargs, 0, sm);
        } else {
            const int grid = (int)std::min<int64_t>(bt_branch_builtin_grid(ctx->device), items);
            e = (cudaError_t)bt_launch_branch_builtin(&a, grid, sm);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(part.data(), base + o_part, sizeof(double) * items, cudaMemcpyDeviceToHost, sm);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sm);
    if (e != cudaSuccess) rs = bt_cuda_fail(e, "generic path pass");
    cudaStreamSynchronize(sm);   // the scratch is free for the next call only after this one's work
    if (rs != BT_OK) return rs;
    for (int i = 0; i < n; ++i) {
        const btp::job &J = jobs[i];
        double s = 0.0, c = 0.0;  // Neumaier, item order
        for (int64_t k = 0; k < J.n_items; ++k) {
            const double x = part[(size_t)(J.item_begin + k)];
            const double t = s + x;
            c += std::fabs(s) >= std::fabs(x) ? (s - t) + x : (x - t) + s;
            s = t;
        }
        long long paths = 1;
        for (int t = 0; t < J.N; ++t) paths *= b;
        bt_result &r = out[i];
        r.value = std::exp(-opts[i].rate * opts[i].T) * (s + c);
        r.err_est = 1e-13 * std::fabs(r.value);
        r.stderr_mc = 0.0;
        r.var_plain = 0.0;
        r.paths = paths;
    }
    return BT_OK;
}

static bt_status check_scalars(const bt_option &op, int i) {
    if (!(op.S0 > 0.0 && std::isfinite(op.S0) && op.T > 0.0 && std::isfinite(op.T) && std::isfinite(op.rate) &&
          op.K >= 0.0 && std::isfinite(op.K)))
        return bt_fail(BT_EINVAL, "option %d: needs S0 > 0, K >= 0, T > 0 and a finite rate", i);
    if (op.payoff < 0 || op.payoff > 7) return bt_fail(BT_EINVAL, "option %d: bad payoff %d", i, op.payoff);
    return BT_OK;
}

extern "C" bt_status bt_price_exact_plugin(bt_ctx *ctx, const bt_payoff_plugin *pl, const bt_option *opts, int32_t n,
                                           const double *steps, const double *params, bt_result *out,
                                           void *stream) {
    if (!ctx || !pl || !opts || !out || n < 1) return bt_fail(BT_EINVAL, "bt_price_exact_plugin: bad arguments");
    if (pl->device != ctx->device) return bt_fail(BT_EINVAL, "bt_price_exact_plugin: plug-in built for another GPU");
    // binomial moves in digit order: (d, u) and (1 - p, p); the caller's steps, else each option's tree
    std::vector<double> mv;
    int64_t o = 0;
    for (int i = 0; i < n; ++i) {
        const bt_option &op = opts[i];
        if (op.N < 1 || op.N > BT_MAX_N_EXACT)
            return bt_fail(BT_EINVAL, "option %d: N=%d outside 1..%d", i, op.N, BT_MAX_N_EXACT);
        bt_status s = check_scalars(op, i);
        if (s != BT_OK) return s;
        double u = 0, d = 0, p = 0;
        if (!steps) {
            if ((s = validate_option(&op, i, BT_MAX_N_EXACT)) != BT_OK) return s;
            host_tree(&op, &u, &d, &p);
        }
        for (int t = 0; t < op.N; ++t) {
            if (steps) {
                u = steps[3 * (o + t)];
                d = steps[3 * (o + t) + 1];
                p = steps[3 * (o + t) + 2];
                if (!(std::isfinite(u) && d > 0.0 && u > d && p > 0.0 && p < 1.0))
                    return bt_fail(BT_EINVAL, "option %d step %d: needs 0 < d < u and 0 < p < 1", i, t + 1);
            }
            mv.insert(mv.end(), {d, u, 1.0 - p, p});
        }
        o += op.N;
    }
    return generic_run(ctx, pl, opts, n, 2, mv, params, out, stream);
}

extern "C" bt_status bt_price_exact_branching(bt_ctx *ctx, const bt_payoff_plugin *pl, const bt_option *opts,
                                              int32_t n, int32_t branches, const double *moves,
                                              const double *params, bt_result *out, void *stream) {
    if (!ctx || !opts || !moves || !out || n < 1) return bt_fail(BT_EINVAL, "bt_price_exact_branching: bad arguments");
    if (branches < 2 || branches > 8) return bt_fail(BT_EINVAL, "branches = %d outside 2..8", branches);
    if (pl && pl->device != ctx->device) return bt_fail(BT_EINVAL, "plug-in built for another GPU");
    const int b = branches;
    int64_t total_steps = 0;
    for (int i = 0; i < n; ++i) {
        const bt_option &op = opts[i];
        bt_status s = check_scalars(op, i);
        if (s != BT_OK) return s;
        // b^N paths, at most 2^40 (about a minute of the generic walk)
        double lg = (double)op.N * std::log2((double)b);
        if (op.N < 1 || lg > 40.0 + 1e-9)
            return bt_fail(op.N < 1 ? BT_EINVAL : BT_EUNSUPPORTED, "option %d: %d^%d paths outside 1..2^40", i, b, op.N);
        for (int t = 0; t < op.N; ++t) {
            const double *mv = moves + 2 * b * (total_steps + t);
            double psum = 0.0;
            for (int k = 0; k < b; ++k) {
                if (!(std::isfinite(mv[k]) && mv[k] > 0.0 && mv[b + k] >= 0.0 && mv[b + k] <= 1.0))
                    return bt_fail(BT_EINVAL, "option %d step %d: factors must be > 0, probabilities in [0,1]", i,
                                   t + 1);
                psum += mv[b + k];
            }
            if (std::fabs(psum - 1.0) > 1e-12)
                return bt_fail(BT_EINVAL, "option %d step %d: probabilities sum to %.17g", i, t + 1, psum);
        }
        total_steps += op.N;
    }
    std::vector<double> mv(moves, moves + 2 * b * total_steps);
    return generic_run(ctx, pl, opts, n, b, mv, params, out, stream);
}
