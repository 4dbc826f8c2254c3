"""Python binding of libbtree: the C ABI of include/btree.h, same names.

Argument marshalling only -- every step of the computation runs in the CUDA
library. Importing this module loads ``lib/libbtree.so`` and raises if it is
missing: there is no CPU fallback.

Streams: pass ``stream=None`` for the context's own stream, an integer
``cudaStream_t`` handle, or a ``torch.cuda.Stream`` (its ``cuda_stream``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libbtree.so")

BT_OK, BT_EINVAL, BT_ENOMEM, BT_EBUDGET, BT_ECUDA, BT_ETIMEOUT, BT_EUNSUPPORTED = range(7)
BT_PREC_FP64, BT_PREC_FP32_COMP = 0, 1
BT_TREE_CRR, BT_TREE_SEYDEL, BT_TREE_EXPLICIT = 0, 1, 2
(BT_EURO_CALL, BT_EURO_PUT, BT_ASIAN_ARITH_CALL, BT_ASIAN_ARITH_PUT, BT_ASIAN_GEO_CALL, BT_ASIAN_GEO_PUT,
 BT_LOOKBACK_FIXED_CALL, BT_LOOKBACK_FIXED_PUT) = range(8)


class BtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_status_name(status), msg))
        self.status = status


def _status_name(s):
    return {0: "BT_OK", 1: "BT_EINVAL", 2: "BT_ENOMEM", 3: "BT_EBUDGET", 4: "BT_ECUDA", 5: "BT_ETIMEOUT",
            6: "BT_EUNSUPPORTED"}.get(s, "BT_%d" % s)


class bt_option(C.Structure):
    _fields_ = [("N", C.c_int32), ("tree_kind", C.c_int32), ("payoff", C.c_int32), ("pad", C.c_int32),
                ("S0", C.c_double), ("K", C.c_double), ("rate", C.c_double), ("sigma", C.c_double),
                ("T", C.c_double), ("u", C.c_double), ("d", C.c_double), ("p", C.c_double)]


class bt_result(C.Structure):
    _fields_ = [("value", C.c_double), ("err_est", C.c_double), ("stderr_mc", C.c_double),
                ("var_plain", C.c_double), ("paths", C.c_int64)]


class bt_exact_plan_info(C.Structure):
    _fields_ = [("n_options", C.c_int32), ("n_jobs", C.c_int32), ("n_items", C.c_int64),
                ("payoff_paths", C.c_int64), ("path_evaluations", C.c_int64), ("device_bytes", C.c_size_t),
                ("h2d_bytes", C.c_size_t), ("d2h_bytes", C.c_size_t)]


class bt_server_cfg(C.Structure):
    _fields_ = [("max_active", C.c_int32), ("n_streams", C.c_int32), ("max_items_per_launch", C.c_int32),
                ("use_fp64", C.c_int32), ("device_budget_bytes", C.c_size_t)]


class bt_server_stats_t(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("launches", C.c_int64),
                ("items", C.c_int64), ("active", C.c_int32), ("pending", C.c_int32), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("max_ms", C.c_double),
                ("throughput_rps", C.c_double), ("paths_per_s", C.c_double), ("busy_s", C.c_double),
                ("peak_active", C.c_int32), ("reserved", C.c_int32), ("pool_bytes", C.c_int64)]


OPTION_DTYPE = np.dtype([("N", "<i4"), ("tree_kind", "<i4"), ("payoff", "<i4"), ("pad", "<i4"),
                         ("S0", "<f8"), ("K", "<f8"), ("rate", "<f8"), ("sigma", "<f8"), ("T", "<f8"),
                         ("u", "<f8"), ("d", "<f8"), ("p", "<f8")])
RESULT_DTYPE = np.dtype([("value", "<f8"), ("err_est", "<f8"), ("stderr_mc", "<f8"), ("var_plain", "<f8"),
                         ("paths", "<i8")])
assert OPTION_DTYPE.itemsize == C.sizeof(bt_option) == 80
assert RESULT_DTYPE.itemsize == C.sizeof(bt_result) == 40

_lib = None
_vp, _i32, _i64, _sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t


def _proto(L, name, args, res=C.c_int):
    f = getattr(L, name)
    f.argtypes = args
    f.restype = res
    return f


def lib():
    """Load libbtree (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libbtree.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        _proto(L, "bt_version", [], C.c_char_p)
        _proto(L, "bt_status_str", [C.c_int], C.c_char_p)
        _proto(L, "bt_last_error", [_vp], C.c_char_p)
        _proto(L, "bt_create", [C.c_int, _sz, C.POINTER(_vp)])
        _proto(L, "bt_destroy", [_vp], None)
        _proto(L, "bt_device_bytes", [_vp], _sz)
        _proto(L, "bt_tree_params", [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)])
        _proto(L, "bt_price_exact", [_vp, _vp, _i32, C.c_int, _vp, _vp])
        _proto(L, "bt_exact_plan_create", [_vp, _vp, _i32, C.c_int, C.POINTER(_vp)])
        _proto(L, "bt_exact_plan_run", [_vp, _vp])
        _proto(L, "bt_exact_plan_run_shard", [_vp, _i32, _i32, _vp])
        _proto(L, "bt_exact_plan_read", [_vp, _vp, _vp])
        _proto(L, "bt_exact_plan_partials", [_vp, _vp, _vp, _vp, _vp])
        _proto(L, "bt_exact_plan_job", [_vp, _i32, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_i32),
                                        C.POINTER(_i32), C.POINTER(_i32)])
        _proto(L, "bt_exact_plan_info_get", [_vp, C.POINTER(bt_exact_plan_info)])
        _proto(L, "bt_exact_split", [_vp, C.c_int, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_i32),
                                     C.POINTER(C.c_int64)])
        _proto(L, "bt_exact_plan_destroy", [_vp], None)
        _proto(L, "bt_exact_plan_kernel_ms", [_vp, C.POINTER(C.c_float)])
        _proto(L, "bt_price_exact_noalloc", [_vp, _i32, C.c_int, _vp, _vp])
        _proto(L, "bt_price_mc", [_vp, _vp, _i32, _i32, _i64, C.c_uint64, _vp, _vp])
        _proto(L, "bt_price_mc_ex", [_vp, _vp, _i32, _i32, _i64, C.c_uint64, _i32, _vp, _vp, _vp])
        _proto(L, "bt_price_exact_steps", [_vp, _vp, _i32, _vp, C.c_int, _vp, _vp])
        _proto(L, "bt_price_exact_moves", [_vp, _vp, _i32, _i32, _vp, C.c_int, _vp, _vp])
        _proto(L, "bt_plugin_compile", [_vp, C.c_char_p, C.c_char_p, C.c_size_t, C.POINTER(_vp)])
        _proto(L, "bt_price_exact_plugin", [_vp, _vp, _vp, _i32, _vp, _vp, _vp, _vp])
        L.bt_plugin_destroy.argtypes = [_vp]
        L.bt_plugin_destroy.restype = None
        _proto(L, "bt_price_exact_branching", [_vp, _vp, _vp, _i32, _i32, _vp, _vp, _vp, _vp])
        _proto(L, "bt_price_mc_shard", [_vp, _vp, _i32, _i32, _i64, C.c_uint64, _i32, _i32, _vp, _vp, _vp])
        _proto(L, "bt_philox4x32_10", [_vp, _vp, _vp, _vp, _i32])
        _proto(L, "bt_greeks_exact", [_vp, _vp, _i32, C.c_int, _vp, _vp, _vp])
        _proto(L, "bt_server_start", [_vp, C.POINTER(bt_server_cfg), C.POINTER(_vp)])
        _proto(L, "bt_submit", [_vp, _vp, C.c_int, C.POINTER(C.c_uint64)])
        _proto(L, "bt_wait", [_vp, C.c_uint64, _i32, _vp])
        _proto(L, "bt_poll", [_vp, C.c_uint64, _vp, C.POINTER(_i32)])
        _proto(L, "bt_server_stats", [_vp, C.POINTER(bt_server_stats_t)])
        _proto(L, "bt_server_stop", [_vp])
        _proto(L, "bt_serve_replay", [_vp, C.POINTER(bt_server_cfg), _vp, _vp, _i32, _i32, _vp, _vp,
                                      C.POINTER(C.c_double)])
        _lib = L
    return _lib


def _check(status):
    if status != BT_OK:
        raise BtError(status, lib().bt_last_error(None).decode())


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def options_array(opts) -> np.ndarray:
    """List of option dicts (workloads.opt) or a structured array -> bt_option array."""
    if isinstance(opts, np.ndarray) and opts.dtype == OPTION_DTYPE:
        return np.ascontiguousarray(opts)
    if isinstance(opts, dict):
        opts = [opts]
    a = np.zeros(len(opts), dtype=OPTION_DTYPE)
    for k in ("N", "tree_kind", "payoff", "S0", "K", "rate", "sigma", "T", "u", "d", "p"):
        a[k] = [o.get(k, 0) for o in opts]   # one column at a time (per-element writes cost ~10 us each)
    return a


# --- same names as the C ABI -------------------------------------------------
def bt_version() -> str:
    """Library version string (names the GPU architecture it was built for)."""
    return lib().bt_version().decode()


def bt_create(device: int = 0, device_budget_bytes: int = 0):
    """A context on CUDA device `device` (handle); raises BtError(BT_ECUDA) without a usable GPU."""
    h = _vp()
    _check(lib().bt_create(device, device_budget_bytes, C.byref(h)))
    return h


def bt_destroy(ctx):
    """Frees a context and everything it holds."""
    lib().bt_destroy(ctx)


def bt_device_bytes(ctx) -> int:
    """Device bytes the context holds right now."""
    return lib().bt_device_bytes(ctx)


def bt_tree_params(opt):
    """(u, d, p) of the option's tree (CRR, Seydel or explicit), computed on the host."""
    a = options_array(opt)
    u, d, p = C.c_double(), C.c_double(), C.c_double()
    _check(lib().bt_tree_params(a.ctypes.data, C.byref(u), C.byref(d), C.byref(p)))
    return u.value, d.value, p.value


def bt_price_exact(ctx, opts, prec=BT_PREC_FP32_COMP, stream=None) -> np.ndarray:
    """Exact expected values over all 2^N paths; returns a RESULT_DTYPE array in option order."""
    a = options_array(opts)
    out = np.zeros(len(a), dtype=RESULT_DTYPE)
    _check(lib().bt_price_exact(ctx, a.ctypes.data, len(a), prec, out.ctypes.data, _stream(stream)))
    return out


def bt_exact_plan_create(ctx, opts, prec=BT_PREC_FP32_COMP):
    """Plans the exhaustive pass for a batch with the options resident on the device (handle)."""
    a = options_array(opts)
    h = _vp()
    _check(lib().bt_exact_plan_create(ctx, a.ctypes.data, len(a), prec, C.byref(h)))
    return h


def bt_exact_plan_run(plan, stream=None):
    """Enqueues one full pass of the plan on `stream` (asynchronous)."""
    _check(lib().bt_exact_plan_run(plan, _stream(stream)))


def bt_exact_plan_run_shard(plan, shard, n_shards, stream=None):
    """Enqueues the work items i with i % n_shards == shard (numbered across the batch)."""
    _check(lib().bt_exact_plan_run_shard(plan, shard, n_shards, _stream(stream)))


def bt_exact_plan_info_get(plan) -> dict:
    """Sizes of the plan: options, jobs, work items, payoff-paths, device and copy bytes."""
    i = bt_exact_plan_info()
    _check(lib().bt_exact_plan_info_get(plan, C.byref(i)))
    return {k: getattr(i, k) for k, _ in bt_exact_plan_info._fields_}


def bt_exact_plan_read(plan, stream=None) -> np.ndarray:
    """Synchronises and returns the plan's results (RESULT_DTYPE, option order)."""
    n = bt_exact_plan_info_get(plan)["n_options"]
    out = np.zeros(n, dtype=RESULT_DTYPE)
    _check(lib().bt_exact_plan_read(plan, out.ctypes.data, _stream(stream)))
    return out


def bt_exact_plan_partials(plan, stream=None):
    """Per-work-item undiscounted (call, put) partial sums, with each item's job and first prefix."""
    n = bt_exact_plan_info_get(plan)["n_items"]
    part = np.zeros((n, 2))
    job = np.zeros(n, dtype=np.int32)
    first = np.zeros(n, dtype=np.int64)
    _check(lib().bt_exact_plan_partials(plan, part.ctypes.data, job.ctypes.data, first.ctypes.data,
                                        _stream(stream)))
    return part, job, first


def bt_exact_plan_job(plan, j):
    """Job j's option slots and split: opt_call, opt_put, P, L, prefixes_per_item."""
    vals = [_i32() for _ in range(5)]
    _check(lib().bt_exact_plan_job(plan, j, *[C.byref(v) for v in vals]))
    keys = ("opt_call", "opt_put", "P", "L", "prefixes_per_item")
    return {k: v.value for k, v in zip(keys, vals)}


def bt_exact_split(opt, prec=BT_PREC_FP32_COMP):
    """The pass's split for one option priced alone (host only, no device)."""
    a = options_array([opt])
    P, L, ppi, n = _i32(), _i32(), _i32(), C.c_int64()
    _check(lib().bt_exact_split(a.ctypes.data, prec, C.byref(P), C.byref(L), C.byref(ppi), C.byref(n)))
    return {"P": P.value, "L": L.value, "prefixes_per_item": ppi.value, "n_items": n.value}


def bt_exact_plan_kernel_ms(plan) -> float:
    """Duration of the last run's path-sum kernel (CUDA events on its stream)."""
    ms = C.c_float()
    _check(lib().bt_exact_plan_kernel_ms(plan, C.byref(ms)))
    return ms.value


def bt_exact_plan_destroy(plan):
    """Frees a plan."""
    lib().bt_exact_plan_destroy(plan)


BT_MC_PARTITIONED, BT_MC_SHARED = 0, 1


def bt_price_mc(ctx, opts, strata_bits, samples_per_stratum, seed, stream=None) -> np.ndarray:
    """Partitioned Monte Carlo with 2^strata_bits strata (0: plain MC); value and standard error per option."""
    a = options_array(opts)
    out = np.zeros(len(a), dtype=RESULT_DTYPE)
    _check(lib().bt_price_mc(ctx, a.ctypes.data, len(a), strata_bits, samples_per_stratum, seed,
                             out.ctypes.data, _stream(stream)))
    return out


def bt_price_mc_ex(ctx, opts, strata_bits, samples_per_stratum, seed, kind=BT_MC_PARTITIONED,
                   with_strata=False, stream=None):
    """bt_price_mc with the estimator kind (Partitioned or Shared-Sample) and optionally the
    per-stratum (mean, variance, probability) statistics."""
    a = options_array(opts)
    out = np.zeros(len(a), dtype=RESULT_DTYPE)
    per = 1 if kind == BT_MC_SHARED else (1 << strata_bits)
    strata = np.zeros((len(a), per, 3)) if with_strata else None
    _check(lib().bt_price_mc_ex(ctx, a.ctypes.data, len(a), strata_bits, samples_per_stratum, seed, kind,
                                out.ctypes.data, strata.ctypes.data if with_strata else None, _stream(stream)))
    return (out, strata) if with_strata else out


def bt_price_exact_steps(ctx, opts, steps, prec=BT_PREC_FP32_COMP, stream=None) -> np.ndarray:
    """Time-varying trees: steps is a sequence of per-option [N][3] arrays
    (u_t, d_t, p_t), or one array of all options' steps concatenated."""
    a = options_array(opts)
    if isinstance(steps, (list, tuple)):
        steps = np.concatenate([np.asarray(s, dtype=np.float64).reshape(-1, 3) for s in steps])
    st = np.ascontiguousarray(np.asarray(steps, dtype=np.float64).reshape(-1, 3))
    if st.shape[0] != int(a["N"].sum()):
        raise ValueError("steps holds %d steps, the options need %d" % (st.shape[0], int(a["N"].sum())))
    out = np.zeros(len(a), dtype=RESULT_DTYPE)
    _check(lib().bt_price_exact_steps(ctx, a.ctypes.data, len(a), st.ctypes.data, prec, out.ctypes.data,
                                      _stream(stream)))
    return out


def bt_plugin_compile(ctx, source: str):
    """Compiles a payoff plug-in (struct Payoff, see include/btree_payoff.cuh).
    Returns (handle, compiler log); raises BtError with the log on errors."""
    log = C.create_string_buffer(16384)
    h = _vp()
    st = lib().bt_plugin_compile(ctx, source.encode(), log, len(log), C.byref(h))
    if st != BT_OK:
        raise BtError(st, lib().bt_last_error(None).decode() + "\n" + log.value.decode(errors="replace"))
    return h, log.value.decode(errors="replace")


def bt_plugin_destroy(plugin):
    """Frees a compiled plug-in."""
    lib().bt_plugin_destroy(plugin)


def bt_price_exact_plugin(ctx, plugin, opts, steps=None, params=None, stream=None) -> np.ndarray:
    """Every path through the plug-in's state machine (FP64); steps as bt_price_exact_steps or None
    for each option's own tree, params [n][<= 8] handed to the plug-in."""
    a = options_array(opts)
    st = None
    if steps is not None:
        if isinstance(steps, (list, tuple)):
            steps = np.concatenate([np.asarray(s, dtype=np.float64).reshape(-1, 3) for s in steps])
        st = np.ascontiguousarray(np.asarray(steps, dtype=np.float64).reshape(-1, 3))
        if st.shape[0] != int(a["N"].sum()):
            raise ValueError("steps holds %d steps, the options need %d" % (st.shape[0], int(a["N"].sum())))
    pr = None
    if params is not None:
        pr = np.zeros((len(a), 8))
        p_in = np.asarray(params, dtype=np.float64).reshape(len(a), -1)
        pr[:, :p_in.shape[1]] = p_in
    out = np.zeros(len(a), dtype=RESULT_DTYPE)
    _check(lib().bt_price_exact_plugin(ctx, plugin, a.ctypes.data, len(a), None if st is None else st.ctypes.data,
                                       None if pr is None else pr.ctypes.data, out.ctypes.data, _stream(stream)))
    return out


def bt_price_exact_branching(ctx, opts, branches, moves, plugin=None, params=None, stream=None) -> np.ndarray:
    """Trees with `branches` branches per node: moves per option [N][2b]
    (factors of digits 0..b-1, then their probabilities), a list of those or
    one concatenated array."""
    a = options_array(opts)
    if isinstance(moves, (list, tuple)):
        moves = np.concatenate([np.asarray(m, dtype=np.float64).reshape(-1, 2 * branches) for m in moves])
    mv = np.ascontiguousarray(np.asarray(moves, dtype=np.float64).reshape(-1, 2 * branches))
    if mv.shape[0] != int(a["N"].sum()):
        raise ValueError("moves holds %d steps, the options need %d" % (mv.shape[0], int(a["N"].sum())))
    pr = None
    if params is not None:
        pr = np.zeros((len(a), 8))
        p_in = np.asarray(params, dtype=np.float64).reshape(len(a), -1)
        pr[:, :p_in.shape[1]] = p_in
    out = np.zeros(len(a), dtype=RESULT_DTYPE)
    _check(lib().bt_price_exact_branching(ctx, plugin, a.ctypes.data, len(a), branches, mv.ctypes.data,
                                          None if pr is None else pr.ctypes.data, out.ctypes.data,
                                          _stream(stream)))
    return out


def bt_price_exact_moves(ctx, opts, branches, moves, prec=BT_PREC_FP32_COMP, stream=None) -> np.ndarray:
    """Affine passes on trees with `branches` branches per node; moves as for
    bt_price_exact_branching."""
    a = options_array(opts)
    if isinstance(moves, (list, tuple)):
        moves = np.concatenate([np.asarray(m, dtype=np.float64).reshape(-1, 2 * branches) for m in moves])
    mv = np.ascontiguousarray(np.asarray(moves, dtype=np.float64).reshape(-1, 2 * branches))
    if mv.shape[0] != int(a["N"].sum()):
        raise ValueError("moves holds %d steps, the options need %d" % (mv.shape[0], int(a["N"].sum())))
    out = np.zeros(len(a), dtype=RESULT_DTYPE)
    _check(lib().bt_price_exact_moves(ctx, a.ctypes.data, len(a), branches, mv.ctypes.data, prec, out.ctypes.data,
                                      _stream(stream)))
    return out


def bt_price_mc_shard(ctx, opts, strata_bits, samples_per_stratum, seed, shard, n_shards, with_strata=False,
                      stream=None):
    """Strata m = shard + j * n_shards of the Partitioned estimator."""
    a = options_array(opts)
    out = np.zeros(len(a), dtype=RESULT_DTYPE)
    per = ((1 << strata_bits) - shard + n_shards - 1) // n_shards
    strata = np.zeros((len(a), per, 3)) if with_strata else None
    _check(lib().bt_price_mc_shard(ctx, a.ctypes.data, len(a), strata_bits, samples_per_stratum, seed, shard,
                                   n_shards, out.ctypes.data, strata.ctypes.data if with_strata else None,
                                   _stream(stream)))
    return (out, strata) if with_strata else out


def bt_philox4x32_10(ctx, ctr, key) -> np.ndarray:
    """Philox-4x32-10 on the device: counters [n][4] and keys [n][2] (uint32) -> words [n][4]."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(-1, 2))
    out = np.zeros_like(c)
    _check(lib().bt_philox4x32_10(ctx, c.ctypes.data, k.ctypes.data, out.ctypes.data, len(c)))
    return out


def bt_greeks_exact(ctx, opts, prec=BT_PREC_FP32_COMP, stream=None):
    """(values[n], grads[n, 4]) with grads = dV/d(S0, sigma, rate, K)."""
    a = options_array(opts)
    val = np.zeros(len(a))
    grad = np.zeros((len(a), 4))
    _check(lib().bt_greeks_exact(ctx, a.ctypes.data, len(a), prec, val.ctypes.data, grad.ctypes.data,
                                 _stream(stream)))
    return val, grad


def _cfg(max_active=0, n_streams=0, max_items_per_launch=0, use_fp64=0, device_budget_bytes=0):
    return bt_server_cfg(max_active, n_streams, max_items_per_launch, use_fp64, device_budget_bytes)


def bt_server_start(ctx, **cfg):
    """Starts a continuous-batching server (max_active, n_streams, max_items_per_launch, use_fp64,
    device_budget_bytes; 0 = the defaults); returns its handle."""
    h = _vp()
    c = _cfg(**cfg)
    _check(lib().bt_server_start(ctx, C.byref(c), C.byref(h)))
    return h


def bt_submit(srv, opt, prec=BT_PREC_FP32_COMP) -> int:
    """Queues one option at precision `prec`; returns its ticket at once."""
    a = options_array(opt)
    t = C.c_uint64()
    _check(lib().bt_submit(srv, a.ctypes.data, prec, C.byref(t)))
    return t.value


def bt_wait(srv, ticket, timeout_ms=60000) -> np.ndarray:
    """Waits up to timeout_ms for the ticket's result and collects it (BtError(BT_ETIMEOUT) on expiry)."""
    out = np.zeros(1, dtype=RESULT_DTYPE)
    _check(lib().bt_wait(srv, ticket, timeout_ms, out.ctypes.data))
    return out[0]


def bt_poll(srv, ticket):
    """The ticket's result if it is done (collecting it), else None."""
    out = np.zeros(1, dtype=RESULT_DTYPE)
    done = _i32()
    _check(lib().bt_poll(srv, ticket, out.ctypes.data, C.byref(done)))
    return (out[0] if done.value else None)


def bt_server_stats(srv) -> dict:
    """Counts, p50/p99/mean/max latency, throughput and pool figures of the server so far."""
    st = bt_server_stats_t()
    _check(lib().bt_server_stats(srv, C.byref(st)))
    return {k: getattr(st, k) for k, _ in bt_server_stats_t._fields_}


def bt_server_stop(srv):
    """Finishes the queued requests and stops the server (no other call on it may run or follow)."""
    _check(lib().bt_server_stop(srv))


def bt_serve_replay(ctx, opts, arrival_s, mode, **cfg):
    """mode 1: through a server; mode 0: one bt_price_exact per request (FIFO).
    Returns (results in request order, latencies in ms, wall seconds)."""
    a = options_array(opts)
    arr = np.ascontiguousarray(np.asarray(arrival_s, dtype=np.float64))
    out = np.zeros(len(a), dtype=RESULT_DTYPE)
    lat = np.zeros(len(a))
    wall = C.c_double()
    c = _cfg(**cfg)
    _check(lib().bt_serve_replay(ctx, C.byref(c), a.ctypes.data, arr.ctypes.data, len(a), mode, out.ctypes.data,
                                 lat.ctypes.data, C.byref(wall)))
    return out, lat, wall.value


BT_NOALLOC_SCRATCH_BYTES = 8 << 20
BT_NOALLOC_MAX_OPTIONS = 64


def bt_price_exact_noalloc(opts, prec=BT_PREC_FP32_COMP, stream=None) -> np.ndarray:
    """Exhaustive pricing without any device allocation: for callers that
    cannot allocate device memory while they run (see the C header). Uses a
    fixed library-owned device array; needs no context."""
    a = options_array(opts)
    out = np.zeros(len(a), dtype=RESULT_DTYPE)
    _check(lib().bt_price_exact_noalloc(a.ctypes.data, len(a), prec, out.ctypes.data, _stream(stream)))
    return out


class Context:
    """Owns a bt_ctx; a convenience over the same-name functions."""

    def __init__(self, device: int = 0, device_budget_bytes: int = 0):
        self.h = bt_create(device, device_budget_bytes)

    def close(self):
        if self.h:
            bt_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def price_exact(self, opts, prec=BT_PREC_FP32_COMP, stream=None):
        return bt_price_exact(self.h, opts, prec, stream)
