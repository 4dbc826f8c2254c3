"""ctypes front end of the CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline use this module. It compiles ``oracle.c`` with gcc on first use
(``build()``) and exposes thin wrappers; all arithmetic lives in the C file.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain FP64, no contraction, no -march)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _SO + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, src, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class Model(C.Structure):
    _fields_ = [("N", C.c_int32), ("payoff", C.c_int32), ("S0", C.c_double), ("K", C.c_double),
                ("u", C.c_double), ("d", C.c_double), ("p", C.c_double), ("disc", C.c_double)]


class StepsModel(C.Structure):
    _fields_ = [("N", C.c_int32), ("payoff", C.c_int32), ("S0", C.c_double), ("K", C.c_double),
                ("disc", C.c_double), ("u", C.POINTER(C.c_double)), ("d", C.POINTER(C.c_double)),
                ("p", C.POINTER(C.c_double))]


class BranchModel(C.Structure):
    _fields_ = [("N", C.c_int32), ("b", C.c_int32), ("payoff", C.c_int32), ("pad", C.c_int32),
                ("S0", C.c_double), ("K", C.c_double), ("disc", C.c_double),
                ("f", C.POINTER(C.c_double)), ("q", C.POINTER(C.c_double))]


# fn(user, count, N, S, x, v) of orc_functional_price
PAYOFF_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int32),
                        C.POINTER(C.c_double))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            d, i32, u64, i64 = C.c_double, C.c_int32, C.c_uint64, C.c_int64
            pd = C.POINTER(C.c_double)
            pm = C.POINTER(Model)
            L.orc_tree.argtypes = [C.c_int, C.c_int, d, d, d, pd, pd, pd]
            L.orc_model_make.argtypes = [C.c_int, C.c_int, C.c_int, d, d, d, d, d, d, d, d, pm]
            L.orc_path_payoff.argtypes = [pm, u64]; L.orc_path_payoff.restype = d
            L.orc_path_prob.argtypes = [pm, u64]; L.orc_path_prob.restype = d
            L.orc_sum_range.argtypes = [pm, u64, u64, pd, pd]
            L.orc_price_exhaustive.argtypes = [pm, C.c_int]; L.orc_price_exhaustive.restype = d
            L.orc_sum_range_mt.argtypes = [pm, u64, u64, C.c_int]; L.orc_sum_range_mt.restype = d
            L.orc_leaf_prob_sums.argtypes = [pm, pd]
            for f in ("orc_price_european_closed", "orc_price_european_backward",
                      "orc_price_geometric_dp", "orc_price_lookback_dp"):
                getattr(L, f).argtypes = [pm]; getattr(L, f).restype = d
            L.orc_price_asian_mitm.argtypes = [pm, C.c_int]; L.orc_price_asian_mitm.restype = d
            L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                            C.POINTER(C.c_uint32)]
            L.orc_bernoulli_threshold.argtypes = [d]; L.orc_bernoulli_threshold.restype = u64
            L.orc_mc.argtypes = [pm, C.c_int, i64, u64, C.c_uint32, C.c_int, pd, pd, pd, pd, pd]
            L.orc_stratum_moments.argtypes = [pm, C.c_int, pd, pd, pd]
            L.orc_mc_stratum.argtypes = [pm, C.c_int, u64, i64, u64, C.c_uint32, pd, pd, pd]
            L.orc_greeks_crr.argtypes = [C.c_int, C.c_int, d, d, d, d, d, pd]
            L.orc_greeks_crr.restype = d
            ps = C.POINTER(StepsModel)
            L.orc_steps_path_payoff.argtypes = [ps, u64]; L.orc_steps_path_payoff.restype = d
            L.orc_steps_path_prob.argtypes = [ps, u64]; L.orc_steps_path_prob.restype = d
            L.orc_steps_sum_range.argtypes = [ps, u64, u64, pd, pd]
            L.orc_steps_price.argtypes = [ps, C.c_int]; L.orc_steps_price.restype = d
            pb = C.POINTER(BranchModel)
            L.orc_branch_path_payoff.argtypes = [pb, u64]; L.orc_branch_path_payoff.restype = d
            L.orc_branch_path_prob.argtypes = [pb, u64]; L.orc_branch_path_prob.restype = d
            L.orc_branch_price.argtypes = [pb, C.c_int]; L.orc_branch_price.restype = d
            L.orc_branch_european_backward.argtypes = [pb]; L.orc_branch_european_backward.restype = d
            pi32 = C.POINTER(C.c_int32)
            L.orc_steps_price_multi.argtypes = [ps, C.c_int, pi32, pd, C.c_int, pd]
            L.orc_branch_price_multi.argtypes = [pb, C.c_int, pi32, pd, C.c_int, pd]
            L.orc_functional_price.argtypes = [pb, PAYOFF_FN, C.c_void_p]
            L.orc_functional_price.restype = d
            _lib = L
    return _lib


def tree(kind, N, sigma, rate, T):
    u, d, p = C.c_double(), C.c_double(), C.c_double()
    rc = lib().orc_tree(kind, N, sigma, rate, T, C.byref(u), C.byref(d), C.byref(p))
    if rc != 0:
        raise ValueError("invalid tree parameters")
    return u.value, d.value, p.value


def model(o: dict) -> Model:
    """Model from an option dict (see workloads.opt)."""
    m = Model()
    rc = lib().orc_model_make(o["N"], o["tree_kind"], o["payoff"], o["S0"], o["K"], o["rate"],
                              o["sigma"], o["T"], o.get("u", 0.0), o.get("d", 0.0), o.get("p", 0.0),
                              C.byref(m))
    if rc != 0:
        raise ValueError("invalid option for the oracle: %r" % (o,))
    return m


def price_exhaustive(o: dict, nthreads: int = 1) -> float:
    return lib().orc_price_exhaustive(C.byref(model(o)), nthreads)


def sum_range(o: dict, lo: int, hi: int):
    s, c = C.c_double(), C.c_double()
    lib().orc_sum_range(C.byref(model(o)), lo, hi, C.byref(s), C.byref(c))
    return s.value + c.value


def sum_range_mt(o: dict, lo: int, hi: int, nthreads: int) -> float:
    return lib().orc_sum_range_mt(C.byref(model(o)), lo, hi, nthreads)


def path_payoff(o: dict, b: int) -> float:
    return lib().orc_path_payoff(C.byref(model(o)), b)


def path_prob(o: dict, b: int) -> float:
    return lib().orc_path_prob(C.byref(model(o)), b)


def leaf_prob_sums(o: dict) -> np.ndarray:
    out = np.zeros(o["N"] + 1)
    lib().orc_leaf_prob_sums(C.byref(model(o)), out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def european_closed(o):
    return lib().orc_price_european_closed(C.byref(model(o)))


def european_backward(o):
    return lib().orc_price_european_backward(C.byref(model(o)))


def geometric_dp(o):
    return lib().orc_price_geometric_dp(C.byref(model(o)))


def lookback_dp(o):
    return lib().orc_price_lookback_dp(C.byref(model(o)))


def asian_mitm(o, L=None):
    if L is None:
        L = (o["N"] + 1) // 2
    return lib().orc_price_asian_mitm(C.byref(model(o)), L)


def exact(o: dict, nthreads: int = 8) -> float:
    """Exact value by the fastest exact oracle routine for the payoff."""
    pay = o["payoff"]
    if pay in (0, 1):
        return european_closed(o)
    if pay in (2, 3):
        return asian_mitm(o) if o["N"] > 16 else price_exhaustive(o, nthreads)
    if pay in (4, 5):
        return geometric_dp(o)
    return lookback_dp(o)


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xffffffff for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xffffffff for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def bernoulli_threshold(p: float) -> int:
    return int(lib().orc_bernoulli_threshold(p))


def mc(o: dict, mb: int, Rm: int, seed: int, stream: int = 0, shared: bool = False,
       with_strata: bool = False):
    """Returns (theta, var) undiscounted, or with per-stratum arrays."""
    th, var = C.c_double(), C.c_double()
    M = 1 << mb
    pd = C.POINTER(C.c_double)
    if with_strata:
        mean, sv, pr = np.zeros(M), np.zeros(M), np.zeros(M)
        args = [mean.ctypes.data_as(pd), sv.ctypes.data_as(pd), pr.ctypes.data_as(pd)]
    else:
        args = [None, None, None]
    lib().orc_mc(C.byref(model(o)), mb, Rm, seed, stream, 1 if shared else 0, C.byref(th),
                 C.byref(var), *args)
    if with_strata:
        return th.value, var.value, mean, sv, pr
    return th.value, var.value


def stratum_moments(o: dict, mb: int):
    M = 1 << mb
    mean, var, prob = np.zeros(M), np.zeros(M), np.zeros(M)
    pd = C.POINTER(C.c_double)
    lib().orc_stratum_moments(C.byref(model(o)), mb, mean.ctypes.data_as(pd), var.ctypes.data_as(pd),
                              prob.ctypes.data_as(pd))
    return mean, var, prob


def greeks_crr(o: dict):
    """(value, [dS0, dsigma, drate, dK]) by pathwise enumeration (CRR only)."""
    g = np.zeros(4)
    v = lib().orc_greeks_crr(o["N"], o["payoff"], o["S0"], o["K"], o["rate"], o["sigma"], o["T"],
                             g.ctypes.data_as(C.POINTER(C.c_double)))
    return v, g


def discount(o: dict) -> float:
    return model(o).disc


# ---------------------------------------------------------------------------
# Time-varying trees (eq. f13 with per-step u_t, d_t, p_t)
# ---------------------------------------------------------------------------
def steps_model(o: dict, steps):
    """(model, keep-alive arrays) for an option dict and steps[N][3] = (u_t, d_t, p_t)."""
    st = np.ascontiguousarray(np.asarray(steps, dtype=np.float64).reshape(o["N"], 3))
    u, d, p = (np.ascontiguousarray(st[:, k]) for k in range(3))
    pd = C.POINTER(C.c_double)
    m = StepsModel(o["N"], o["payoff"], o["S0"], o["K"], math.exp(-o["rate"] * o["T"]),
                   u.ctypes.data_as(pd), d.ctypes.data_as(pd), p.ctypes.data_as(pd))
    return m, (u, d, p)


def steps_price(o: dict, steps, nthreads: int = 8) -> float:
    m, keep = steps_model(o, steps)
    return lib().orc_steps_price(C.byref(m), nthreads)


def steps_sum_range(o: dict, steps, lo: int, hi: int) -> float:
    m, keep = steps_model(o, steps)
    s, c = C.c_double(), C.c_double()
    lib().orc_steps_sum_range(C.byref(m), lo, hi, C.byref(s), C.byref(c))
    return s.value + c.value


def steps_path_payoff(o: dict, steps, b: int) -> float:
    m, keep = steps_model(o, steps)
    return lib().orc_steps_path_payoff(C.byref(m), b)


def steps_path_prob(o: dict, steps, b: int) -> float:
    m, keep = steps_model(o, steps)
    return lib().orc_steps_path_prob(C.byref(m), b)


# ---------------------------------------------------------------------------
# b-ary trees: moves[N][2b] = (factor of digit 0..b-1, probability of digit 0..b-1)
# ---------------------------------------------------------------------------
def branch_model(o: dict, moves, b: int):
    mv = np.asarray(moves, dtype=np.float64).reshape(o["N"], 2 * b)
    f = np.ascontiguousarray(mv[:, :b])
    q = np.ascontiguousarray(mv[:, b:])
    pd = C.POINTER(C.c_double)
    m = BranchModel(o["N"], b, o["payoff"], 0, o["S0"], o["K"], math.exp(-o["rate"] * o["T"]),
                    f.ctypes.data_as(pd), q.ctypes.data_as(pd))
    return m, (f, q)


def branch_price(o: dict, moves, b: int, nthreads: int = 8) -> float:
    m, keep = branch_model(o, moves, b)
    return lib().orc_branch_price(C.byref(m), nthreads)


def branch_european_backward(o: dict, moves, b: int) -> float:
    m, keep = branch_model(o, moves, b)
    return lib().orc_branch_european_backward(C.byref(m))


def branch_path_prob(o: dict, moves, b: int, idx: int) -> float:
    m, keep = branch_model(o, moves, b)
    return lib().orc_branch_path_prob(C.byref(m), idx)


def mc_stratum(o: dict, mb: int, z: int, Rm: int, seed: int, stream: int = 0):
    """(mean, unbiased variance, P(D_z)) of one stratum, the same draws as mc()."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    lib().orc_mc_stratum(C.byref(model(o)), mb, z, Rm, seed, stream, C.byref(a), C.byref(b), C.byref(c))
    return a.value, b.value, c.value


def _pay_strikes(pays_ks):
    pays = np.ascontiguousarray([int(p) for p, _ in pays_ks], dtype=np.int32)
    ks = np.ascontiguousarray([float(k) for _, k in pays_ks], dtype=np.float64)
    return pays, ks


def steps_price_multi(o: dict, steps, pays_ks, nthreads: int = 8) -> np.ndarray:
    """Discounted values of every (payoff, K) in pays_ks on one time-varying
    tree (o's S0, rate, T, N), each path walked once for all of them."""
    m, keep = steps_model(o, steps)
    pays, ks = _pay_strikes(pays_ks)
    out = np.zeros(len(pays))
    lib().orc_steps_price_multi(C.byref(m), len(pays), pays.ctypes.data_as(C.POINTER(C.c_int32)),
                                ks.ctypes.data_as(C.POINTER(C.c_double)), nthreads,
                                out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def branch_price_multi(o: dict, moves, b: int, pays_ks, nthreads: int = 8) -> np.ndarray:
    m, keep = branch_model(o, moves, b)
    pays, ks = _pay_strikes(pays_ks)
    out = np.zeros(len(pays))
    lib().orc_branch_price_multi(C.byref(m), len(pays), pays.ctypes.data_as(C.POINTER(C.c_int32)),
                                 ks.ctypes.data_as(C.POINTER(C.c_double)), nthreads,
                                 out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def functional_price(o: dict, moves, b: int, V) -> float:
    """eq. expval for a payoff V given as a Python function of whole paths:
    V(S, x) receives S[count, N] (S_1..S_N) and x[count, N] (the digits) of a
    block of consecutive paths and returns their payoffs. moves as for
    branch_price (for a time-varying binomial tree: (d_t, u_t, 1-p_t, p_t))."""
    m, keep = branch_model(o, moves, b)
    err = []

    def cb(user, count, N, S, x, v):
        try:
            s = np.ctypeslib.as_array(S, shape=(count, N))
            xs = np.ctypeslib.as_array(x, shape=(count, N))
            np.ctypeslib.as_array(v, shape=(count,))[:] = np.asarray(V(s, xs), dtype=np.float64)
        except Exception as e:  # surfaced after the call
            err.append(e)
            np.ctypeslib.as_array(v, shape=(count,))[:] = np.nan

    fn = PAYOFF_FN(cb)
    r = lib().orc_functional_price(C.byref(m), fn, None)
    if err:
        raise err[0]
    return r


def steps_as_moves(steps) -> np.ndarray:
    """(u_t, d_t, p_t) rows as binomial moves (d_t, u_t, 1 - p_t, p_t): digit 1 = up."""
    st = np.asarray(steps, dtype=np.float64)
    return np.stack([st[:, 1], st[:, 0], 1.0 - st[:, 2], st[:, 2]], axis=1)
