"""Payoff plug-ins compiled at run time (bt_plugin_compile): re-stated
built-in payoffs against the built-in FP64 passes, and payoffs the library
does not have (an up-and-out barrier call, a pattern count of the bits)
against an independent numpy brute force."""
import math

import numpy as np
import pytest

from paper_1701_03512_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ARITH_CALL = r"""
struct Payoff {
    struct state { double sum; };
    __device__ static state start(double, const double *) { return {0.0}; }
    __device__ static state step(const state &s, double S, int, int, const double *) { return {s.sum + S}; }
    __device__ static double value(const state &s, int N, const double *p) {
        return fmax(s.sum / N - p[0], 0.0);
    }
};
"""

LOOKBACK_PUT = r"""
struct Payoff {
    struct state { double mn; };
    __device__ static state start(double, const double *) { return {1e300}; }
    __device__ static state step(const state &s, double S, int, int, const double *) { return {fmin(s.mn, S)}; }
    __device__ static double value(const state &s, int, const double *p) { return fmax(p[0] - s.mn, 0.0); }
};
"""

BARRIER_CALL = r"""
// up-and-out call: pays max(S_N - K, 0) unless some S_t >= B (param[1])
struct Payoff {
    struct state { double S; int out; };
    __device__ static state start(double S0, const double *) { return {S0, 0}; }
    __device__ static state step(const state &s, double S, int, int, const double *p) {
        return {S, s.out || S >= p[1]};
    }
    __device__ static double value(const state &s, int, const double *p) {
        return s.out ? 0.0 : fmax(s.S - p[0], 0.0);
    }
};
"""

UP_RUNS = r"""
// number of maximal runs of at least three consecutive up moves (a function
// of the bits alone, the general V(x) of the expected value)
struct Payoff {
    struct state { int run; int count; };
    __device__ static state start(double, const double *) { return {0, 0}; }
    __device__ static state step(const state &s, double, int, int x, const double *) {
        if (x) return {s.run + 1, s.count + (s.run + 1 == 3)};
        return {0, s.count};
    }
    __device__ static double value(const state &s, int, const double *) { return (double)s.count; }
};
"""


@pytest.fixture(scope="module")
def bt():
    from paper_1701_03512_gb300 import build as b
    b.build()
    from paper_1701_03512_gb300 import btree
    return btree


@pytest.fixture(scope="module")
def ctx(bt):
    c = bt.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def plugins(bt, ctx):
    made = {name: bt.bt_plugin_compile(ctx.h, src)[0] for name, src in
            (("arith", ARITH_CALL), ("lookput", LOOKBACK_PUT), ("barrier", BARRIER_CALL), ("runs", UP_RUNS))}
    yield made
    for h in made.values():
        bt.bt_plugin_destroy(h)


def _brute(o, steps, V):
    N = o["N"]
    b = np.arange(1 << N, dtype=np.int64)
    x = ((b[:, None] >> (N - 1 - np.arange(N))[None, :]) & 1).astype(bool)
    S = o["S0"] * np.cumprod(np.where(x, steps[:, 0], steps[:, 1]), axis=1)
    w = np.prod(np.where(x, steps[:, 2], 1.0 - steps[:, 2]), axis=1)
    return math.exp(-o["rate"] * o["T"]) * math.fsum(w * V(S, x))


def test_restated_builtins_match_the_builtin_passes(bt, ctx, plugins):
    for N in (9, 20, 26):
        opts = [W.opt(N, 100.0, 97.0, 0.05, 0.25, 1.0, W.ASIAN_ARITH_CALL),
                W.opt(N, 100.0, 104.0, 0.05, 0.25, 1.0, W.LOOKBACK_FIXED_PUT, W.TREE_SEYDEL)]
        ref = ctx.price_exact(opts, 0)["value"]
        a = bt.bt_price_exact_plugin(ctx.h, plugins["arith"], opts[:1])[0]
        b = bt.bt_price_exact_plugin(ctx.h, plugins["lookput"], opts[1:])[0]
        assert abs(a["value"] - ref[0]) <= 1e-12 * ref[0] and a["paths"] == 2 ** N
        assert abs(b["value"] - ref[1]) <= 1e-12 * ref[1]


def test_time_varying_steps_match_the_steps_pass(bt, ctx, plugins):
    o = W.opt(24, 100.0, 99.0, 0.03, 0.2, 1.0, W.ASIAN_ARITH_CALL)
    steps = W.step_factors(77, 24)
    ref = bt.bt_price_exact_steps(ctx.h, [o], [steps], 0)["value"][0]
    got = bt.bt_price_exact_plugin(ctx.h, plugins["arith"], [o], steps=[steps])["value"][0]
    assert abs(got - ref) <= 1e-12 * ref


def test_barrier_call_against_brute_force(bt, ctx, plugins):
    for N, B in ((12, 120.0), (16, 112.0)):
        o = W.opt(N, 100.0, 98.0, 0.04, 0.3, 1.0, W.EURO_CALL)
        steps = W.step_factors(5 + N, N)
        ref = _brute(o, steps, lambda S, x: np.where(S.max(axis=1) >= B, 0.0, np.maximum(S[:, -1] - 98.0, 0.0)))
        got = bt.bt_price_exact_plugin(ctx.h, plugins["barrier"], [o], steps=[steps], params=[[98.0, B]])
        assert abs(got["value"][0] - ref) <= 1e-12 * abs(ref) + 1e-14


def test_bit_pattern_functional_against_brute_force(bt, ctx, plugins):
    def runs(S, x):
        xi = x.astype(np.int64)
        c = np.zeros(len(x))
        run = np.zeros(len(x), dtype=np.int64)
        for t in range(x.shape[1]):
            run = np.where(xi[:, t] == 1, run + 1, 0)
            c += run == 3
        return c
    o = W.opt(15, 100.0, 100.0, 0.0, 0.2, 1.0, W.EURO_CALL)
    steps = W.step_factors(8, 15)
    ref = _brute(o, steps, runs)
    got = bt.bt_price_exact_plugin(ctx.h, plugins["runs"], [o], steps=[steps])["value"][0]
    assert abs(got - ref) <= 1e-13 * ref


def test_compile_error_reports_the_log(bt, ctx):
    with pytest.raises(bt.BtError) as e:
        bt.bt_plugin_compile(ctx.h, "struct Payoff { this is not C++ };")
    assert e.value.status == bt.BT_EINVAL and "error" in str(e.value)
