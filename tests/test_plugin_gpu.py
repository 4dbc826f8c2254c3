"""Payoff plug-ins compiled at run time (bt_plugin_compile), against the
oracle: re-stated built-in payoffs against its exact values on lattice trees
and its path walk on time-varying trees, and payoffs the library does not
have (an up-and-out barrier call, a pattern count of the bits) against its
enumeration of the same payoff written as a function of the whole path
(eq. expval)."""
import os

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


def test_restated_builtins_against_the_oracle(bt, ctx, plugins, oracle):
    """Plug-ins restating two built-in payoffs on lattice trees, against the
    oracle's exact values (meet in the middle / the lookback DP above N = 16,
    its enumeration below)."""
    for N in (9, 20, 26):
        opts = [W.opt(N, 100.0, 97.0, 0.05, 0.25, 1.0, W.ASIAN_ARITH_CALL),
                W.opt(N, 100.0, 104.0, 0.05, 0.25, 1.0, W.LOOKBACK_FIXED_PUT, W.TREE_SEYDEL)]
        ref = [oracle.exact(o) for o in opts]
        a = bt.bt_price_exact_plugin(ctx.h, plugins["arith"], opts[:1])[0]
        b = bt.bt_price_exact_plugin(ctx.h, plugins["lookput"], opts[1:])[0]
        assert abs(a["value"] - ref[0]) <= 1e-12 * ref[0] and a["paths"] == 2 ** N, (N, a["value"], ref[0])
        assert abs(b["value"] - ref[1]) <= 1e-12 * ref[1], (N, b["value"], ref[1])


def test_restated_builtin_on_a_time_varying_tree_against_the_oracle(bt, ctx, plugins, oracle):
    for N in (16, 24):
        o = W.opt(N, 100.0, 99.0, 0.03, 0.2, 1.0, W.ASIAN_ARITH_CALL)
        steps = W.step_factors(77 + N, N)
        ref = oracle.steps_price(o, steps, os.cpu_count() or 8)
        got = bt.bt_price_exact_plugin(ctx.h, plugins["arith"], [o], steps=[steps])["value"][0]
        assert abs(got - ref) <= 1e-12 * ref, (N, got, ref)


def test_barrier_call_against_the_oracle(bt, ctx, plugins, oracle):
    """A payoff outside the built-ins, against the oracle's enumeration of
    the same payoff written as a function of the whole path."""
    for N, B in ((12, 120.0), (16, 112.0), (20, 115.0)):
        o = W.opt(N, 100.0, 98.0, 0.04, 0.3, 1.0, W.EURO_CALL)
        steps = W.step_factors(5 + N, N)
        ref = oracle.functional_price(
            o, oracle.steps_as_moves(steps), 2,
            lambda S, x: np.where(S.max(axis=1) >= B, 0.0, np.maximum(S[:, -1] - 98.0, 0.0)))
        got = bt.bt_price_exact_plugin(ctx.h, plugins["barrier"], [o], steps=[steps], params=[[98.0, B]])
        assert abs(got["value"][0] - ref) <= 1e-12 * abs(ref) + 1e-14, (N, got["value"][0], ref)


def test_bit_pattern_functional_against_the_oracle(bt, ctx, plugins, oracle):
    def runs(S, x):
        c = np.zeros(len(x))
        run = np.zeros(len(x), dtype=np.int64)
        for t in range(x.shape[1]):
            run = np.where(x[:, t] == 1, run + 1, 0)
            c += run == 3
        return c
    for N in (15, 20):
        o = W.opt(N, 100.0, 100.0, 0.0, 0.2, 1.0, W.EURO_CALL)
        steps = W.step_factors(8 + N, N)
        ref = oracle.functional_price(o, oracle.steps_as_moves(steps), 2, runs)
        got = bt.bt_price_exact_plugin(ctx.h, plugins["runs"], [o], steps=[steps])["value"][0]
        assert abs(got - ref) <= 1e-13 * ref, (N, got, ref)


def test_compile_error_reports_the_log(bt, ctx):
    with pytest.raises(bt.BtError) as e:
        bt.bt_plugin_compile(ctx.h, "struct Payoff { this is not C++ };")
    assert e.value.status == bt.BT_EINVAL and "error" in str(e.value)
