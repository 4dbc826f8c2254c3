"""Trees with b branches per node (the end of Section 3) on the GPU: the
generic pass with the built-in payoffs against the oracle's b-ary
enumeration, a recombining trinomial lattice against backward induction,
b = 2 against the built-in binomial pass, a plug-in on a trinomial tree
against the oracle's enumeration of a payoff given as a path function, and
the affine pass against the oracle at every size it runs (the FP32 pass from
2^28 paths: 3^18 and 4^14)."""
import math
import os

import numpy as np
import pytest

from paper_1701_03512_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("b,N", [(3, 1), (3, 6), (3, 10), (4, 6), (5, 5), (6, 4), (7, 4), (8, 4)])
def test_builtin_payoffs_against_the_oracle(bt, ctx, oracle, b, N):
    opts = [W.opt(N, 100.0, K, 0.03, 0.2, 1.0, pay) for pay in range(8) for K in (95.0, 103.0)]
    moves = [W.branch_moves(7 * N + i + b, N, b) for i in range(len(opts))]
    got = bt.bt_price_exact_branching(ctx.h, opts, b, moves)
    for o, m, g in zip(opts, moves, got):
        ref = oracle.branch_price(o, m, b, 8)
        assert abs(g["value"] - ref) <= 1e-12 * abs(ref) + 1e-13, (o, g["value"], ref)
        assert g["paths"] == b ** N


def test_recombining_trinomial_european_against_backward_induction(bt, ctx, oracle):
    N = 15
    u = math.exp(0.25 * math.sqrt(3 / 15))
    moves = np.tile([1 / u, 1.0, u, 0.18, 0.64, 0.18], (N, 1))
    for pay in (W.EURO_CALL, W.EURO_PUT):
        o = W.opt(N, 100.0, 100.0, 0.0, 0.25, 1.0, pay)
        got = bt.bt_price_exact_branching(ctx.h, [o], 3, [moves])["value"][0]
        assert abs(got - oracle.branch_european_backward(o, moves, 3)) <= 1e-12 * got


def test_two_branches_match_the_binomial_pass(bt, ctx):
    N = 22
    opts = [W.opt(N, 100.0, 101.0, 0.05, 0.3, 1.0, pay) for pay in range(8)]
    u, d, p = bt.bt_tree_params(opts[0])
    moves = [np.tile([d, u, 1 - p, p], (N, 1))] * len(opts)
    got = bt.bt_price_exact_branching(ctx.h, opts, 2, moves)["value"]
    ref = ctx.price_exact(opts, 0)["value"]
    assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref) + 1e-13)


def test_plugin_on_a_trinomial_tree(bt, ctx, oracle):
    src = r"""
    struct Payoff {   // up-and-out call, barrier param[1]
        struct state { double S; int out; };
        __device__ static state start(double S0, const double *) { return {S0, 0}; }
        __device__ static state step(const state &s, double S, int, int, const double *p) {
            return {S, s.out || S >= p[1]};
        }
        __device__ static double value(const state &s, int, const double *p) {
            return s.out ? 0.0 : fmax(s.S - p[0], 0.0);
        }
    };"""
    h, _ = bt.bt_plugin_compile(ctx.h, src)
    try:
        N, b = 9, 3
        moves = W.branch_moves(3, N, b)
        o = W.opt(N, 100.0, 97.0, 0.02, 0.2, 1.0, W.EURO_CALL)
        got = bt.bt_price_exact_branching(ctx.h, [o], b, [moves], plugin=h, params=[[97.0, 115.0]])["value"][0]
        ref = oracle.functional_price(
            o, moves, b, lambda S, x: np.where(S.max(axis=1) >= 115.0, 0.0, np.maximum(S[:, -1] - 97.0, 0.0)))
        assert abs(got - ref) <= 1e-12 * ref
    finally:
        bt.bt_plugin_destroy(h)


def test_invalid_moves(bt, ctx):
    o = W.opt(4, 100.0, 100.0, 0.0, 0.2, 1.0, W.EURO_CALL)
    mv = W.branch_moves(1, 4, 3)
    bad = mv.copy()
    bad[2, 4] += 0.01     # probabilities no longer sum to 1
    with pytest.raises(bt.BtError) as e:
        bt.bt_price_exact_branching(ctx.h, [o], 3, [bad])
    assert e.value.status == bt.BT_EINVAL
    with pytest.raises(bt.BtError) as e:
        bt.bt_price_exact_branching(ctx.h, [dict(o, N=31)], 3, [W.branch_moves(1, 31, 3)])
    assert e.value.status == bt.BT_EUNSUPPORTED


def _tol(prec, paths):
    """FP64 1e-12; FP32_COMP 1e-9: from 2^28 paths the FP32 pass, whose
    per-path roundings average out over that many paths; smaller trees are
    priced by the FP64 pass under FP32_COMP."""
    return 1e-12 if prec == 0 else 1e-9


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("b,N", [(3, 1), (3, 9), (3, 13), (4, 8), (5, 7), (6, 4), (7, 4), (8, 5)])
def test_affine_moves_pass_against_the_oracle(bt, ctx, oracle, prec, b, N):
    """bt_price_exact_moves (the prefix/suffix tables and per-suffix weights of
    the time-varying pass, in base b) on non-recombining trees."""
    opts = [W.opt(N, 100.0, K, 0.03, 0.2, 1.0, pay) for pay in range(8) for K in (96.0, 104.0)]
    moves = [W.branch_moves(31 * N + i + b, N, b) for i in range(len(opts))]
    got = bt.bt_price_exact_moves(ctx.h, opts, b, moves, prec)
    for o, m, g in zip(opts, moves, got):
        ref = oracle.branch_price(o, m, b, 8)
        assert abs(g["value"] - ref) <= _tol(prec, b ** N) * abs(ref) + 1e-12 * o["S0"], (prec, o, g["value"], ref)
        assert abs(g["value"] - ref) <= g["err_est"] + 1e-12 * o["S0"], (prec, o, g["err_est"])   # stated error
        assert g["paths"] == b ** N


def test_affine_moves_probability_floor(bt, ctx, oracle):
    """From 2^28 paths (and 2^27 effective paths) FP32_COMP runs the FP32
    pass, which refuses a branch probability in (0, 0.004) (its weights would
    leave the FP32 pair range); FP64 takes it. A smaller tree runs the FP64
    pass under FP32_COMP too, so there the rare probability is taken. A zero
    probability (a branch that never happens) is taken by the FP32 pass as
    well."""
    o = W.opt(6, 100.0, 100.0, 0.02, 0.2, 1.0, W.ASIAN_ARITH_CALL)
    rare = W.branch_moves(5, 6, 3)
    rare[3, 3:] = [0.001, 0.5, 0.499]
    r = bt.bt_price_exact_moves(ctx.h, [o], 3, [rare], bt.BT_PREC_FP32_COMP)[0]
    assert abs(r["value"] - oracle.branch_price(o, rare, 3, 8)) <= 1e-12 * abs(r["value"])
    assert r["err_est"] == pytest.approx(1e-12 * abs(r["value"]))      # priced by the FP64 pass
    ob = W.opt(18, 100.0, 100.0, 0.02, 0.2, 1.0, W.ASIAN_ARITH_CALL)   # 3^18 = 3.9e8 paths
    mvb = W.branch_moves(6, 18, 3, conc=50.0)                          # near 1/3: 2^28 effective paths
    rareb = mvb.copy()
    rareb[9, 3:] = [0.001, 0.5, 0.499]
    with pytest.raises(bt.BtError) as e:
        bt.bt_price_exact_moves(ctx.h, [ob], 3, [rareb], bt.BT_PREC_FP32_COMP)
    assert e.value.status == bt.BT_EUNSUPPORTED
    assert bt.bt_price_exact_moves(ctx.h, [ob], 3, [rareb], bt.BT_PREC_FP64)[0]["value"] > 0.0
    never = mvb.copy()
    never[9, 3:] = [0.0, 0.5, 0.5]
    v64 = bt.bt_price_exact_moves(ctx.h, [ob], 3, [never], bt.BT_PREC_FP64)[0]["value"]
    v32 = bt.bt_price_exact_moves(ctx.h, [ob], 3, [never], bt.BT_PREC_FP32_COMP)[0]["value"]
    assert abs(v32 - v64) <= 1e-9 * abs(v64) + 1e-12 * ob["S0"], (v32, v64)


@pytest.mark.parametrize("b,N", [(3, 18), (4, 14), (6, 11)])   # 3.9e8, 2.7e8, 3.6e8 paths
def test_affine_moves_fp32_pass_against_the_oracle_at_full_size(bt, ctx, oracle, b, N):
    """From 2^28 paths FP32_COMP runs the FP32 pass: every payoff at two
    strikes on one non-recombining b-ary tree (call and put of one field
    adjacent, sharing a pass) against the oracle's enumeration of all b^N
    paths, at the 1e-9 contract and within the stated error. The senary
    tree fills the suffix table nearly to its 2^13 entries (6^5 = 7776)."""
    opts = [W.opt(N, 100.0, K, 0.03, 0.2, 1.0, pay) for K in (95.0, 105.0) for pay in range(8)]
    mv = W.branch_moves(700 + 10 * b, N, b, 0.01, 0.05, 50.0)
    assert not np.any((mv[:, b:] > 0) & (mv[:, b:] < 0.004))   # above the FP32 pass's probability floor
    assert -np.sum(np.log2(np.sum(mv[:, b:] ** 2, axis=1))) >= 27   # enough effective paths for it
    got = bt.bt_price_exact_moves(ctx.h, opts, b, [mv] * len(opts), 1)
    ref = oracle.branch_price_multi(opts[0], mv, b, [(o["payoff"], o["K"]) for o in opts], os.cpu_count() or 8)
    s0 = np.array([o["S0"] for o in opts])
    err = np.abs(got["value"] - ref)
    assert np.all(err <= 1e-9 * np.abs(ref) + 1e-12 * s0), (b, N, err / np.abs(ref))
    assert np.all(err <= got["err_est"] + 1e-12 * s0)
    assert np.all(got["err_est"] <= 1e-9 * np.abs(got["value"]) * (1 + 1e-12))
    assert np.all(got["paths"] == b ** N)


@pytest.mark.parametrize("b,N", [(3, 20), (8, 10)])   # 3.5e9, 1.1e9 paths
def test_affine_moves_large_trees_fp32_against_fp64(bt, ctx, b, N):
    """A consistency check beyond the oracle's reach in a test: the FP32 pass
    against the FP64 pass of the same library at the 1e-9 contract (the
    oracle pins both at 3^18 and 4^14 paths above)."""
    opts = [W.opt(N, 100.0, K, 0.03, 0.2, 1.0, pay) for K in (95.0, 105.0) for pay in range(8)]
    mv = W.branch_moves(700 + 10 * b, N, b, 0.01, 0.05, 50.0)
    assert not np.any((mv[:, b:] > 0) & (mv[:, b:] < 0.004))
    v32 = bt.bt_price_exact_moves(ctx.h, opts, b, [mv] * len(opts), 1)
    v64 = bt.bt_price_exact_moves(ctx.h, opts, b, [mv] * len(opts), 0)["value"]
    s0 = np.array([o["S0"] for o in opts])
    assert np.all(np.abs(v32["value"] - v64) <= 1e-9 * np.abs(v64) + 1e-12 * s0)


def test_affine_moves_recombining_trinomial_fp64(bt, ctx, oracle):
    N = 16
    u = math.exp(0.25 * math.sqrt(3 / 16))
    moves = np.tile([1 / u, 1.0, u, 0.2, 0.6, 0.2], (N, 1))
    for pay in (W.EURO_CALL, W.EURO_PUT):
        o = W.opt(N, 100.0, 101.0, 0.0, 0.25, 1.0, pay)
        got = bt.bt_price_exact_moves(ctx.h, [o], 3, [moves], 0)["value"][0]
        assert abs(got - oracle.branch_european_backward(o, moves, 3)) <= 1e-12 * got


def test_steps_pass_is_the_binomial_case(bt, ctx):
    N = 21
    opts = [W.opt(N, 100.0, 100.0, 0.02, 0.2, 1.0, pay) for pay in range(8)]
    steps = [W.step_factors(50 + i, N) for i in range(len(opts))]
    moves = [np.stack([s[:, 1], s[:, 0], 1 - s[:, 2], s[:, 2]], axis=1) for s in steps]
    for prec in (0, 1):
        a = bt.bt_price_exact_steps(ctx.h, opts, steps, prec)["value"]
        b = bt.bt_price_exact_moves(ctx.h, opts, 2, moves, prec)["value"]
        assert np.array_equal(a, b)
