"""GPU parity of the time-varying tree pass (eq. f13 with per-step u_t, d_t,
p_t) against the oracle's path walk, at every size the passes run: the FP64
pass, FP32_COMP below 2^28 paths (which runs the FP64 pass), and the FP32
pass from 2^28 paths (N = 28, 30 against the oracle's full enumeration).
Tolerances: FP64 1e-12; FP32_COMP 1e-9 (plus 1e-12 S0 for values near 0)."""
import os

import numpy as np
import pytest

from paper_1701_03512_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def tol(prec, N):
    """FP64 1e-12; FP32_COMP 1e-9 (trees below 2^28 paths are priced by the
    FP64 pass under FP32_COMP, larger ones by the FP32 pass)."""
    return 1e-12 if prec == 0 else 1e-9


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


def _check(got, ref, opts, prec, what):
    for o, g, r in zip(opts, got, ref):
        assert abs(g - r) <= tol(prec, o["N"]) * abs(r) + 1e-12 * o["S0"], (what, o, g, r, (g - r) / r)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("N", [1, 5, 12, 17, 22])
def test_all_payoffs_against_the_oracle(bt, ctx, oracle, prec, N):
    opts = [W.opt(N, 100.0, K, 0.04, 0.2, 1.25, pay) for pay in range(8) for K in (90.0, 104.0)]
    steps = [W.step_factors(100 + N + 7 * i, N) for i in range(len(opts))]
    got = bt.bt_price_exact_steps(ctx.h, opts, steps, prec)
    ref = [oracle.steps_price(o, s, 8) for o, s in zip(opts, steps)]
    _check(got["value"], ref, opts, prec, "N=%d" % N)
    s0 = np.array([o["S0"] for o in opts])
    assert np.all(np.abs(got["value"] - np.array(ref)) <= got["err_est"] + 1e-12 * s0)   # the stated error
    assert np.all(got["paths"] == 2 ** N)


@pytest.mark.parametrize("prec", [0, 1])
def test_constant_factors_match_the_lattice_pass(bt, ctx, prec):
    """Constant CRR factors: the same tree as bt_price_exact prices."""
    opts = [W.opt(26, 100.0, 100.0, 0.05, 0.25, 1.0, pay) for pay in range(8)]
    u, d, p = bt.bt_tree_params(opts[0])
    steps = [np.tile([u, d, p], (26, 1))] * len(opts)
    got = bt.bt_price_exact_steps(ctx.h, opts, steps, prec)["value"]
    ref = ctx.price_exact(opts, 0)["value"]
    _check(got, ref, opts, prec, "constant factors")


def _pairs(N, strikes, S0=100.0, rate=0.03, T=1.0):
    """Every payoff at every strike, call and put of one field adjacent (so
    that a call/put pair of one tree shares a pass)."""
    return [W.opt(N, S0, K, rate, 0.2, T, pay) for K in strikes for pay in range(8)]


@pytest.mark.parametrize("N", [28, 30])
def test_fp32_pass_against_the_oracle_at_full_size(bt, ctx, oracle, N):
    """From 2^28 paths and 2^27 effective paths FP32_COMP prices a
    non-recombining tree with the FP32 pass: all eight payoffs at two strikes
    against the oracle's path walk (one enumeration of the 2^N paths for all
    sixteen), at the 1e-9 contract and within each result's stated error."""
    opts = _pairs(N, (95.0, 110.0))
    steps = W.step_factors(500 + N, N, 0.01, 0.05, 0.45, 0.55)   # p_t near 1/2: 2^27.9 effective paths at N=28
    got = bt.bt_price_exact_steps(ctx.h, opts, [steps] * len(opts), 1)
    ref = oracle.steps_price_multi(opts[0], steps, [(o["payoff"], o["K"]) for o in opts], os.cpu_count() or 8)
    _check(got["value"], ref, opts, 1, "N=%d FP32 pass vs oracle" % N)
    s0 = np.array([o["S0"] for o in opts])
    assert np.all(np.abs(got["value"] - ref) <= got["err_est"] + 1e-12 * s0)
    assert np.all(got["err_est"] <= 1e-9 * np.abs(got["value"]) * (1 + 1e-12))
    assert np.all(got["paths"] == 2 ** N)


def test_fp32_against_fp64_at_n34(bt, ctx):
    """A consistency check beyond the oracle's reach in a test (2^34 paths):
    the FP32 pass against the FP64 pass of the same library; the oracle pins
    both at N = 28 and 30 above."""
    N = 34
    opts = _pairs(N, (95.0, 110.0))
    steps = W.step_factors(500 + N, N, 0.01, 0.05)   # 2^31.5 effective paths
    v32 = bt.bt_price_exact_steps(ctx.h, opts, [steps] * len(opts), 1)["value"]
    v64 = bt.bt_price_exact_steps(ctx.h, opts, [steps] * len(opts), 0)["value"]
    _check(v32, v64, opts, 1, "N=34 fp32 vs fp64")


def test_skewed_and_repeating_trees_take_the_fp64_pass(bt, ctx, oracle):
    """FP32_COMP keeps 1e-9 where per-path FP32 roundings would not average
    out: a tree with fewer than 2^27 effective paths (p_t in [0.6, 0.7] at
    N = 28: about 2^24), and European, geometric and lookback payoffs on a
    recombining tree (equal suffix values), are priced by the FP64 pass --
    their stated error is then 1e-12. The arithmetic Asian on the
    recombining tree keeps the FP32 pass."""
    N = 28
    skew = W.step_factors(61, N, 0.01, 0.05, 0.6, 0.7)
    opts = _pairs(N, (100.0,))
    got = bt.bt_price_exact_steps(ctx.h, opts, [skew] * len(opts), 1)
    ref = oracle.steps_price_multi(opts[0], skew, [(o["payoff"], o["K"]) for o in opts], os.cpu_count() or 8)
    _check(got["value"], ref, opts, 0, "skewed tree")
    assert np.allclose(got["err_est"], 1e-12 * np.abs(got["value"]), rtol=1e-9)
    lat = W.opt(N, 100.0, 100.0, 0.05, 0.25, 1.0, W.EURO_CALL)
    u, d, p = bt.bt_tree_params(lat)
    flat = np.tile([u, d, p], (N, 1))
    opts = [dict(lat, payoff=pay) for pay in range(8)]
    got = bt.bt_price_exact_steps(ctx.h, opts, [flat] * 8, 1)
    ref = [oracle.exact(o) for o in opts]
    _check(got["value"], ref, opts, 1, "recombining tree")
    for o, r in zip(opts, got):
        rel = 1e-9 if o["payoff"] in (W.ASIAN_ARITH_CALL, W.ASIAN_ARITH_PUT) else 1e-12
        assert r["err_est"] == pytest.approx(rel * abs(r["value"]), rel=1e-9), o["payoff"]


def test_batch_matches_singles_bit_for_bit(bt, ctx):
    opts = [W.opt(N, 100.0, 100.0, 0.05, 0.2, 1.0, pay) for N, pay in ((8, 2), (23, 6), (15, 4), (24, 1))]
    steps = [W.step_factors(40 + i, o["N"]) for i, o in enumerate(opts)]
    batch = bt.bt_price_exact_steps(ctx.h, opts, steps, 1)["value"]
    for i, o in enumerate(opts):
        assert bt.bt_price_exact_steps(ctx.h, [o], [steps[i]], 1)["value"][0] == batch[i]


@pytest.mark.parametrize("N,prec", [(30, 1), (22, 0), (22, 1)])
def test_call_put_pair_matches_each_alone(bt, ctx, N, prec):
    """A call followed by the put of the same steps and strike share one pass
    (the affine form computed once); each payoff's arithmetic is that of its
    own pass, so the values are the same bits as pricing each alone. A pair
    whose steps differ is not fused and prices the same way."""
    steps = W.step_factors(70 + N, N, 0.01, 0.05, 0.45, 0.55)
    for field in ((W.EURO_CALL, W.EURO_PUT), (W.ASIAN_ARITH_CALL, W.ASIAN_ARITH_PUT),
                  (W.ASIAN_GEO_PUT, W.ASIAN_GEO_CALL)):
        pair = [W.opt(N, 100.0, 101.0, 0.03, 0.2, 1.0, pay) for pay in field]
        fused = bt.bt_price_exact_steps(ctx.h, pair, [steps, steps], prec)["value"]
        alone = [bt.bt_price_exact_steps(ctx.h, [o], [steps], prec)["value"][0] for o in pair]
        assert fused.tolist() == alone, (N, prec, field)
    other = steps.copy()
    other[3, 0] *= 1.001
    pair = [W.opt(N, 100.0, 101.0, 0.03, 0.2, 1.0, pay) for pay in (W.ASIAN_ARITH_CALL, W.ASIAN_ARITH_PUT)]
    two = bt.bt_price_exact_steps(ctx.h, pair, [steps, other], prec)["value"]
    assert two[0] == bt.bt_price_exact_steps(ctx.h, pair[:1], [steps], prec)["value"][0]
    assert two[1] == bt.bt_price_exact_steps(ctx.h, pair[1:], [other], prec)["value"][0]


def test_invalid_steps(bt, ctx):
    o = W.opt(6, 100.0, 100.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL)
    good = W.step_factors(1, 6)
    for bad, status in (((0, 0), 0.5), ((2, 1), 2.0), ((3, 2), 1.0), ((4, 2), 0.0)):
        st = good.copy()
        st[bad] = status
        with pytest.raises(bt.BtError) as e:
            bt.bt_price_exact_steps(ctx.h, [o], [st], 0)
        assert e.value.status == bt.BT_EINVAL
    st = good.copy()
    st[1, 2] = 0.001
    v64 = bt.bt_price_exact_steps(ctx.h, [o], [st], 0)["value"][0]   # FP64 takes it
    # so does FP32_COMP below 2^28 paths (it runs the FP64 pass there) ...
    assert bt.bt_price_exact_steps(ctx.h, [o], [st], 1)["value"][0] == v64
    # ... while the FP32 pass (2^28 paths and 2^27 effective paths) refuses p_t < 0.004
    o30 = dict(o, N=30)
    st30 = W.step_factors(2, 30, p_lo=0.45, p_hi=0.55)
    st30[5, 2] = 0.001
    with pytest.raises(bt.BtError) as e:
        bt.bt_price_exact_steps(ctx.h, [o30], [st30], 1)
    assert e.value.status == bt.BT_EUNSUPPORTED
    with pytest.raises(ValueError):
        bt.bt_price_exact_steps(ctx.h, [o], [good[:5]], 0)
