"""GPU parity of the time-varying tree pass (eq. f13 with per-step u_t, d_t,
p_t) against the oracle's path walk. Tolerances: FP64 1e-12; FP32_COMP the
arithmetic-Asian bands of test_exact_gpu (every payoff here is one rounded
FP32 value per path, weighted by its suffix weight)."""
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


def test_fp32_against_fp64_at_large_n(bt, ctx):
    """N = 30 and 34 non-recombining trees (beyond the oracle's reach in a
    test): the FP32 pass against the FP64 pass, which the oracle pins below."""
    for N in (30, 34):
        opts = [W.opt(N, 100.0, K, 0.03, 0.2, 1.0, pay) for pay in range(8) for K in (95.0, 110.0)]
        steps = [W.step_factors(500 + N + i, N, 0.01, 0.05) for i in range(len(opts))]
        v32 = bt.bt_price_exact_steps(ctx.h, opts, steps, 1)["value"]
        v64 = bt.bt_price_exact_steps(ctx.h, opts, steps, 0)["value"]
        _check(v32, v64, opts, 1, "N=%d fp32 vs fp64" % N)


def test_batch_matches_singles_bit_for_bit(bt, ctx):
    opts = [W.opt(N, 100.0, 100.0, 0.05, 0.2, 1.0, pay) for N, pay in ((8, 2), (23, 6), (15, 4), (24, 1))]
    steps = [W.step_factors(40 + i, o["N"]) for i, o in enumerate(opts)]
    batch = bt.bt_price_exact_steps(ctx.h, opts, steps, 1)["value"]
    for i, o in enumerate(opts):
        assert bt.bt_price_exact_steps(ctx.h, [o], [steps[i]], 1)["value"][0] == batch[i]


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
    # ... while the FP32 pass (2^28 paths and more) refuses p_t < 0.004
    o28 = dict(o, N=28)
    st28 = W.step_factors(2, 28)
    st28[5, 2] = 0.001
    with pytest.raises(bt.BtError) as e:
        bt.bt_price_exact_steps(ctx.h, [o28], [st28], 1)
    assert e.value.status == bt.BT_EUNSUPPORTED
    with pytest.raises(ValueError):
        bt.bt_price_exact_steps(ctx.h, [o], [good[:5]], 0)
