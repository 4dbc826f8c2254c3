"""The synthetic input recipe (paper_1701_03512_gb300/workloads.py) against
its stated distributions: the parameter sets of the batched, Greeks and
serving workloads, the serving stream's depths, payoffs and arrivals, and the
per-step moves of the time-varying and b-ary trees. CPU only."""
import numpy as np
import pytest

from paper_1701_03512_gb300 import workloads as W


def test_option_sets_ranges_and_seeding():
    s = W.option_sets(0, 64)
    for key, lo, hi in (("S0", 80, 120), ("K", 80, 120), ("sigma", 0.1, 0.5), ("rate", 0.0, 0.08),
                        ("T", 0.25, 2.0)):
        v = np.asarray(s[key])
        assert v.shape == (64,) and np.all(v >= lo) and np.all(v <= hi), key
    again = W.option_sets(0, 64)
    assert all(np.array_equal(s[k], again[k]) for k in s)
    other = W.option_sets(1, 64)
    assert not np.array_equal(s["S0"], other["S0"])


def test_every_set_has_a_risk_neutral_crr_probability():
    """p = (e^{rate dt} - d)/(u - d) in (0, 1) for every set at every depth
    the workloads use (rate sqrt(dt) < sigma throughout)."""
    for seed, n in ((0, 64), (1, 256), (2, 10000)):
        s = W.option_sets(seed, n)
        for N in (16, 28, 36):
            dt = np.asarray(s["T"]) / N
            u = np.exp(np.asarray(s["sigma"]) * np.sqrt(dt))
            d = 1.0 / u
            p = (np.exp(np.asarray(s["rate"]) * dt) - d) / (u - d)
            assert np.all((p > 0.0) & (p < 1.0)), (seed, N)


def test_batched_and_greeks_workloads():
    b = W.batched_exact_workload(36, 0, 64)
    assert len(b) == 128 and {o["payoff"] for o in b} == {W.ASIAN_ARITH_CALL, W.ASIAN_ARITH_PUT}
    assert all(o["N"] == 36 for o in b)
    g = W.greeks_workload(28, 1, 256)
    assert len(g) == 512 and {o["payoff"] for o in g} == {W.ASIAN_ARITH_CALL, W.LOOKBACK_FIXED_CALL}


def test_serving_stream():
    arr, opts = W.serving_stream(2, 10000, 1000.0)
    assert len(arr) == len(opts) == 10000
    assert np.all(np.diff(arr) >= 0.0)
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert abs(gaps.mean() - 1e-3) < 5e-5          # Poisson at 1000/s: mean gap 1 ms
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05   # exponential gaps
    Ns = np.array([o["N"] for o in opts])
    assert Ns.min() == 16 and Ns.max() == 34 and len(set(Ns)) == 19
    pays = {o["payoff"] for o in opts}
    assert pays == {W.ASIAN_ARITH_CALL, W.ASIAN_ARITH_PUT, W.ASIAN_GEO_CALL, W.LOOKBACK_FIXED_CALL}


@pytest.mark.parametrize("N", [1, 12, 32])
def test_step_factors(N):
    st = np.asarray(W.step_factors(7, N, 0.01, 0.05))
    assert st.shape == (N, 3)
    u, d, p = st[:, 0], st[:, 1], st[:, 2]
    assert np.all(u > 1.0) and np.all(d > 0.0) and np.all(d < 1.0) and np.all((p > 0.0) & (p < 1.0))


@pytest.mark.parametrize("b", [2, 3, 5, 8])
def test_branch_moves(b):
    mv = W.branch_moves(11, 9, b)
    assert mv.shape == (9, 2 * b)
    f, q = mv[:, :b], mv[:, b:]
    assert np.all(np.diff(f, axis=1) >= 0.0)            # factors ascending by digit
    assert np.all(f[:, 0] < 1.0) and np.all(f[:, -1] > 1.0)
    assert np.allclose(q.sum(axis=1), 1.0, rtol=0, atol=1e-12) and np.all(q > 0.0)
