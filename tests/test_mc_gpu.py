"""GPU parity of the Monte Carlo estimators (Section 4) against the oracle.

The device draws the same Bernoulli bits as the oracle (same Philox counters,
key and threshold), so with equal seeds the estimates agree up to FP32
per-sample rounding (relative 2e-5 here); statistical properties are checked
against exact values from the exhaustive oracle.
"""
import math

import numpy as np
import pytest
from scipy import stats

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


def test_device_philox_matches_oracle(bt, ctx, oracle):
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2 ** 32, (257, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (257, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    got = bt.bt_philox4x32_10(ctx.h, ctr, key)
    for i in range(len(ctr)):
        assert got[i].tolist() == oracle.philox(ctr[i].tolist(), key[i].tolist()), i


@pytest.mark.parametrize("kind", [0, 1])
# suffix tails 0, 3, 2, 1, 0; the last two have 41 and 301 work items of 1024 samples per stratum, so
# a warp and a block combine each stratum's items (one thread does for the others)
@pytest.mark.parametrize("mb,R", [(0, 700), (1, 300), (2, 200), (3, 100), (4, 1500), (2, 40 * 1024 + 17),
                                  (1, 300 * 1024 + 3)])
def test_same_draws_as_oracle(bt, ctx, oracle, kind, mb, R):
    opts = [W.opt(12, 100.0, 101.0, 0.04, 0.3, 1.0, pay, W.TREE_SEYDEL if pay % 3 == 0 else W.TREE_CRR)
            for pay in range(8)]
    seed = 0x1234_5678_9ABC
    got = bt.bt_price_mc_ex(ctx.h, opts, mb, R, seed, kind)
    for i, o in enumerate(opts):
        th, var = oracle.mc(o, mb, R, seed, stream=i, shared=bool(kind))
        disc = oracle.discount(o)
        assert got["value"][i] == pytest.approx(disc * th, rel=2e-5, abs=1e-9), (i, kind, mb)
        assert got["stderr_mc"][i] == pytest.approx(disc * math.sqrt(var), rel=2e-4, abs=1e-9), (i, kind, mb)
        assert got["paths"][i] == (1 if kind else 2 ** mb) * R


def test_per_stratum_statistics_match_oracle(bt, ctx, oracle):
    o = W.opt(11, 97.0, 100.0, 0.05, 0.25, 1.0, W.ASIAN_ARITH_CALL)
    out, strata = bt.bt_price_mc_ex(ctx.h, [o], 5, 300, 99, 0, with_strata=True)
    th, var, mean, sv, pr = oracle.mc(o, 5, 300, 99, stream=0, with_strata=True)
    np.testing.assert_allclose(strata[0, :, 0], mean, rtol=2e-5, atol=1e-9)
    np.testing.assert_allclose(strata[0, :, 1], sv, rtol=5e-4, atol=1e-9)
    np.testing.assert_allclose(strata[0, :, 2], pr, rtol=1e-13)


def test_all_strata_is_exact(bt, ctx, oracle):
    """2^N strata: every stratum is one full path, the estimator is the exact sum."""
    opts = [W.opt(10, 100.0, 100.0, 0.05, 0.3, 1.0, pay) for pay in range(8)]
    got = bt.bt_price_mc(ctx.h, opts, 10, 2, 7)
    for i, o in enumerate(opts):
        assert got["value"][i] == pytest.approx(oracle.price_exhaustive(o, 1), rel=1e-6, abs=1e-9)
        assert got["stderr_mc"][i] == 0.0


@pytest.mark.parametrize("sigma", [5.0, 10.0])
def test_shared_sample_at_extreme_volatility(bt, ctx, oracle, sigma):
    """The Shared-Sample pair loop scales its table by 2^k with 2^k >= 2 max(sign (tau + f)); at
    sigma = 5 (a bound of f near 2^55) the scale is 2^57, at sigma = 10 (2^109) the table stays
    unscaled and the loop clamps with max. Both against the oracle on the same draws."""
    for pay in (W.ASIAN_ARITH_CALL, W.ASIAN_ARITH_PUT, W.LOOKBACK_FIXED_CALL):
        o = W.opt(64, 100.0, 100.0, 0.05, sigma, 1.0, pay)
        got = bt.bt_price_mc_ex(ctx.h, [o], 4, 300, 17, bt.BT_MC_SHARED)[0]
        th, var = oracle.mc(o, 4, 300, 17, stream=0, shared=True)
        disc = oracle.discount(o)
        assert got["value"] == pytest.approx(disc * th, rel=2e-5), (sigma, pay, got["value"], disc * th)
        assert got["stderr_mc"] == pytest.approx(disc * math.sqrt(var), rel=2e-4)


def test_shared_sample_over_all_prefixes_is_exact(bt, ctx, oracle):
    """Shared-Sample with 2^N prefixes: the suffixes are empty, every sample scores the whole tree,
    h_i = sum_x p(x) V(x) for each i (eq. mc16 with L = 0). The FP32 strata table and the blocked
    FP32 sum over 1024 prefixes bound the error near 80 ulps of the sum."""
    opts = [W.opt(10, 100.0, 100.0, 0.05, 0.3, 1.0, pay) for pay in range(8)]
    got = bt.bt_price_mc_ex(ctx.h, opts, 10, 300, 7, bt.BT_MC_SHARED)
    for i, o in enumerate(opts):
        ex = oracle.price_exhaustive(o, 1)
        assert got["value"][i] == pytest.approx(ex, rel=1e-5, abs=1e-9), (i, got["value"][i], ex)
        assert got["stderr_mc"][i] <= 1e-12 * max(abs(ex), 1.0)
        assert got["paths"][i] == 300


def test_maximum_strata_bits(bt, ctx, oracle):
    """2^24 strata (the largest Partitioned stratification) at N=24, one sample each: every
    stratum is one whole path, so the estimator is the exact sum over the 2^24 paths."""
    o = W.opt(24, 100.0, 98.0, 0.05, 0.25, 1.0, W.ASIAN_ARITH_CALL)
    got = bt.bt_price_mc(ctx.h, [o], 24, 1, 3)[0]
    ex = oracle.price_exhaustive(o, 16)
    assert got["value"] == pytest.approx(ex, rel=1e-6)
    assert got["paths"] == 1 << 24


@pytest.mark.parametrize("kind", [0, 1])
def test_maximum_depth(bt, ctx, oracle, kind):
    """N = 4096, the deepest tree the Monte Carlo path takes, against the oracle on the same draws.
    The FP32 walk of 4094 steps (a running product and a running sum of 4096 terms) departs from
    the oracle's FP64 walk by up to about N 2^-24 relative, so the check is at 1e-3."""
    o = W.opt(4096, 100.0, 100.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL)
    got = bt.bt_price_mc_ex(ctx.h, [o], 2, 64, 21, kind)[0]
    th, var = oracle.mc(o, 2, 64, 21, stream=0, shared=bool(kind))
    disc = oracle.discount(o)
    assert got["value"] == pytest.approx(disc * th, rel=1e-3)
    assert got["stderr_mc"] == pytest.approx(disc * math.sqrt(var), rel=1e-2)


def test_unbiased_at_n30_and_stderr_calibrated(bt, ctx, oracle):
    """N=30, 2^10 strata x 2^10 samples: within 3 SE of the exact value; the
    spread over seeds matches the reported standard error."""
    o = W.opt(30, 100.0, 100.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL)
    exact = oracle.asian_mitm(o, 15)
    vals, ses = [], []
    for seed in range(24):
        r = bt.bt_price_mc(ctx.h, [o], 10, 1024, 1000 + seed)
        vals.append(r["value"][0])
        ses.append(r["stderr_mc"][0])
    vals, ses = np.array(vals), np.array(ses)
    assert np.all(np.abs(vals - exact) <= 4 * ses)
    assert abs(vals.mean() - exact) <= 3 * ses.mean() / math.sqrt(len(vals))
    ratio = vals.var(ddof=1) / np.mean(ses ** 2)
    lo, hi = stats.chi2.ppf([1e-3, 1 - 1e-3], len(vals) - 1) / (len(vals) - 1)
    assert lo < ratio < hi


def test_stratification_reduces_variance(bt, ctx):
    """eq. mc15: at equal total samples the Partitioned estimator's variance is
    Var(plain) - Var_D E[V|D]/R, i.e. strictly below plain MC's; the reported
    var_plain (law of total variance) agrees with the plain estimate."""
    o = W.opt(64, 100.0, 100.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL)
    strat = bt.bt_price_mc(ctx.h, [o], 10, 1024, 3)[0]
    plain = bt.bt_price_mc(ctx.h, [o], 0, 1024 * 1024, 4)[0]
    assert strat["stderr_mc"] < 0.95 * plain["stderr_mc"]
    assert abs(strat["value"] - plain["value"]) < 4 * math.hypot(strat["stderr_mc"], plain["stderr_mc"])
    disc = math.exp(-0.05)
    sd_plain_from_strat = disc * math.sqrt(strat["var_plain"] / (1024 * 1024))
    assert sd_plain_from_strat == pytest.approx(plain["stderr_mc"], rel=0.05)


@pytest.mark.parametrize("N,mb,R", [(64, 12, 1024), (252, 10, 1024), (252, 16, 64)])
def test_put_call_parity_deep_trees(bt, ctx, N, mb, R):
    """Per draw, max(A-K,0) - max(K-A,0) = A - K, and E[A] = (S0/N) sum_t e^{q t dt}:
    the call and put estimates from the same draws differ by that forward."""
    S0, K, r, T = 100.0, 103.0, 0.05, 1.0
    opts = [W.opt(N, S0, K, r, 0.2, T, W.ASIAN_ARITH_CALL), W.opt(N, S0, K, r, 0.2, T, W.ASIAN_ARITH_PUT)]
    out = bt.bt_price_mc(ctx.h, opts, mb, R, 11)
    # same seed and counters: both options draw identical paths only if their stream ids
    # match, so price them one at a time
    c = bt.bt_price_mc(ctx.h, opts[:1], mb, R, 11)[0]
    p = bt.bt_price_mc(ctx.h, opts[1:], mb, R, 11)[0]
    dt = T / N
    fwd = math.exp(-r * T) * (S0 / N * sum(math.exp(r * t * dt) for t in range(1, N + 1)) - K)
    assert abs((c["value"] - p["value"]) - fwd) <= 4 * (c["stderr_mc"] + p["stderr_mc"])
    assert np.all(np.isfinite(out["value"])) and np.all(out["stderr_mc"] > 0)


def test_theorem1_on_gpu(bt, ctx, oracle):
    """Var(partitioned) <= Var(shared) <= Var(plain) with R_m = R (Theorem 1),
    Asian put as in Table 5, from the spread over seeds."""
    o = W.opt(16, 100.0, 100.0, 0.05, 0.4, 1.0, W.ASIAN_ARITH_PUT)
    part = [bt.bt_price_mc_ex(ctx.h, [o], 4, 256, s, 0)["value"][0] for s in range(60)]
    shar = [bt.bt_price_mc_ex(ctx.h, [o], 4, 256, s, 1)["value"][0] for s in range(60)]
    basic = [bt.bt_price_mc_ex(ctx.h, [o], 0, 256, s, 0)["value"][0] for s in range(60)]
    assert np.var(part) < np.var(shar) < np.var(basic)


def test_mc_invalid(bt, ctx):
    o = W.single_asian_n20()
    with pytest.raises(bt.BtError):
        bt.bt_price_mc(ctx.h, [o], 21, 10, 1)
    with pytest.raises(bt.BtError) as e:
        bt.bt_price_mc_ex(ctx.h, [o], 11, 10, 1, 1)
    assert e.value.status == bt.BT_EUNSUPPORTED
    with pytest.raises(bt.BtError):
        bt.bt_price_mc(ctx.h, [dict(o, N=5000)], 2, 10, 1)


@pytest.mark.parametrize("n_shards", [1, 3, 16])
def test_strata_shards_add_up(bt, ctx, n_shards):
    """bt_price_mc_shard: the shards' strata are the unsharded call's strata
    (bit for bit), their value terms sum to its value and their variance
    terms to its squared standard error."""
    o = W.opt(64, 100.0, 100.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL)
    full, st_full = bt.bt_price_mc_ex(ctx.h, [o], 4, 2000, 11, with_strata=True)
    v = se2 = paths = 0.0
    for s in range(n_shards):
        r, st = bt.bt_price_mc_shard(ctx.h, [o], 4, 2000, 11, s, n_shards, with_strata=True)
        assert np.array_equal(st[0], st_full[0][s::n_shards])
        v += r[0]["value"]
        se2 += r[0]["stderr_mc"] ** 2
        paths += r[0]["paths"]
    assert abs(v - full[0]["value"]) <= 1e-13 * full[0]["value"]
    assert abs(np.sqrt(se2) - full[0]["stderr_mc"]) <= 1e-12 * full[0]["stderr_mc"]
    assert paths == full[0]["paths"]


@pytest.mark.parametrize("pay,R", [(W.ASIAN_ARITH_CALL, 4096 + 333), (W.ASIAN_GEO_PUT, 2048 + 5)])
def test_shared_sample_at_the_benchmark_strata(bt, ctx, oracle, pay, R):
    """The Shared-Sample kernel at the benchmark's N=64 and 2^10 prefixes (the whole per-job strata
    table, 16 blocks of 64 prefixes in the pair loop), with a ragged last work item, against the
    oracle's estimator on the same Philox draws. Tolerances: the FP32 suffix walk (under 1e-6
    relative at N=64) and the blocked FP32 sum over 1024 prefixes (under 80 ulps)."""
    o = W.opt(64, 100.0, 100.0, 0.05, 0.2, 1.0, pay)
    seed = 11
    got = bt.bt_price_mc_ex(ctx.h, [o], 10, R, seed, bt.BT_MC_SHARED)[0]
    th, var = oracle.mc(o, 10, R, seed, stream=0, shared=True)
    disc = oracle.discount(o)
    assert got["value"] == pytest.approx(disc * th, rel=2e-5), (got["value"], disc * th)
    assert got["stderr_mc"] == pytest.approx(disc * math.sqrt(var), rel=5e-4)
    assert got["paths"] == R


def test_full_size_strata_sampled_against_the_oracle(bt, ctx, oracle):
    """The benchmark's Monte Carlo configuration at full size (N=252, 2^16
    strata x 2^14 samples): sampled strata recomputed one by one by the
    oracle with the same Philox draws. The GPU walks the 236 suffix steps in
    FP32, so the stratum means agree to about 1e-5, not bit for bit."""
    o = W.opt(252, 100.0, 100.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL)
    mb, R, seed = 16, 1 << 14, 5
    r, st = bt.bt_price_mc_ex(ctx.h, [o], mb, R, seed, with_strata=True)
    assert r[0]["paths"] == R << mb
    for z in (0, 1, 4660, 32768, 65535):
        mz, vz, pz = oracle.mc_stratum(o, mb, z, R, seed)
        g_mean, g_var, g_prob = st[0][z]
        assert abs(g_mean - mz) <= 1e-4 * abs(mz) + 1e-6 * o["S0"], (z, g_mean, mz)
        assert abs(g_var - vz) <= 1e-3 * vz + 1e-9, (z, g_var, vz)
        assert abs(g_prob - pz) <= 1e-12 * pz, (z, g_prob, pz)
