"""GPU parity of the exhaustive sums (eq. f13) against the CPU oracle.

Tolerances (relative, plus an absolute floor of 1e-12 * S0 for values that are
(nearly) zero, where a relative bound has no meaning):
  FP64 kernel: 1e-12.
  FP32_COMP kernel: 1e-9 at every N. From 2^28 paths the arithmetic Asian's
  per-path pass rounds each path's payoff once in FP32 (relative error <=
  2^-24) and those errors average out over the many paths; below 2^28 paths
  it takes the class pass with each suffix its own class. The European,
  geometric and lookback payoffs are summed over recombined suffix classes in
  FP32-pair arithmetic with no per-path FP32 rounding.
All calls go through the C ABI.
"""
import math

import numpy as np
import pytest

from paper_1701_03512_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-9}   # BT_PREC_FP64, BT_PREC_FP32_COMP at N >= 28


def tol(prec, N, payoff=2):
    """The accuracy contract: FP64 1e-12; FP32_COMP 1e-9 at every N (the
    arithmetic Asian below 2^28 paths sums each suffix as a class in FP32
    pairs, like the other payoffs)."""
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


def _check(got, ref, opts, prec, what=""):
    got = np.asarray(got, dtype=float)
    ref = np.asarray(ref, dtype=float)
    s0 = np.array([o["S0"] for o in opts])
    err = np.abs(got - ref)
    bound = np.array([tol(prec, o["N"], o["payoff"]) for o in opts]) * np.abs(ref) + 1e-12 * s0
    bad = np.nonzero(~(err <= bound))[0]
    assert bad.size == 0, "%s prec=%d: %s" % (what, prec, [(int(i), opts[i]["payoff"], opts[i]["N"], got[i], ref[i],
                                                           err[i] / max(abs(ref[i]), 1e-300)) for i in bad[:8]])


@pytest.mark.parametrize("prec", [0, 1])
def test_single_asian_n20(bt, ctx, oracle, prec):
    """One arithmetic-average Asian call, N=20, CRR, S0=K=100, r=5%, sigma=20%, T=1."""
    o = W.single_asian_n20()
    ref = oracle.price_exhaustive(o, 8)
    r = ctx.price_exact([o], prec)
    _check(r["value"], [ref], [o], prec, "N=20")
    assert r["paths"][0] == 2 ** 20


@pytest.mark.parametrize("prec", [0, 1])
def test_all_payoffs_small_trees(bt, ctx, oracle, prec):
    """Every payoff, N = 1..16, three tree kinds, against plain enumeration."""
    opts = []
    rng = np.random.default_rng(7)
    for N in list(range(1, 17)):
        for pay in range(8):
            kind = [W.TREE_CRR, W.TREE_SEYDEL, W.TREE_EXPLICIT][(N + pay) % 3]
            S0, K = rng.uniform(80, 120, 2)
            if kind == W.TREE_EXPLICIT:
                u = 1.0 + rng.uniform(0.01, 0.08)
                opts.append(W.opt(N, S0, K, 0.03, 0.2, 1.0, pay, kind, u=u, d=1.0 / u, p=rng.uniform(0.3, 0.7)))
            else:
                opts.append(W.opt(N, S0, K, rng.uniform(0, 0.08), rng.uniform(0.1, 0.5), rng.uniform(0.25, 2), pay, kind))
    ref = [oracle.price_exhaustive(o, 8) for o in opts]
    r = ctx.price_exact(opts, prec)
    _check(r["value"], ref, opts, prec, "small")
    assert r["paths"].tolist() == [2 ** o["N"] for o in opts]


def test_two_step_worked_example(bt, ctx, golden_dir):
    import json, os
    g = json.load(open(os.path.join(golden_dir, "n2_worked_example.json")))
    t = g["tree"]
    names = list(g["values"])
    opts = [W.opt(2, t["S0"], t["K"], t["rate"], 0.2, t["T"],
                  [k for k, v in W.PAYOFF_NAMES.items() if v == n][0], W.TREE_EXPLICIT, u=t["u"], d=t["d"], p=t["p"])
            for n in names]
    for prec in (0, 1):
        got = ctx.price_exact(opts, prec)["value"]
        assert np.allclose(got, [g["values"][n] for n in names], rtol=tol(prec, 2), atol=1e-13), (prec, got)


def test_paper_exact_values(bt, ctx, golden_dir):
    """The Section 5 exact values (N=32, Seydel) from the GPU path."""
    import json, os
    g = json.load(open(os.path.join(golden_dir, "paper_section5_exact.json")))
    c = g["common"]
    opts = [W.opt(c["N"], c["S0"], c["K"], c["rate"], c["sigma"], c["T"], W.ASIAN_ARITH_PUT, W.TREE_SEYDEL),
            W.opt(c["N"], c["S0"], c["K"], c["rate"], c["sigma"], c["T"], W.LOOKBACK_FIXED_PUT, W.TREE_SEYDEL)]
    got = ctx.price_exact(opts, 1)["value"]
    assert abs(got[0] - g["values"]["asian_arith_put"]) <= 5e-4
    assert abs(got[1] - g["values"]["lookback_fixed_put"]) <= 5e-4


@pytest.mark.parametrize("N", [11, 12, 15, 16, 17, 22, 27, 28, 29])
def test_split_boundaries(bt, ctx, oracle, N):
    """Around the prefix/suffix split changes (L = N - 15 from N = 16, 13 from N = 28; the class pass
    of the FP32 arithmetic Asian up to N = 27)."""
    opts = W.batch(N, W.option_sets(N, 2), list(range(8)))
    ref = [oracle.exact(o) if N > 18 else oracle.price_exhaustive(o, 8) for o in opts]
    for prec in (0, 1):
        _check(ctx.price_exact(opts, prec)["value"], ref, opts, prec, "N=%d" % N)


def test_call_put_pair_matches_singles(bt, ctx):
    """A fused call/put pass gives bit-identical values to separate passes."""
    sets = W.option_sets(3, 3)
    pair = W.batch(24, sets, (W.ASIAN_ARITH_CALL, W.ASIAN_ARITH_PUT))
    calls = [o for o in pair if o["payoff"] == W.ASIAN_ARITH_CALL]
    puts = [o for o in pair if o["payoff"] == W.ASIAN_ARITH_PUT]
    for prec in (0, 1):
        rp = ctx.price_exact(pair, prec)["value"]
        rc = ctx.price_exact(calls, prec)["value"]
        rq = ctx.price_exact(puts, prec)["value"]
        assert np.array_equal(rp[0::2], rc) and np.array_equal(rp[1::2], rq)


def test_deterministic_alone_and_batched(bt, ctx):
    opts = W.random_options(11, 24, 10, 28)
    for prec in (0, 1):
        a = ctx.price_exact(opts, prec)["value"]
        b = ctx.price_exact(opts, prec)["value"]
        assert np.array_equal(a, b)
        for i in (0, 5, 17):
            assert ctx.price_exact([opts[i]], prec)["value"][0] == a[i]


def test_work_item_partials_against_enumeration(bt, ctx, oracle):
    """Sampled work items of an N=32 pass: each covers a contiguous range of
    path indices, whose sum the oracle enumerates directly (eq. f14)."""
    opts = W.batched_exact_workload(32, 0, 2)[:2] + [W.opt(32, 100.0, 95.0, 0.04, 0.3, 1.0, W.LOOKBACK_FIXED_CALL)]
    for prec in (0, 1):
        plan = bt.bt_exact_plan_create(ctx.h, opts, prec)
        try:
            bt.bt_exact_plan_run(plan)
            part, job, first = bt.bt_exact_plan_partials(plan)
            for item in (0, 137, len(job) - 1):
                jd = bt.bt_exact_plan_job(plan, int(job[item]))
                L = jd["L"]
                lo = int(first[item]) << L
                hi = (int(first[item]) + jd["prefixes_per_item"]) << L
                for slot, oi in ((0, jd["opt_call"]), (1, jd["opt_put"])):
                    if oi < 0:
                        continue
                    ref = oracle.sum_range(opts[oi], lo, hi)
                    got = part[item, slot]
                    # one work item holds 2^22 paths: the N >= 20 band
                    assert abs(got - ref) <= tol(prec, 22) * abs(ref) + 1e-15 * opts[oi]["S0"], (prec, item, slot, got, ref)
        finally:
            bt.bt_exact_plan_destroy(plan)


@pytest.mark.parametrize("N", [32, 36])
def test_batched_workload_full_size(bt, ctx, oracle, N):
    """The batched workload (64 sets, arithmetic Asian call and put) at full
    size against the exact meet-in-the-middle oracle, FP32_COMP kernel."""
    opts = W.batched_exact_workload(N, 0, 64)
    ref = [oracle.asian_mitm(o, N // 2) for o in opts]
    r = ctx.price_exact(opts, 1)
    _check(r["value"], ref, opts, 1, "N=%d" % N)
    rel = np.abs(r["value"] - ref) / np.maximum(np.abs(ref), 1e-300)
    print("N=%d max rel err %.3g (values > 1e-6): %.3g" % (N, rel.max(), rel[np.abs(ref) > 1e-6].max()))


def test_batched_workload_fp64_n32(bt, ctx, oracle):
    opts = W.batched_exact_workload(32, 0, 64)
    ref = [oracle.asian_mitm(o, 16) for o in opts]
    _check(ctx.price_exact(opts, 0)["value"], ref, opts, 0, "fp64 N=32")


@pytest.mark.parametrize("N", [30, 36])
def test_geometric_and_lookback_full_size(bt, ctx, oracle, N):
    sets = W.option_sets(5, 6)
    opts = W.batch(N, sets, (W.ASIAN_GEO_CALL, W.ASIAN_GEO_PUT, W.LOOKBACK_FIXED_CALL, W.LOOKBACK_FIXED_PUT))
    ref = [oracle.exact(o) for o in opts]
    _check(ctx.price_exact(opts, 1)["value"], ref, opts, 1, "geo/lookback N=%d" % N)


@pytest.mark.parametrize("N", [5, 14, 24, 30, 34])
def test_recombined_payoffs_against_oracle(bt, ctx, oracle, N):
    """European, geometric and lookback payoffs on 24 option sets (K/S0 from
    about 0.67 to 1.5, so deep in and out of the money) against the oracle's
    closed form and exact DPs: 1e-9 relative at every N. Before the class
    tables, per-path FP32 rounding repeated identically over equal suffix
    values and deep out-of-the-money sets missed 1e-9 by up to 2x."""
    sets = W.option_sets(300 + N, 24)
    opts = W.batch(N, sets, (W.EURO_CALL, W.EURO_PUT, W.ASIAN_GEO_CALL, W.ASIAN_GEO_PUT,
                             W.LOOKBACK_FIXED_CALL, W.LOOKBACK_FIXED_PUT))
    got = ctx.price_exact(opts, 1)["value"]
    for o, g in zip(opts, got):
        ref = oracle.exact(o)
        assert abs(g - ref) <= 1e-9 * abs(ref) + 1e-12 * o["S0"], (o, g, ref, (g - ref) / ref)


def test_shards_add_up(bt, ctx):
    opts = W.random_options(21, 10, 18, 30)
    for prec in (0, 1):
        plan = bt.bt_exact_plan_create(ctx.h, opts, prec)
        try:
            bt.bt_exact_plan_run(plan)
            full = bt.bt_exact_plan_read(plan)["value"]
            tot = np.zeros(len(opts))
            for s in range(3):
                bt.bt_exact_plan_run_shard(plan, s, 3)
                tot += bt.bt_exact_plan_read(plan)["value"]
            assert np.allclose(tot, full, rtol=1e-14, atol=0)
        finally:
            bt.bt_exact_plan_destroy(plan)


def test_invalid_inputs(bt, ctx):
    good = W.single_asian_n20()
    with pytest.raises(bt.BtError) as e:
        ctx.price_exact([good, dict(good, N=41)], 1)
    assert e.value.status == bt.BT_EINVAL and "N=41" in str(e.value)
    with pytest.raises(bt.BtError) as e:
        ctx.price_exact([good, dict(good, S0=0.0)], 1)
    assert e.value.status == bt.BT_EINVAL and "option 1" in str(e.value)
    o = W.opt(10, 100.0, 100.0, 0.0, 0.2, 1.0, W.EURO_CALL, W.TREE_EXPLICIT, u=1.2, d=1 / 1.2, p=0.001)
    with pytest.raises(bt.BtError) as e:
        ctx.price_exact([o], 1)
    assert e.value.status == bt.BT_EUNSUPPORTED
    assert ctx.price_exact([o], 0)["value"][0] >= 0.0


def test_budget_is_enforced(bt):
    c = bt.Context(0, device_budget_bytes=1 << 20)
    try:
        with pytest.raises(bt.BtError) as e:
            c.price_exact(W.batched_exact_workload(36, 0, 4), 1)
        assert e.value.status == bt.BT_EBUDGET
        assert bt.bt_device_bytes(c.h) == 0
    finally:
        c.close()


def test_maximum_size_n40(bt, ctx, oracle):
    """N = 40, the largest tree the exhaustive pass takes: an arithmetic call
    and put pair (one fused pass of 2^40 paths each) against the oracle's
    meet-in-the-middle value, and the class payoffs against the exact DPs."""
    opts = [W.opt(40, 100.0, 102.0, 0.04, 0.25, 1.0, W.ASIAN_ARITH_CALL),
            W.opt(40, 100.0, 102.0, 0.04, 0.25, 1.0, W.ASIAN_ARITH_PUT),
            W.opt(40, 100.0, 97.0, 0.04, 0.25, 1.0, W.ASIAN_GEO_CALL),
            W.opt(40, 100.0, 110.0, 0.04, 0.25, 1.0, W.LOOKBACK_FIXED_CALL),
            W.opt(40, 100.0, 92.0, 0.04, 0.25, 1.0, W.LOOKBACK_FIXED_PUT)]
    got = ctx.price_exact(opts, 1)
    assert np.all(got["paths"] == 2 ** 40)
    ref = [oracle.asian_mitm(o, 20) if o["payoff"] in (2, 3) else oracle.exact(o) for o in opts]
    _check(got["value"], ref, opts, 1, "N=40")


def test_degenerate_strikes(bt, ctx, oracle):
    """K = 0: every path is in the money and the arithmetic call is the mean
    of the average price, (S0/N) sum_t e^{rate t dt} on a risk-neutral tree;
    a strike far above every price gives exactly 0 for the calls (and the
    puts are the discounted strike minus that mean)."""
    N, r, T = 30, 0.05, 1.0
    mean_avg = 100.0 / N * sum(math.exp(r * t * T / N) for t in range(1, N + 1))
    disc = math.exp(-r * T)
    zero_k = [W.opt(N, 100.0, 0.0, r, 0.2, T, W.ASIAN_ARITH_CALL), W.opt(N, 100.0, 0.0, r, 0.2, T, W.EURO_CALL)]
    got = ctx.price_exact(zero_k, 1)["value"]
    assert abs(got[0] - disc * mean_avg) <= 1e-9 * disc * mean_avg
    assert abs(got[1] - 100.0) <= 1e-9 * 100.0
    big = 1e7
    far = [W.opt(N, 100.0, big, r, 0.2, T, pay) for pay in (0, 2, 4, 6)]
    assert np.all(ctx.price_exact(far, 1)["value"] == 0.0)
    put = ctx.price_exact([W.opt(N, 100.0, big, r, 0.2, T, W.ASIAN_ARITH_PUT)], 1)["value"][0]
    ref = disc * (big - mean_avg)
    assert abs(put - ref) <= 1e-9 * ref


def test_empty_and_single_step(bt, ctx, oracle):
    with pytest.raises(bt.BtError) as e:
        bt.bt_price_exact(ctx.h, [], 1)
    assert e.value.status == bt.BT_EINVAL
    for pay in range(8):
        o = W.opt(1, 100.0, 100.0, 0.05, 0.2, 1.0, pay)
        for prec in (0, 1):
            got = ctx.price_exact([o], prec)["value"][0]
            ref = oracle.price_exhaustive(o, 1)
            assert abs(got - ref) <= tol(prec, 1, pay) * abs(ref) + 1e-12 * 100.0, (pay, prec, got, ref)


@pytest.mark.parametrize("N", [9, 16, 22, 26])
def test_stated_error_covers_the_difference_to_the_oracle(bt, ctx, oracle, N):
    """err_est of every result (the accuracy contract for its depth, payoff
    and precision) bounds its distance to the oracle."""
    opts = W.batch(N, W.option_sets(70 + N, 3), list(range(8)))
    ref = np.array([oracle.exact(o) if N > 18 else oracle.price_exhaustive(o, 8) for o in opts])
    s0 = np.array([o["S0"] for o in opts])
    for prec in (0, 1):
        r = ctx.price_exact(opts, prec)
        assert np.all(np.abs(r["value"] - ref) <= r["err_est"] + 1e-12 * s0), (prec, N)
        assert np.all(r["err_est"] <= np.array([tol(prec, N, o["payoff"]) for o in opts]) * np.abs(r["value"]) * 1.01)


def test_probability_limit_of_the_fp32_path(bt, ctx, oracle):
    """min(p, 1-p) >= 0.004 is accepted in FP32 and meets the 1e-9 contract;
    below it FP32 is refused and FP64 still prices. Skewed trees (p = 0.9,
    0.996: the all-up path alone carries 89 % of the probability at 0.996)
    have far fewer than 2^27 effective paths, 1 / sum_x p(x)^2, so per-path
    FP32 roundings could not average out: they take the pair-sum class pass
    (L <= 12), which rounds no single path, and every stated error is
    1e-9 |V|."""
    u = 1.05
    d = 1 / u
    for p, ok in ((0.004, True), (0.996, True), (0.9, True), (0.0039, False)):
        o = W.opt(28, 100.0, 100.0, 0.0, 0.2, 1.0, W.ASIAN_ARITH_CALL, W.TREE_EXPLICIT, u=u, d=d, p=p)
        if ok:
            r = ctx.price_exact([o], 1)[0]
            ref = oracle.exact(o)
            assert r["err_est"] == pytest.approx(1e-9 * abs(r["value"]), rel=1e-12)
            assert abs(r["value"] - ref) <= 1e-9 * abs(ref) + 1e-12 * 100.0, (p, r["value"], ref)
            assert bt.bt_exact_split(o, 1)["L"] == 12          # the class pass's split
        else:
            with pytest.raises(bt.BtError) as e:
                ctx.price_exact([o], 1)
            assert e.value.status == bt.BT_EUNSUPPORTED
            assert ctx.price_exact([o], 0)["value"][0] > 0.0


def _p_at_neff(N, bits):
    """p with (p^2 + (1-p)^2)^-N = 2^bits, p >= 1/2."""
    c = 2.0 ** (-bits / N)
    return 0.5 * (1.0 + math.sqrt(2.0 * c - 1.0))


@pytest.mark.parametrize("N", [28, 32])
def test_effective_path_threshold(bt, ctx, oracle, N):
    """Either side of the routing bound of 2^27 effective paths: p just
    inside it keeps the per-path pass (L = 13), just outside takes the class
    pass (L = 12); both at the 1e-9 contract against the oracle, for calls
    and puts in and out of the money, with drift up and down."""
    pc = _p_at_neff(N, 27.0)
    u = 1.03
    for p, L in ((pc - 0.005, 13), (pc + 0.005, 12), (1 - pc - 0.005, 12), (1 - pc + 0.005, 13)):
        opts = [W.opt(N, 100.0, K, 0.0, 0.2, 1.0, pay, W.TREE_EXPLICIT, u=u, d=1 / u, p=p)
                for K in (80.0, 100.0, 125.0) for pay in (W.ASIAN_ARITH_CALL, W.ASIAN_ARITH_PUT)]
        assert bt.bt_exact_split(opts[0], 1)["L"] == L, (p, L)
        got = ctx.price_exact(opts, 1)
        ref = [oracle.exact(o) for o in opts]
        _check(got["value"], ref, opts, 1, "N=%d p=%.4f" % (N, p))
        assert np.allclose(got["err_est"], 1e-9 * np.abs(got["value"]), rtol=1e-12)


@pytest.mark.parametrize("N", [28, 32])
def test_per_path_pass_across_the_accepted_skews(bt, ctx, oracle, N):
    """The per-path FP32 pass over the trees it accepts, from p = 1/2 to the
    effective-path bound (2^27): explicit lattices with small and large moves,
    calls and puts from deep in to deep out of the money, every value within
    1e-9 of the oracle's meet-in-the-middle value (plus 1e-12 S0)."""
    pc = _p_at_neff(N, 27.0)
    opts = []
    for u in (1.02, 1.05):
        for p in np.linspace(0.5, pc - 1e-3, 4):
            for pp in (p, 1.0 - p):
                opts += [W.opt(N, 100.0, K, 0.0, 0.2, 1.0, pay, W.TREE_EXPLICIT, u=u, d=1 / u, p=pp)
                         for K in (70.0, 95.0, 105.0, 140.0) for pay in (W.ASIAN_ARITH_CALL, W.ASIAN_ARITH_PUT)]
    assert all(bt.bt_exact_split(o, 1)["L"] == 13 for o in opts)     # all on the per-path pass
    got = ctx.price_exact(opts, 1)["value"]
    ref = [oracle.exact(o) for o in opts]
    _check(got, ref, opts, 1, "per-path pass, N=%d" % N)


def test_paper_section5_parameters_to_the_contract(bt, ctx, oracle):
    """The Section 5 tree (Seydel, sigma = 3, S0 = 20, K = 100, N = 32: prices
    spread over ten decades) for every payoff, FP32 and FP64, against the
    oracle at the contract tolerance -- not only the paper's three decimals."""
    opts = [W.opt(32, 20.0, 100.0, 0.06, 3.0, 1.0, pay, W.TREE_SEYDEL) for pay in range(8)]
    ref = [oracle.asian_mitm(o, 16) if o["payoff"] in (2, 3) else oracle.exact(o) for o in opts]
    for prec in (0, 1):
        _check(ctx.price_exact(opts, prec)["value"], ref, opts, prec, "Section 5 tree")
