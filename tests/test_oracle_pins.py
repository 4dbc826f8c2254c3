"""Pins of the CPU oracle to things other than itself.

Each test ties an oracle routine to the paper's printed values, a closed form,
an identity of the model, a library routine, or an independent brute force on
tiny inputs -- chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

from paper_1701_03512_gb300 import workloads as W

PAYOFFS = list(range(8))


def _explicit(N, S0, K, u, p, payoff, rate=0.0, T=1.0):
    return W.opt(N, S0, K, rate, 0.2, T, payoff, W.TREE_EXPLICIT, u=u, d=1.0 / u, p=p)


# --------------------------------------------------------------------------
# Tree parameters (Section 2, A1-A3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind", [W.TREE_CRR, W.TREE_SEYDEL])
@pytest.mark.parametrize("N,sigma,rate,T", [(20, 0.2, 0.05, 1.0), (32, 3.0, 0.06, 1.0), (7, 0.45, 0.0, 2.0)])
def test_tree_mean_condition(oracle, kind, N, sigma, rate, T):
    u, d, p = oracle.tree(kind, N, sigma, rate, T)
    dt = T / N
    assert abs(u * d - 1.0) < 1e-15                                   # A1
    assert 0.0 < p < 1.0                                               # A2
    assert abs(p * u + (1 - p) * d - math.exp(rate * dt)) < 1e-14     # A3


@pytest.mark.parametrize("N,sigma,rate,T", [(20, 0.2, 0.05, 1.0), (32, 3.0, 0.06, 1.0), (5, 0.7, 0.03, 0.5)])
def test_seydel_second_moment(oracle, N, sigma, rate, T):
    """Seydel's tree also matches the lognormal second moment:
    p u^2 + (1-p) d^2 = e^{(2q + sigma^2) dt}. This is what fixes the sign
    under the square root of u = beta + sqrt(beta^2 -+ 1)."""
    u, d, p = oracle.tree(W.TREE_SEYDEL, N, sigma, rate, T)
    dt = T / N
    lhs = p * u * u + (1 - p) * d * d
    assert abs(lhs / math.exp((2 * rate + sigma ** 2) * dt) - 1.0) < 1e-13


def test_crr_u(oracle):
    u, d, p = oracle.tree(W.TREE_CRR, 20, 0.2, 0.05, 1.0)
    assert u == pytest.approx(math.exp(0.2 * math.sqrt(1 / 20)), rel=1e-15)


# --------------------------------------------------------------------------
# The worked two-step tree and the paper's printed exact values
# --------------------------------------------------------------------------
def test_two_step_worked_example(oracle, golden_dir):
    g = json.load(open(os.path.join(golden_dir, "n2_worked_example.json")))
    t = g["tree"]
    for name, val in g["values"].items():
        pay = [k for k, v in W.PAYOFF_NAMES.items() if v == name][0]
        o = W.opt(2, t["S0"], t["K"], t["rate"], 0.2, t["T"], pay, W.TREE_EXPLICIT,
                  u=t["u"], d=t["d"], p=t["p"])
        assert oracle.price_exhaustive(o, 1) == pytest.approx(val, abs=1e-13), name
    # the four paths' prices: (up,down) and (down,up) both return to S
    o = W.opt(2, t["S0"], t["K"], 0.0, 0.2, 1.0, W.EURO_CALL, W.TREE_EXPLICIT, u=2.0, d=0.5, p=0.5)
    assert oracle.path_payoff(o, 0b11) == 11.0 and oracle.path_payoff(o, 0b10) == 0.0
    assert oracle.path_prob(o, 0b01) == 0.25


def test_paper_exact_values(oracle, golden_dir):
    g = json.load(open(os.path.join(golden_dir, "paper_section5_exact.json")))
    c = g["common"]
    asian = W.opt(c["N"], c["S0"], c["K"], c["rate"], c["sigma"], c["T"], W.ASIAN_ARITH_PUT, W.TREE_SEYDEL)
    look = W.opt(c["N"], c["S0"], c["K"], c["rate"], c["sigma"], c["T"], W.LOOKBACK_FIXED_PUT, W.TREE_SEYDEL)
    half_ulp = 0.5 * 10 ** (-g["printed_decimals"])
    assert abs(oracle.asian_mitm(asian, 16) - g["values"]["asian_arith_put"]) <= half_ulp
    assert abs(oracle.lookback_dp(look) - g["values"]["lookback_fixed_put"]) <= half_ulp


def test_paper_values_reject_other_readings(oracle, golden_dir):
    """The CRR tree does not reproduce the printed values, so the Seydel
    reading is not a free choice."""
    g = json.load(open(os.path.join(golden_dir, "paper_section5_exact.json")))
    c = g["common"]
    asian = W.opt(c["N"], c["S0"], c["K"], c["rate"], c["sigma"], c["T"], W.ASIAN_ARITH_PUT, W.TREE_CRR)
    assert abs(oracle.asian_mitm(asian, 16) - g["values"]["asian_arith_put"]) > 0.1


# --------------------------------------------------------------------------
# Weights: eq. f11 and sum-to-one
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N,p", [(1, 0.3), (9, 0.52), (13, 0.81)])
def test_leaf_probabilities_binomial(oracle, N, p):
    o = _explicit(N, 100.0, 100.0, 1.05, p, W.EURO_CALL)
    leaf = oracle.leaf_prob_sums(o)
    ref = stats.binom.pmf(np.arange(N + 1), N, p)
    np.testing.assert_allclose(leaf, ref, rtol=1e-13, atol=1e-300)
    assert abs(leaf.sum() - 1.0) < 1e-14


# --------------------------------------------------------------------------
# European: enumeration == eq. f8 == backward induction; martingale; Black-Scholes
# --------------------------------------------------------------------------
@pytest.mark.parametrize("payoff", [W.EURO_CALL, W.EURO_PUT])
@pytest.mark.parametrize("N,kind", [(6, W.TREE_CRR), (13, W.TREE_SEYDEL), (14, W.TREE_CRR)])
def test_european_three_ways(oracle, payoff, N, kind):
    o = W.opt(N, 97.0, 103.0, 0.04, 0.3, 1.5, payoff, kind)
    a = oracle.price_exhaustive(o, 4)
    b = oracle.european_closed(o)
    c = oracle.european_backward(o)
    assert a == pytest.approx(b, rel=1e-13) and b == pytest.approx(c, rel=1e-13)


def test_european_zero_strike_is_spot(oracle):
    """E[S_N] = S0 e^{qT} under A3, so a zero-strike call is worth S0."""
    for N in (5, 12):
        o = W.opt(N, 87.5, 0.0, 0.07, 0.25, 2.0, W.EURO_CALL, W.TREE_SEYDEL)
        assert oracle.price_exhaustive(o, 2) == pytest.approx(87.5, rel=1e-13)
        assert oracle.european_closed(o) == pytest.approx(87.5, rel=1e-13)


def test_european_converges_to_black_scholes(oracle):
    S0, K, r, s, T = 100.0, 95.0, 0.05, 0.25, 1.0
    d1 = (math.log(S0 / K) + (r + 0.5 * s * s) * T) / (s * math.sqrt(T))
    d2 = d1 - s * math.sqrt(T)
    bs = S0 * stats.norm.cdf(d1) - K * math.exp(-r * T) * stats.norm.cdf(d2)
    v = oracle.european_closed(W.opt(2000, S0, K, r, s, T, W.EURO_CALL, W.TREE_CRR))
    assert abs(v - bs) < 5e-3


# --------------------------------------------------------------------------
# Arithmetic Asian: closed forms, parity, MITM vs brute force
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind", [W.TREE_CRR, W.TREE_SEYDEL])
def test_asian_zero_strike_closed_form(oracle, kind):
    """K=0: V = e^{-qT} (S0/N) sum_{t=1}^N e^{q t dt}."""
    N, S0, r, T = 11, 100.0, 0.05, 1.25
    o = W.opt(N, S0, 0.0, r, 0.35, T, W.ASIAN_ARITH_CALL, kind)
    dt = T / N
    ref = math.exp(-r * T) * S0 / N * sum(math.exp(r * t * dt) for t in range(1, N + 1))
    assert oracle.price_exhaustive(o, 2) == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("N", [3, 10, 15])
def test_asian_put_call_parity(oracle, N):
    S0, K, r, T = 95.0, 101.0, 0.03, 0.8
    c = oracle.price_exhaustive(W.opt(N, S0, K, r, 0.4, T, W.ASIAN_ARITH_CALL), 4)
    p = oracle.price_exhaustive(W.opt(N, S0, K, r, 0.4, T, W.ASIAN_ARITH_PUT), 4)
    dt = T / N
    fwd = S0 / N * sum(math.exp(r * t * dt) for t in range(1, N + 1))
    assert c - p == pytest.approx(math.exp(-r * T) * (fwd - K), rel=1e-12)


@pytest.mark.parametrize("payoff", [W.ASIAN_ARITH_CALL, W.ASIAN_ARITH_PUT])
@pytest.mark.parametrize("N,L", [(8, 4), (13, 6), (16, 9), (16, 16)])
def test_asian_mitm_matches_enumeration(oracle, payoff, N, L):
    for seed in range(3):
        s = W.option_sets(seed + 50, 1)
        o = W.opt(N, s["S0"][0], s["K"][0], s["rate"][0], s["sigma"][0], s["T"][0], payoff,
                  W.TREE_SEYDEL if seed == 2 else W.TREE_CRR)
        assert oracle.asian_mitm(o, L) == pytest.approx(oracle.price_exhaustive(o, 8), rel=1e-12, abs=1e-14)


# --------------------------------------------------------------------------
# Geometric Asian and lookback: exact DPs vs brute force
# --------------------------------------------------------------------------
@pytest.mark.parametrize("payoff", [W.ASIAN_GEO_CALL, W.ASIAN_GEO_PUT])
@pytest.mark.parametrize("N", [1, 7, 14])
def test_geometric_dp_matches_enumeration(oracle, payoff, N):
    o = W.opt(N, 104.0, 99.0, 0.02, 0.3, 1.0, payoff, W.TREE_CRR)
    assert oracle.geometric_dp(o) == pytest.approx(oracle.price_exhaustive(o, 8), rel=1e-12)


@pytest.mark.parametrize("payoff", [W.LOOKBACK_FIXED_CALL, W.LOOKBACK_FIXED_PUT])
@pytest.mark.parametrize("N", [1, 6, 14])
def test_lookback_dp_matches_enumeration(oracle, payoff, N):
    o = W.opt(N, 100.0, 102.0, 0.05, 0.25, 1.0, payoff, W.TREE_SEYDEL)
    assert oracle.lookback_dp(o) == pytest.approx(oracle.price_exhaustive(o, 8), rel=1e-12)


def test_geometric_below_arithmetic(oracle):
    """AM >= GM on every path, so the geometric call is worth less."""
    o_a = W.opt(12, 100.0, 95.0, 0.05, 0.3, 1.0, W.ASIAN_ARITH_CALL)
    o_g = dict(o_a, payoff=W.ASIAN_GEO_CALL)
    assert oracle.price_exhaustive(o_g, 2) < oracle.price_exhaustive(o_a, 2)


# --------------------------------------------------------------------------
# Independent brute force (vectorised numpy) on tiny trees, all payoffs
# --------------------------------------------------------------------------
def _numpy_enumeration(N, S0, K, u, d, p, payoff):
    b = np.arange(2 ** N, dtype=np.int64)[:, None]
    t = np.arange(1, N + 1)[None, :]
    x = (b >> (N - t)) & 1
    U = np.cumsum(x, axis=1)
    S = S0 * u ** U * d ** (t - U)
    q = {0: S[:, -1], 1: S[:, -1], 2: S.mean(1), 3: S.mean(1),
         4: np.exp(np.log(S).mean(1)), 5: np.exp(np.log(S).mean(1)), 6: S.max(1), 7: S.min(1)}[payoff]
    pay = np.maximum(q - K, 0) if payoff % 2 == 0 else np.maximum(K - q, 0)
    w = p ** U[:, -1] * (1 - p) ** (N - U[:, -1])
    return math.fsum(w * pay)


@pytest.mark.parametrize("payoff", PAYOFFS)
def test_enumeration_matches_numpy(oracle, payoff):
    for N, u, p in ((1, 1.1, 0.4), (5, 1.07, 0.55), (10, 1.03, 0.47)):
        o = _explicit(N, 100.0, 101.5, u, p, payoff)
        ref = _numpy_enumeration(N, 100.0, 101.5, u, 1.0 / u, p, payoff)
        assert oracle.price_exhaustive(o, 1) == pytest.approx(ref, rel=1e-13, abs=1e-13)


def test_spmd_partition_sums_to_total(oracle):
    """eq. f14/f15: the rank-prefix partials add up to the full sum for any M."""
    o = W.opt(12, 100.0, 100.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL)
    full = oracle.price_exhaustive(o, 1)
    for M in (2, 4, 8):
        assert oracle.price_exhaustive(o, M) == pytest.approx(full, rel=1e-14)
    n = 1 << 12
    parts = [oracle.sum_range(o, r * n // 4, (r + 1) * n // 4) for r in range(4)]
    assert oracle.discount(o) * math.fsum(parts) == pytest.approx(full, rel=1e-14)


# --------------------------------------------------------------------------
# Philox-4x32-10 and the Monte Carlo estimators (Section 4)
# --------------------------------------------------------------------------
_TRITON_PHILOX = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
@triton.jit
def k(out, cptr, seed):
    c0 = tl.load(cptr + 0).to(tl.uint32, bitcast=True)
    c1 = tl.load(cptr + 1).to(tl.uint32, bitcast=True)
    c2 = tl.load(cptr + 2).to(tl.uint32, bitcast=True)
    c3 = tl.load(cptr + 3).to(tl.uint32, bitcast=True)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out + 0, a.to(tl.int32, bitcast=True)); tl.store(out + 1, b.to(tl.int32, bitcast=True))
    tl.store(out + 2, c.to(tl.int32, bitcast=True)); tl.store(out + 3, d.to(tl.int32, bitcast=True))
res = []
for (c, key) in json.loads(sys.argv[1]):
    out = torch.zeros(4, dtype=torch.int32)
    seed = key[0] | (key[1] << 32)
    ct = torch.tensor([v if v < 2**31 else v - 2**32 for v in c], dtype=torch.int32)
    k[(1,)](out, ct, seed)
    res.append([v & 0xffffffff for v in out.tolist()])
print(json.dumps(res))
"""


def test_philox_matches_independent_implementation(oracle):
    """Triton ships its own Philox-4x32-10; its CPU interpreter is an
    implementation independent of the oracle's."""
    pytest.importorskip("triton")
    cases = [([0, 0, 0, 0], [0, 0]), ([1, 2, 3, 4], [5, 6]),
             ([0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff], [0xffffffff, 0xffffffff]),
             ([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0]),
             ([17, 123456, 4095, 63], [0x9e3779b9, 7])]
    r = subprocess.run([sys.executable, "-c", _TRITON_PHILOX, json.dumps(cases)], capture_output=True,
                       text=True, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
    ref = json.loads(r.stdout.strip().splitlines()[-1])
    for (c, key), want in zip(cases, ref):
        assert oracle.philox(c, key) == want


def test_bernoulli_threshold(oracle):
    assert oracle.bernoulli_threshold(0.5) == 2 ** 31
    assert oracle.bernoulli_threshold(1e-12) == 1
    assert oracle.bernoulli_threshold(1 - 1e-12) == 2 ** 32 - 1


def test_mc_all_strata_is_exact(oracle):
    """With 2^N strata every stratum is one path: the Partitioned estimator
    is the exact sum (Section 4, the M = 2^N case)."""
    for pay in (W.ASIAN_ARITH_CALL, W.LOOKBACK_FIXED_PUT, W.ASIAN_GEO_PUT):
        o = W.opt(9, 100.0, 100.0, 0.05, 0.3, 1.0, pay)
        th, var = oracle.mc(o, 9, 3, seed=11)
        assert th * oracle.discount(o) == pytest.approx(oracle.price_exhaustive(o, 1), rel=1e-13)
        assert var == 0.0


def test_mc_bit_frequency(oracle):
    """Stratum 0 of an N-step tree with mb=0 and p far from 1/2: the ups of the
    drawn paths follow Binomial(N, p)."""
    o = _explicit(1, 100.0, 0.0, 1.1, 0.3, W.EURO_CALL)
    # one step, zero strike: V = S1, so theta = p u S0 + (1-p) d S0 in expectation
    th, var = oracle.mc(o, 0, 20000, seed=3)
    pd = (th / 100.0 - 1 / 1.1) / (1.1 - 1 / 1.1)   # estimated p
    assert abs(pd - 0.3) < 4 * math.sqrt(0.3 * 0.7 / 20000)


def test_mc_unbiased_and_variance_formula(oracle):
    """Mean over independent seeds within 4 SE of the exact value, and the
    spread across seeds matches sum_m P(D_m)^2 Var[V|D_m] / R_m (eq. mc13's
    first line) computed exactly."""
    o = W.opt(10, 100.0, 100.0, 0.05, 0.3, 1.0, W.ASIAN_ARITH_CALL)
    exact = oracle.price_exhaustive(o, 1) / oracle.discount(o)
    mb, Rm, reps = 3, 16, 300
    mean, var, prob = oracle.stratum_moments(o, mb)
    var_exact = float(np.sum(prob ** 2 * var / Rm))
    assert math.fsum(prob * mean) == pytest.approx(exact, rel=1e-13)
    ths = np.array([oracle.mc(o, mb, Rm, seed=1000 + s)[0] for s in range(reps)])
    assert abs(ths.mean() - exact) < 4 * math.sqrt(var_exact / reps)
    ratio = ths.var(ddof=1) / var_exact
    lo, hi = stats.chi2.ppf([1e-4, 1 - 1e-4], reps - 1) / (reps - 1)
    assert lo < ratio < hi


def test_law_of_total_variance(oracle):
    """eq. mc14: Var[V] = sum_m Var[V|D_m] P(D_m) + Var_D E[V|D]."""
    o = W.opt(11, 100.0, 98.0, 0.05, 0.35, 1.0, W.ASIAN_ARITH_PUT)
    m0, v0, _ = oracle.stratum_moments(o, 0)
    mean, var, prob = oracle.stratum_moments(o, 4)
    theta = math.fsum(prob * mean)
    rhs = math.fsum(prob * var) + math.fsum(prob * (mean - theta) ** 2)
    assert v0[0] == pytest.approx(rhs, rel=1e-12)
    assert m0[0] == pytest.approx(theta, rel=1e-13)


def test_theorem1_variance_ordering(oracle):
    """Theorem 1 with R_m = R: Var(partitioned) <= Var(shared) <= Var(basic),
    checked on the empirical spread over seeds (Asian put, as in Table 5)."""
    o = W.opt(10, 100.0, 100.0, 0.05, 0.4, 1.0, W.ASIAN_ARITH_PUT)
    mb, R, reps = 3, 32, 250
    part = np.array([oracle.mc(o, mb, R, seed=5000 + s)[0] for s in range(reps)])
    shar = np.array([oracle.mc(o, mb, R, seed=5000 + s, shared=True)[0] for s in range(reps)])
    basic = np.array([oracle.mc(o, 0, R, seed=5000 + s)[0] for s in range(reps)])
    assert part.var() < shar.var() < basic.var()
    exact = oracle.price_exhaustive(o, 1) / oracle.discount(o)
    assert abs(shar.mean() - exact) < 4 * shar.std() / math.sqrt(reps)


# --------------------------------------------------------------------------
# Pathwise Greeks (CRR)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("payoff", [W.ASIAN_ARITH_CALL, W.LOOKBACK_FIXED_CALL, W.ASIAN_GEO_PUT, W.EURO_PUT])
def test_greeks_match_central_differences(oracle, payoff):
    base = dict(N=10, S0=101.0, K=99.3, rate=0.04, sigma=0.27, T=1.1)
    o = W.opt(payoff=payoff, **base)
    v, g = oracle.greeks_crr(o)
    assert v == pytest.approx(oracle.price_exhaustive(o, 1), rel=1e-13)
    for i, key in enumerate(("S0", "sigma", "rate", "K")):
        h = 1e-6 * abs(base[key])
        up = W.opt(payoff=payoff, **dict(base, **{key: base[key] + h}))
        dn = W.opt(payoff=payoff, **dict(base, **{key: base[key] - h}))
        fd = (oracle.price_exhaustive(up, 1) - oracle.price_exhaustive(dn, 1)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-7), key


def test_greeks_euler_identity(oracle):
    """V is homogeneous of degree one in (S0, K): S0 dV/dS0 + K dV/dK = V."""
    for pay in (W.ASIAN_ARITH_PUT, W.LOOKBACK_FIXED_CALL, W.ASIAN_GEO_CALL):
        o = W.opt(12, 96.0, 104.0, 0.05, 0.3, 0.7, pay)
        v, g = oracle.greeks_crr(o)
        assert 96.0 * g[0] + 104.0 * g[3] == pytest.approx(v, rel=1e-12)


# ---------------------------------------------------------------------------
# Time-varying trees (eq. f13 with per-step u_t, d_t, p_t)
# ---------------------------------------------------------------------------
def _numpy_steps(o, steps):
    """Independent brute force: every path at once with numpy."""
    N = o["N"]
    b = np.arange(1 << N, dtype=np.int64)
    x = ((b[:, None] >> (N - 1 - np.arange(N))[None, :]) & 1).astype(bool)
    u, d, p = steps[:, 0], steps[:, 1], steps[:, 2]
    S = o["S0"] * np.cumprod(np.where(x, u, d), axis=1)
    w = np.prod(np.where(x, p, 1.0 - p), axis=1)
    pay = o["payoff"]
    X = {0: S[:, -1], 1: S[:, -1], 2: S.mean(axis=1), 3: S.mean(axis=1),
         4: np.exp(np.log(S).mean(axis=1)), 5: np.exp(np.log(S).mean(axis=1)),
         6: S.max(axis=1), 7: S.min(axis=1)}[pay]
    v = np.maximum(X - o["K"], 0.0) if pay % 2 == 0 else np.maximum(o["K"] - X, 0.0)
    return math.exp(-o["rate"] * o["T"]) * math.fsum(w * v)


@pytest.mark.parametrize("payoff", range(8))
def test_steps_constant_factors_match_the_lattice_oracle(oracle, payoff):
    """Constant u, d, p reduce the time-varying walk to the recombining tree."""
    for kind in (W.TREE_CRR, W.TREE_SEYDEL):
        o = W.opt(12, 100.0, 98.0, 0.05, 0.3, 1.0, payoff, kind)
        u, d, p = oracle.tree(kind, 12, 0.3, 0.05, 1.0)
        steps = np.tile([u, d, p], (12, 1))
        assert oracle.steps_price(o, steps, 4) == pytest.approx(oracle.price_exhaustive(o, 4), rel=1e-13, abs=1e-13)


@pytest.mark.parametrize("payoff", range(8))
def test_steps_match_numpy_brute_force(oracle, payoff):
    steps = W.step_factors(3, 11)
    o = W.opt(11, 100.0, 101.0, 0.04, 0.2, 1.0, payoff)
    assert oracle.steps_price(o, steps, 4) == pytest.approx(_numpy_steps(o, steps), rel=1e-13, abs=1e-13)


def test_steps_zero_strike_closed_forms(oracle):
    """With K = 0 the calls are plain expectations of products of independent
    steps: E[S_N] = S0 prod g_t, E[A] = (S0/N) sum_t prod_{i<=t} g_i with
    g_i = p_i u_i + (1 - p_i) d_i, and E[G] = S0 prod_i E[m_i^{(N-i+1)/N}]."""
    N = 14
    steps = W.step_factors(5, N)
    u, d, p = steps[:, 0], steps[:, 1], steps[:, 2]
    g = p * u + (1 - p) * d
    disc = math.exp(-0.03 * 1.5)
    c = (N - np.arange(N)) / N
    closed = {W.EURO_CALL: 100.0 * np.prod(g),
              W.ASIAN_ARITH_CALL: 100.0 / N * np.sum(np.cumprod(g)),
              W.ASIAN_GEO_CALL: 100.0 * np.prod(p * u ** c + (1 - p) * d ** c)}
    for pay, v in closed.items():
        o = W.opt(N, 100.0, 0.0, 0.03, 0.2, 1.5, pay)
        assert oracle.steps_price(o, steps, 4) == pytest.approx(disc * v, rel=1e-13)


def test_steps_put_call_parity_and_weights(oracle):
    N = 13
    steps = W.step_factors(9, N)
    u, d, p = steps[:, 0], steps[:, 1], steps[:, 2]
    g = p * u + (1 - p) * d
    disc = math.exp(-0.05)
    EA = 100.0 / N * np.sum(np.cumprod(g))
    c = oracle.steps_price(W.opt(N, 100.0, 97.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL), steps, 4)
    q = oracle.steps_price(W.opt(N, 100.0, 97.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_PUT), steps, 4)
    assert c - q == pytest.approx(disc * (EA - 97.0), rel=1e-12)
    o = W.opt(N, 100.0, 97.0, 0.05, 0.2, 1.0, W.EURO_CALL)
    assert math.fsum(oracle.steps_path_prob(o, steps, b) for b in range(1 << N)) == pytest.approx(1.0, abs=1e-14)


# ---------------------------------------------------------------------------
# b-ary trees (the end of Section 3: trinomial and wider trees)
# ---------------------------------------------------------------------------
def _numpy_branch(o, moves, b):
    N = o["N"]
    idx = np.arange(b ** N, dtype=np.int64)
    x = (idx[:, None] // (b ** (N - 1 - np.arange(N)))[None, :]) % b
    f = moves[:, :b][np.arange(N)[None, :], x]
    q = moves[:, b:][np.arange(N)[None, :], x]
    S = o["S0"] * np.cumprod(f, axis=1)
    w = np.prod(q, axis=1)
    pay = o["payoff"]
    X = {0: S[:, -1], 1: S[:, -1], 2: S.mean(axis=1), 3: S.mean(axis=1),
         4: np.exp(np.log(S).mean(axis=1)), 5: np.exp(np.log(S).mean(axis=1)),
         6: S.max(axis=1), 7: S.min(axis=1)}[pay]
    v = np.maximum(X - o["K"], 0.0) if pay % 2 == 0 else np.maximum(o["K"] - X, 0.0)
    return math.exp(-o["rate"] * o["T"]) * math.fsum(w * v)


@pytest.mark.parametrize("payoff", range(8))
def test_branch_trinomial_matches_numpy_brute_force(oracle, payoff):
    moves = W.branch_moves(11, 8, 3)
    o = W.opt(8, 100.0, 101.0, 0.03, 0.2, 1.0, payoff)
    assert oracle.branch_price(o, moves, 3, 4) == pytest.approx(_numpy_branch(o, moves, 3), rel=1e-13, abs=1e-13)


@pytest.mark.parametrize("payoff", range(8))
def test_branch_binary_and_zero_middle_reduce_to_the_binomial_walk(oracle, payoff):
    N = 11
    steps = W.step_factors(21, N)
    o = W.opt(N, 100.0, 99.0, 0.04, 0.2, 1.0, payoff)
    ref = oracle.steps_price(o, steps, 4)
    u, d, p = steps[:, 0], steps[:, 1], steps[:, 2]
    two = np.stack([d, u, 1 - p, p], axis=1)                       # digit 1 = up
    assert oracle.branch_price(o, two, 2, 4) == pytest.approx(ref, rel=1e-13, abs=1e-13)
    three = np.stack([d, np.sqrt(u * d), u, 1 - p, np.zeros(N), p], axis=1)
    assert oracle.branch_price(o, three, 3, 4) == pytest.approx(ref, rel=1e-13, abs=1e-13)


def test_branch_european_on_a_recombining_trinomial_lattice(oracle):
    """Constant moves (1/u, 1, u): the path sum equals backward induction."""
    N, u = 12, math.exp(0.3 * math.sqrt(3 * 1.0 / 12))
    q = [0.2, 0.5, 0.3]
    moves = np.tile([1 / u, 1.0, u] + q, (N, 1))
    for pay in (W.EURO_CALL, W.EURO_PUT):
        o = W.opt(N, 100.0, 103.0, 0.05, 0.3, 1.0, pay)
        assert oracle.branch_price(o, moves, 3, 4) == pytest.approx(
            oracle.branch_european_backward(o, moves, 3), rel=1e-12)


def test_branch_zero_strike_closed_forms(oracle):
    N = 9
    moves = W.branch_moves(5, N, 3)
    g = np.sum(moves[:, :3] * moves[:, 3:], axis=1)
    disc = math.exp(-0.02)
    for pay, v in ((W.EURO_CALL, 100.0 * np.prod(g)), (W.ASIAN_ARITH_CALL, 100.0 / N * np.sum(np.cumprod(g)))):
        o = W.opt(N, 100.0, 0.0, 0.02, 0.2, 1.0, pay)
        assert oracle.branch_price(o, moves, 3, 4) == pytest.approx(disc * v, rel=1e-13)


def test_mc_single_stratum_matches_the_full_run(oracle):
    """orc_mc_stratum reproduces orc_mc's per-stratum statistics exactly."""
    o = W.opt(40, 100.0, 100.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL)
    th, var, mean, sv, pr = oracle.mc(o, 5, 300, 17, 0, False, True)
    for z in (0, 7, 31):
        mz, vz, pz = oracle.mc_stratum(o, 5, z, 300, 17)
        assert (mz, vz, pz) == (mean[z], sv[z], pr[z])


def test_paper_table5_variances_loosely(oracle, golden_dir):
    """Table 5 as a loose pin: one run of the Partitioned and Shared-Sample
    estimators (R = R_m = 1024, Asian put, N=32, Seydel) has its estimate
    within 4 standard errors of the exact 82.115 and its variance estimate
    within a factor of two of the paper's 1000-repetition average."""
    g = json.load(open(os.path.join(golden_dir, "paper_table5_mc.json")))
    c = g["common"]
    o = W.opt(c["N"], c["S0"], c["K"], c["rate"], c["sigma"], c["T"], W.ASIAN_ARITH_PUT, W.TREE_SEYDEL)
    disc2 = math.exp(-2 * c["rate"] * c["T"])
    disc = math.sqrt(disc2)
    for i, M in enumerate(g["M"]):
        if M not in (1, 8, 64):
            continue
        mb = M.bit_length() - 1
        for kind, shared in (("partitioned", False), ("shared", True)):
            th, var = oracle.mc(o, mb, c["R"], 1000 + M, 0, shared)
            v, se2 = disc * th, disc2 * var
            assert abs(v - 82.115) <= 4 * math.sqrt(se2), (kind, M, v, se2)
            ref = g[kind]["var"][i]
            assert 0.5 * ref <= se2 <= 2.0 * ref, (kind, M, se2, ref)


# ---------------------------------------------------------------------------
# Several payoffs per enumeration, and payoffs given as functions of the path
# ---------------------------------------------------------------------------
ALL_PAYOFF_STRIKES = [(pay, K) for pay in range(8) for K in (92.0, 106.0)]


def test_steps_multi_matches_numpy_brute_force(oracle):
    """Every payoff and two strikes from one walk of the time-varying tree,
    each against the independent numpy enumeration."""
    N = 11
    steps = W.step_factors(31, N)
    o = W.opt(N, 100.0, 100.0, 0.04, 0.2, 1.3, W.EURO_CALL)
    got = oracle.steps_price_multi(o, steps, ALL_PAYOFF_STRIKES, 4)
    for (pay, K), g in zip(ALL_PAYOFF_STRIKES, got):
        ref = _numpy_steps(dict(o, payoff=pay, K=K), steps)
        assert g == pytest.approx(ref, rel=1e-13, abs=1e-13), (pay, K)


@pytest.mark.parametrize("b,N", [(3, 8), (4, 6)])
def test_branch_multi_matches_numpy_brute_force(oracle, b, N):
    moves = W.branch_moves(40 + b, N, b)
    o = W.opt(N, 100.0, 100.0, 0.03, 0.2, 1.0, W.EURO_CALL)
    got = oracle.branch_price_multi(o, moves, b, ALL_PAYOFF_STRIKES, 3)
    for (pay, K), g in zip(ALL_PAYOFF_STRIKES, got):
        ref = _numpy_branch(dict(o, payoff=pay, K=K), moves, b)
        assert g == pytest.approx(ref, rel=1e-13, abs=1e-13), (b, pay, K)


def test_multi_partition_does_not_change_the_sum(oracle):
    """The rank partition (1, 2, 4, 8 workers) changes only the rounding order."""
    N = 14
    steps = W.step_factors(12, N)
    o = W.opt(N, 100.0, 100.0, 0.04, 0.2, 1.0, W.EURO_CALL)
    ref = oracle.steps_price_multi(o, steps, ALL_PAYOFF_STRIKES, 1)
    for M in (2, 4, 8):
        assert np.allclose(oracle.steps_price_multi(o, steps, ALL_PAYOFF_STRIKES, M), ref, rtol=1e-14, atol=1e-14)


def test_functional_constant_and_end_price_closed_forms(oracle):
    """V = 1 sums the path probabilities (to e^{-qT}); V = S_N gives
    e^{-qT} S0 prod_t g_t with g_t = sum_k f_tk q_tk (independent steps)."""
    for b, N, moves in ((2, 10, oracle.steps_as_moves(W.step_factors(6, 10))), (3, 7, W.branch_moves(8, 7, 3))):
        o = W.opt(N, 100.0, 0.0, 0.05, 0.2, 1.2, W.EURO_CALL)
        disc = math.exp(-0.05 * 1.2)
        one = oracle.functional_price(o, moves, b, lambda S, x: np.ones(len(S)))
        assert one == pytest.approx(disc, rel=1e-14)
        g = np.sum(moves[:, :b] * moves[:, b:], axis=1)
        end = oracle.functional_price(o, moves, b, lambda S, x: S[:, -1])
        assert end == pytest.approx(disc * 100.0 * np.prod(g), rel=1e-13)


def test_functional_digits_and_prices_agree(oracle):
    """The digits handed to the payoff are the path index's base-b digits
    (first step most significant) and the prices their running products."""
    b, N = 3, 5
    moves = W.branch_moves(9, N, b)
    seen = []

    def V(S, x):
        seen.append((S.copy(), x.copy()))
        return np.zeros(len(S))
    oracle.functional_price(W.opt(N, 100.0, 0.0, 0.0, 0.2, 1.0, W.EURO_CALL), moves, b, V)
    S = np.concatenate([s for s, _ in seen])
    x = np.concatenate([d for _, d in seen])
    idx = np.arange(b ** N)
    want = (idx[:, None] // (b ** (N - 1 - np.arange(N)))[None, :]) % b
    assert np.array_equal(x, want)
    f = moves[:, :b][np.arange(N)[None, :], want]
    assert np.allclose(S, 100.0 * np.cumprod(f, axis=1), rtol=1e-15)


@pytest.mark.parametrize("payoff", [W.ASIAN_ARITH_CALL, W.LOOKBACK_FIXED_PUT, W.ASIAN_GEO_PUT, W.EURO_CALL])
def test_functional_restated_payoffs_match_numpy_brute_force(oracle, payoff):
    """Built-in payoffs written as path functions agree with the independent
    numpy enumeration (and so with the walk oracle)."""
    N, K = 12, 101.0
    steps = W.step_factors(17, N)
    o = W.opt(N, 100.0, K, 0.04, 0.2, 1.0, payoff)
    V = {W.ASIAN_ARITH_CALL: lambda S, x: np.maximum(S.mean(axis=1) - K, 0.0),
         W.LOOKBACK_FIXED_PUT: lambda S, x: np.maximum(K - S.min(axis=1), 0.0),
         W.ASIAN_GEO_PUT: lambda S, x: np.maximum(K - np.exp(np.log(S).mean(axis=1)), 0.0),
         W.EURO_CALL: lambda S, x: np.maximum(S[:, -1] - K, 0.0)}[payoff]
    got = oracle.functional_price(o, oracle.steps_as_moves(steps), 2, V)
    assert got == pytest.approx(_numpy_steps(o, steps), rel=1e-13, abs=1e-13)


def test_functional_barrier_against_numpy_brute_force(oracle):
    """A path-dependent payoff outside the built-ins: an up-and-out call."""
    N, K, B = 12, 98.0, 112.0
    steps = W.step_factors(23, N)
    o = W.opt(N, 100.0, K, 0.04, 0.3, 1.0, W.EURO_CALL)
    got = oracle.functional_price(o, oracle.steps_as_moves(steps), 2,
                                  lambda S, x: np.where(S.max(axis=1) >= B, 0.0, np.maximum(S[:, -1] - K, 0.0)))
    bb = np.arange(1 << N, dtype=np.int64)
    xx = ((bb[:, None] >> (N - 1 - np.arange(N))[None, :]) & 1).astype(bool)
    S = 100.0 * np.cumprod(np.where(xx, steps[:, 0], steps[:, 1]), axis=1)
    w = np.prod(np.where(xx, steps[:, 2], 1.0 - steps[:, 2]), axis=1)
    v = np.where(S.max(axis=1) >= B, 0.0, np.maximum(S[:, -1] - K, 0.0))
    assert got == pytest.approx(math.exp(-0.04) * math.fsum(w * v), rel=1e-13)
