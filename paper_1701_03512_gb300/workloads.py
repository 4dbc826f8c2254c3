"""Seeded synthetic inputs shared by the tests, the bench and the oracle callers.

This module only draws parameters. It holds none of the pricing arithmetic
(no tree parameters, no weights, no payoffs): the CUDA path and the CPU
oracle each derive everything else from these plain numbers on their own.

Recipes (all numbers are synthetic; the paper uses no dataset):

* ``single_asian_n20`` -- one arithmetic-average Asian call, N=20, S0=100,
  K=100, rate=0.05, sigma=0.2, T=1, CRR tree.
* ``option_sets(seed, n)`` -- ``n`` parameter sets drawn with
  ``numpy.random.default_rng(seed)`` as whole n-vectors in the order
  S0~U[80,120], K~U[80,120], sigma~U[0.1,0.5], rate~U[0,0.08], T~U[0.25,2].
  Seed 0 / n=64 is the batched exhaustive workload, seed 1 / n=256 the
  Greeks workload.
* ``paper_mc_workload`` -- the parameters of the paper's Monte Carlo study
  (Section 5: K=100, S=20, q=6%, sigma=3.0, T=1, N=32, Seydel tree).
* ``paper_runtime_workload`` -- the put of the paper's runtime tables
  (Section 5: K=10, S=5, sigma=0.30, q=6%, T=1).
* ``serving_stream(seed, n, rate_per_s)`` -- a Poisson request stream:
  exponential inter-arrival gaps, N~U{16..34}, payoff uniform over
  {arith Asian call, arith Asian put, geometric Asian call, fixed-strike
  lookback call}, parameters drawn as in ``option_sets``.
"""
from __future__ import annotations

import numpy as np

# Payoff codes; the numbering matches the public C header (an interface both
# sides must agree on, nothing more).
EURO_CALL = 0
EURO_PUT = 1
ASIAN_ARITH_CALL = 2
ASIAN_ARITH_PUT = 3
ASIAN_GEO_CALL = 4
ASIAN_GEO_PUT = 5
LOOKBACK_FIXED_CALL = 6
LOOKBACK_FIXED_PUT = 7

PAYOFF_NAMES = {
    EURO_CALL: "euro_call", EURO_PUT: "euro_put",
    ASIAN_ARITH_CALL: "asian_arith_call", ASIAN_ARITH_PUT: "asian_arith_put",
    ASIAN_GEO_CALL: "asian_geo_call", ASIAN_GEO_PUT: "asian_geo_put",
    LOOKBACK_FIXED_CALL: "lookback_fixed_call", LOOKBACK_FIXED_PUT: "lookback_fixed_put",
}

TREE_CRR = 0
TREE_SEYDEL = 1
TREE_EXPLICIT = 2


def opt(N, S0, K, rate, sigma, T, payoff, tree=TREE_CRR, u=0.0, d=0.0, p=0.0):
    """One option as a plain dict (the field names of the C struct)."""
    return dict(N=int(N), tree_kind=int(tree), payoff=int(payoff), S0=float(S0), K=float(K),
                rate=float(rate), sigma=float(sigma), T=float(T), u=float(u), d=float(d), p=float(p))


def single_asian_n20():
    return opt(20, 100.0, 100.0, 0.05, 0.2, 1.0, ASIAN_ARITH_CALL)


def option_sets(seed: int, n: int):
    """``n`` parameter sets as a dict of float64 arrays (see module doc)."""
    rng = np.random.default_rng(seed)
    S0 = rng.uniform(80.0, 120.0, n)
    K = rng.uniform(80.0, 120.0, n)
    sigma = rng.uniform(0.1, 0.5, n)
    rate = rng.uniform(0.0, 0.08, n)
    T = rng.uniform(0.25, 2.0, n)
    return dict(S0=S0, K=K, sigma=sigma, rate=rate, T=T)


def batch(N: int, sets: dict, payoffs, tree=TREE_CRR):
    """Cartesian product: every set priced under every payoff, set-major."""
    out = []
    n = len(sets["S0"])
    for i in range(n):
        for pay in payoffs:
            out.append(opt(N, sets["S0"][i], sets["K"][i], sets["rate"][i], sets["sigma"][i],
                           sets["T"][i], pay, tree))
    return out


def batched_exact_workload(N: int, seed: int = 0, n: int = 64):
    """The batched exhaustive workload: arith Asian call and put per set."""
    return batch(N, option_sets(seed, n), (ASIAN_ARITH_CALL, ASIAN_ARITH_PUT))


def greeks_workload(N: int = 28, seed: int = 1, n: int = 256):
    """The Greeks workload: arith Asian call and fixed-strike lookback call."""
    return batch(N, option_sets(seed, n), (ASIAN_ARITH_CALL, LOOKBACK_FIXED_CALL))


def paper_mc_workload(payoff=ASIAN_ARITH_PUT, N=32):
    return opt(N, 20.0, 100.0, 0.06, 3.0, 1.0, payoff, TREE_SEYDEL)


def paper_runtime_workload(N=24, payoff=EURO_PUT):
    return opt(N, 5.0, 10.0, 0.06, 0.30, 1.0, payoff, TREE_CRR)


def random_options(seed: int, n: int, N_lo: int, N_hi: int, payoffs=tuple(range(8)),
                   trees=(TREE_CRR, TREE_SEYDEL)):
    """Mixed small problems for parity sweeps: N~U{N_lo..N_hi}, random payoff and tree."""
    rng = np.random.default_rng(seed)
    sets = option_sets(seed + 1000, n)
    Ns = rng.integers(N_lo, N_hi + 1, n)
    pays = rng.choice(np.asarray(payoffs), n)
    tr = rng.choice(np.asarray(trees), n)
    return [opt(Ns[i], sets["S0"][i], sets["K"][i], sets["rate"][i], sets["sigma"][i], sets["T"][i],
                pays[i], tr[i]) for i in range(n)]


SERVING_PAYOFFS = (ASIAN_ARITH_CALL, ASIAN_ARITH_PUT, ASIAN_GEO_CALL, LOOKBACK_FIXED_CALL)


def serving_stream(seed: int = 2, n: int = 10000, rate_per_s: float = 1000.0, N_lo=16, N_hi=34):
    """Poisson arrivals: returns (arrival_s[n], options[n])."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, n)
    arrivals = np.cumsum(gaps) - gaps[0]
    Ns = rng.integers(N_lo, N_hi + 1, n)
    pays = rng.choice(np.asarray(SERVING_PAYOFFS), n)
    sets = option_sets(seed + 1, n)
    opts = [opt(Ns[i], sets["S0"][i], sets["K"][i], sets["rate"][i], sets["sigma"][i], sets["T"][i],
                pays[i]) for i in range(n)]
    return arrivals, opts


def step_factors(seed: int, N: int, lo: float = 0.02, hi: float = 0.15, p_lo: float = 0.3, p_hi: float = 0.7):
    """Per-step moves and probabilities for a time-varying tree: steps[N][3] =
    (u_t, d_t, p_t) with ln u_t ~ U[lo, hi], ln d_t ~ -U[lo, hi] (drawn
    independently, so the tree does not recombine) and p_t ~ U[p_lo, p_hi]."""
    rng = np.random.default_rng(seed)
    lu = rng.uniform(lo, hi, N)
    ld = rng.uniform(lo, hi, N)
    p = rng.uniform(p_lo, p_hi, N)
    return np.stack([np.exp(lu), np.exp(-ld), p], axis=1)


def branch_moves(seed: int, N: int, b: int = 3, lo: float = 0.02, hi: float = 0.12, conc: float = 2.0):
    """Per-step moves of a b-ary tree: moves[N][2b] = (factors of digits
    0..b-1, ascending, then their probabilities). Factors: exp of sorted
    draws from U[-hi, hi] with the smallest below -lo and the largest above
    lo; probabilities: a Dirichlet(conc,...,conc) draw (conc = 2 spreads
    them widely; a large conc keeps them near 1/b)."""
    rng = np.random.default_rng(seed)
    out = np.zeros((N, 2 * b))
    for t in range(N):
        z = np.sort(rng.uniform(-hi, hi, b))
        z[0] = min(z[0], -lo)
        z[-1] = max(z[-1], lo)
        out[t, :b] = np.exp(z)
        out[t, b:] = rng.dirichlet(np.full(b, float(conc)))
    return out
