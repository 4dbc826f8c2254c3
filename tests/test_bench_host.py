"""Host-side pieces of bench.py, without a GPU: the class-pass work count
and the compact summary that closes the bench line."""
import importlib.util
import os

import pytest

from paper_1701_03512_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def bt():
    from paper_1701_03512_gb300 import build as b
    b.build()
    from paper_1701_03512_gb300 import btree
    return btree


def test_class_evaluations_count_the_distinct_classes(bench, bt):
    """At N=36 the split keeps 13 suffix steps: 2^23 prefixes times 14
    (European), 62 (lookback) and 378 (geometric) recombined classes; the
    arithmetic Asian below 2^28 paths has one class per suffix."""
    base = dict(N=36, S0=100.0, K=100.0, rate=0.05, sigma=0.2, T=1.0)
    for pay, classes in ((W.EURO_PUT, 14), (W.LOOKBACK_FIXED_CALL, 62), (W.ASIAN_GEO_CALL, 378)):
        o = W.opt(base["N"], base["S0"], base["K"], base["rate"], base["sigma"], base["T"], pay)
        assert bench.class_evaluations(bt, o) == 2.0 ** 23 * classes
    o = W.opt(24, 100.0, 100.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL)
    sp = bt.bt_exact_split(o, bt.BT_PREC_FP32_COMP)
    assert bench.class_evaluations(bt, o) == 2.0 ** 24 and sp["P"] + sp["L"] == 24


def test_summary_holds_every_part(bench):
    line = {"value": 1.0e13, "scaling": "strong", "n_gpus": 1, "roofline": {"frac": 0.8}, "e2e": {"value": 9.9e12},
            "serving": {"capacity_rps": {"plain": 3000.0, "batched": 7000.0}, "identical_values": True,
                        "loads": [{"load_vs_plain_capacity": 0.8,
                                   "plain": {"p50_ms": 1.4, "p99_ms": 9.8},
                                   "batched": {"p50_ms": 0.45, "p99_ms": 4.9}}]},
            "mc": {"samples_per_s": 7.6e9, "frac_of_issue_peak": 0.63},
            "greeks": {"ms": 25.0, "frac_of_issue_peak": 0.68},
            "widened": {"steps": {"payoff_paths_per_s": 9.5e12, "frac_of_issue_peak": 0.71}}}
    s = bench.summary(line)
    assert s["exact_n36_paths_per_s"] == 1.0e13 and s["exact_n36_frac_of_issue_peak"] == 0.8
    assert s["serving_p50_p99_ms"]["0.80"]["batched"] == [0.45, 4.9]
    assert s["mc_frac_of_issue_peak"] == 0.63 and s["greeks_n28_ms"] == 25.0
    assert s["steps_frac_of_issue_peak"] == 0.71 and s["class_pass_n36_frac_of_issue_peak"] is None
    assert bench.summary({"value": 1.0, "scaling": "weak", "n_gpus": 2})["n_gpus"] == 2
