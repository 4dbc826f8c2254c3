"""Sharded pricing across processes (gloo on the CPU): the per-rank parts
come from the oracle, so this checks the split, the exchange, the fixed-order
combination and the failure detection without a GPU."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
WORKER = os.path.join(HERE, "shard_worker.py")
sys.path.insert(0, HERE)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def run_ranks(tmp_path, world, mode, providers, fails=None, timeout=90):
    port = free_port()
    fails = fails or ["none"] * world
    procs, outs = [], []
    for r in range(world):
        out = str(tmp_path / ("rank%d.json" % r))
        outs.append(out)
        env = dict(os.environ, CUDA_VISIBLE_DEVICES=os.environ.get("CUDA_VISIBLE_DEVICES", "0"))
        procs.append(subprocess.Popen([sys.executable, WORKER, str(r), str(world), str(port), out, mode,
                                       providers[r], fails[r]], env=env))
    codes = [p.wait(timeout=timeout) for p in procs]
    res = [json.load(open(o)) if os.path.exists(o) else None for o in outs]
    return codes, res


@pytest.mark.parametrize("world", [2, 3])
def test_exact_shards_sum_to_the_oracle_value(tmp_path, oracle, world):
    import shard_worker as SW
    codes, res = run_ranks(tmp_path, world, "exact", ["oracle"] * world)
    assert codes == [0] * world
    ref = np.array([oracle.exact(o) for o in SW.EXACT_OPTS])
    for r in res:
        assert np.allclose(r["value"], ref, rtol=1e-13, atol=1e-14)
    assert all(r["value"] == res[0]["value"] for r in res)   # every rank returns the same numbers


@pytest.mark.parametrize("world", [2, 3])
def test_bench_split_step_sums_to_the_oracle_value(tmp_path, oracle, world):
    """bench.py's multi-GPU step (every rank runs its share of the work items
    of one batch, then one all-gather of the per-option partials combined in
    rank order): the exchange and combination path with oracle parts."""
    import shard_worker as SW
    codes, res = run_ranks(tmp_path, world, "bench", ["oracle"] * world)
    assert codes == [0] * world
    ref = np.array([oracle.exact(o) for o in SW.EXACT_OPTS])
    for r in res:
        assert np.allclose(r["value"], ref, rtol=1e-13, atol=1e-14)
    assert all(r["value"] == res[0]["value"] for r in res)


def test_bench_split_step_names_a_nan_rank(tmp_path):
    codes, res = run_ranks(tmp_path, 2, "bench", ["oracle", "oracle"], ["none", "nan"])
    assert codes == [0, 0]
    for r in res:
        assert "error" in r and "ranks [1]" in r["error"], r


def test_mc_strata_shards_sum_to_the_full_estimate(tmp_path, oracle):
    import shard_worker as SW
    codes, res = run_ranks(tmp_path, 2, "mc", ["oracle", "oracle"])
    assert codes == [0, 0]
    th, var = oracle.mc(SW.MC_OPT, SW.MC_BITS, SW.MC_R, SW.MC_SEED)
    disc = oracle.discount(SW.MC_OPT)
    for r in res:
        assert abs(r["value"][0] - disc * th) <= 1e-13 * abs(disc * th)
        assert abs(r["stderr"][0] - disc * np.sqrt(var)) <= 1e-12 * disc * np.sqrt(var)
        assert r["samples"][0] == (1 << SW.MC_BITS) * SW.MC_R


def test_missing_rank_is_reported_not_hung(tmp_path):
    codes, res = run_ranks(tmp_path, 2, "exact", ["oracle", "oracle"], ["none", "die"], timeout=60)
    assert codes[1] == 3 and codes[0] == 0
    assert "error" in res[0] and "[1]" in res[0]["error"], res[0]


def test_nan_partials_are_reported_with_the_rank(tmp_path):
    codes, res = run_ranks(tmp_path, 2, "mc", ["oracle", "oracle"], ["none", "nan"])
    assert codes == [0, 0]
    for r in res:
        assert "error" in r and "ranks [1]" in r["error"] and "non-finite" in r["error"], r


def test_combine_is_fixed_order_and_compensated():
    from paper_1701_03512_gb300 import sharded as S
    parts = np.array([[1e16, 1.0], [1.0, 2.0], [-1e16, 3.0]])
    assert S.combine(parts).tolist() == [1.0, 6.0]
    assert S.neumaier([0.1] * 10) == 1.0
