"""Sharded pricing with the GPU owning one part: rank 0 prices its work items
(or strata) on the GPU through the C ABI, rank 1 computes its part with the
CPU oracle, and the combined result must equal the full one."""
import os
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

from test_sharded import run_ranks  # noqa: E402


def test_exact_gpu_rank_plus_oracle_rank(tmp_path, oracle):
    import shard_worker as SW
    codes, res = run_ranks(tmp_path, 2, "exact", ["gpu", "oracle"], timeout=300)
    assert codes == [0, 0], res
    ref = np.array([oracle.exact(o) for o in SW.EXACT_OPTS])
    s0 = np.array([o["S0"] for o in SW.EXACT_OPTS])
    for r in res:
        assert np.all(np.abs(np.array(r["value"]) - ref) <= 1e-9 * np.abs(ref) + 1e-12 * s0), (r, ref)
    assert res[0]["value"] == res[1]["value"]


def test_mc_gpu_rank_plus_oracle_rank(tmp_path):
    import shard_worker as SW
    from paper_1701_03512_gb300 import btree as bt
    codes, res = run_ranks(tmp_path, 2, "mc", ["gpu", "oracle"], timeout=300)
    assert codes == [0, 0], res
    ctx = bt.Context(0)
    try:
        full = bt.bt_price_mc(ctx.h, [SW.MC_OPT], SW.MC_BITS, SW.MC_R, SW.MC_SEED)[0]
    finally:
        ctx.close()
    # the same Philox draws on both sides; the GPU's path sums are FP32
    assert abs(res[0]["value"][0] - full["value"]) <= 1e-5 * abs(full["value"])
    assert abs(res[0]["stderr"][0] - full["stderr_mc"]) <= 1e-4 * full["stderr_mc"]
