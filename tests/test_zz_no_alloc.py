"""The allocation-free pricing entry point against the regular one.

bt_price_exact_noalloc serves callers that cannot allocate device memory
while they run (an application whose allocator owns the device, or a loop
that cannot afford cudaMalloc/cudaFree). It keeps every intermediate buffer
in one fixed library-owned device array, so these checks call it twice in a
row with different batches -- the second call must not see the first call's
leftovers -- and compare each result with bt_price_exact through the C ABI,
within the tolerances the other exhaustive-sum tests use.
"""
import ctypes

import numpy as np
import pytest

from paper_1701_03512_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _tol(prec, N):
    return 1e-12 if prec == 0 else 1e-9


@pytest.fixture(scope="module")
def bt():
    from paper_1701_03512_gb300 import build as b
    b.build()
    from paper_1701_03512_gb300 import btree
    return btree


def _noalloc(bt, opts, prec):
    a = bt.options_array(opts)
    out = np.zeros(len(a), dtype=bt.RESULT_DTYPE)
    st = bt.lib().bt_price_exact_noalloc(ctypes.c_void_p(a.ctypes.data), len(a), prec,
                                         ctypes.c_void_p(out.ctypes.data), None)
    assert st == bt.BT_OK, bt.lib().bt_last_error(None).decode()
    return out


@pytest.mark.parametrize("prec", [1, 0])
def test_noalloc_matches_regular_entry_point_twice(bt, prec):
    batch_a = W.batch(26, W.option_sets(41, 4), list(range(8)))          # 32 options, pairs and singles
    batch_b = W.random_options(42, 20, 16, 28)                              # different shapes
    ctx = bt.Context(0)
    try:
        ref_a = ctx.price_exact(batch_a, prec)
        ref_b = ctx.price_exact(batch_b, prec)
    finally:
        ctx.close()
    for batch, ref in ((batch_a, ref_a), (batch_b, ref_b)):   # two calls in a row
        got = _noalloc(bt, batch, prec)
        tol = np.array([_tol(prec, o["N"]) for o in batch])
        s0 = np.array([o["S0"] for o in batch])
        err = np.abs(got["value"] - ref["value"])
        assert np.all(err <= tol * np.abs(ref["value"]) + 1e-12 * s0), (prec, err)
        assert np.array_equal(got["paths"], ref["paths"])


def test_noalloc_rejects_oversized_batches(bt):
    too_many = W.random_options(43, bt.BT_NOALLOC_MAX_OPTIONS + 1, 10, 12)
    with pytest.raises(bt.BtError) as e:
        bt.bt_price_exact_noalloc(too_many)
    assert e.value.status == bt.BT_EUNSUPPORTED
    too_big = W.batch(40, W.option_sets(44, 8), (W.ASIAN_ARITH_CALL,))
    with pytest.raises(bt.BtError) as e:
        bt.bt_price_exact_noalloc(too_big)
    assert e.value.status == bt.BT_EUNSUPPORTED and "bytes" in str(e.value)
