"""The allocation-free pricing entry point against the regular one.

bt_price_exact_noalloc serves callers that cannot allocate device memory
while they run (an application whose allocator owns the device, or a loop
that cannot afford cudaMalloc/cudaFree). It keeps every intermediate buffer
in one fixed library-owned device array, so these checks call it three
times in a row with different batches -- a later call must not see an
earlier call's leftovers -- and compare each result with bt_price_exact
through the C ABI bit for bit (same plan, split and kernels), and the last
batch with the oracle within the tolerances the other exhaustive-sum tests
use.
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
def test_noalloc_matches_regular_entry_point_twice(bt, oracle, prec):
    """Both entry points run the same plan, split and kernels, so their
    results must be the same bits; the second call must not see the first
    call's leftovers in the shared array. The small batch is also checked
    against the oracle at the contract tolerance."""
    batch_a = W.batch(26, W.option_sets(41, 4), list(range(8)))          # 32 options, pairs and singles
    batch_b = W.random_options(42, 20, 16, 28)                              # different shapes
    batch_c = W.random_options(45, 12, 8, 18)                               # small enough for the oracle
    ctx = bt.Context(0)
    try:
        refs = [ctx.price_exact(b, prec) for b in (batch_a, batch_b, batch_c)]
    finally:
        ctx.close()
    for batch, ref in zip((batch_a, batch_b, batch_c), refs):   # three calls in a row
        got = _noalloc(bt, batch, prec)
        assert np.array_equal(got["value"], ref["value"]), (prec, got["value"] - ref["value"])
        assert np.array_equal(got["err_est"], ref["err_est"])
        assert np.array_equal(got["paths"], ref["paths"])
    exact = np.array([oracle.exact(o) for o in batch_c])
    s0 = np.array([o["S0"] for o in batch_c])
    assert np.all(np.abs(got["value"] - exact) <= _tol(prec, 18) * np.abs(exact) + 1e-12 * s0)


def test_noalloc_rejects_oversized_batches(bt):
    too_many = W.random_options(43, bt.BT_NOALLOC_MAX_OPTIONS + 1, 10, 12)
    with pytest.raises(bt.BtError) as e:
        bt.bt_price_exact_noalloc(too_many)
    assert e.value.status == bt.BT_EUNSUPPORTED
    too_big = W.batch(40, W.option_sets(44, 8), (W.ASIAN_ARITH_CALL,))
    with pytest.raises(bt.BtError) as e:
        bt.bt_price_exact_noalloc(too_big)
    assert e.value.status == bt.BT_EUNSUPPORTED and "bytes" in str(e.value)
