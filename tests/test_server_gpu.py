"""The continuous-batching server: results, overlap, admission, bounded waits."""
import time

import numpy as np
import pytest

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
    c = bt.Context(0, device_budget_bytes=16 << 30)
    yield c
    c.close()


def _stream(n, seed, N_lo=16, N_hi=28):
    _, opts = W.serving_stream(seed, n, 1000.0, N_lo, N_hi)
    return opts


def test_results_identical_alone_and_in_the_mix(bt, ctx):
    """Each request's result is bit-identical to pricing it alone."""
    opts = _stream(60, 5)
    srv = bt.bt_server_start(ctx.h, max_active=32, n_streams=3, max_items_per_launch=300)
    try:
        tickets = [bt.bt_submit(srv, o) for o in opts]
        got = [bt.bt_wait(srv, t, 120000) for t in tickets]
    finally:
        bt.bt_server_stop(srv)
    for o, g in zip(opts, got):
        alone = bt.bt_price_exact(ctx.h, [o])[0]
        assert g["value"] == alone["value"] and g["paths"] == alone["paths"]


def test_late_arrivals_overlap_a_running_request(bt, ctx):
    """A large request is on the GPU; small requests submitted after it are
    admitted and finish while it is still running."""
    big = W.opt(38, 100.0, 100.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL)
    small = _stream(16, 6, 16, 20)
    srv = bt.bt_server_start(ctx.h, max_active=64, n_streams=3, max_items_per_launch=256)
    try:
        tb = bt.bt_submit(srv, big)
        time.sleep(0.0005)
        ts = [bt.bt_submit(srv, o) for o in small]
        res = [bt.bt_wait(srv, t, 60000) for t in ts]
        assert bt.bt_poll(srv, tb) is None, "small requests should finish while the large one runs"
        rb = bt.bt_wait(srv, tb, 120000)
        st = bt.bt_server_stats(srv)
    finally:
        bt.bt_server_stop(srv)
    assert rb["paths"] == 2 ** 38 and st["completed"] == 17 and st["launches"] > 2
    for o, r in zip(small, res):
        assert r["value"] == bt.bt_price_exact(ctx.h, [o])[0]["value"]


def test_admission_by_memory(bt, ctx):
    """A pool that holds only a few requests' partials at a time still
    completes every request, admitting as memory frees up."""
    opts = [W.opt(38, 100.0, 90.0 + 2 * i, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL) for i in range(8)]
    # N = 38 (13 suffix steps, 25 prefix steps): 2^15 work items x 16 B of
    # partials = 512 KiB per request, plus 2^12 + 2^13 prefix entries x 32 B
    # and the 65 KiB suffix table: about 0.94 MiB; the pool holds two
    budget = (2 << 20) + (512 << 10)
    srv = bt.bt_server_start(ctx.h, max_active=64, n_streams=2, device_budget_bytes=budget)
    try:
        tickets = [bt.bt_submit(srv, o) for o in opts]
        got = [bt.bt_wait(srv, t, 120000) for t in tickets]
        st = bt.bt_server_stats(srv)
    finally:
        bt.bt_server_stop(srv)
    assert st["pool_bytes"] < budget
    assert 1 <= st["peak_active"] <= 2, st
    assert st["completed"] == len(opts)
    for o, g in zip(opts, got):
        assert g["value"] == bt.bt_price_exact(ctx.h, [o])[0]["value"]


def test_wait_is_bounded(bt, ctx):
    big = W.opt(34, 100.0, 100.0, 0.05, 0.2, 1.0, W.LOOKBACK_FIXED_CALL)
    srv = bt.bt_server_start(ctx.h)
    try:
        t = bt.bt_submit(srv, big)
        with pytest.raises(bt.BtError) as e:
            bt.bt_wait(srv, t, 0)
        assert e.value.status == bt.BT_ETIMEOUT
        r = bt.bt_wait(srv, t, 120000)
        assert r["paths"] == 2 ** 34
        with pytest.raises(bt.BtError):
            bt.bt_wait(srv, t, 10)   # collected already
    finally:
        bt.bt_server_stop(srv)


def test_replay_plain_and_batched_agree(bt, ctx):
    arrivals, opts = W.serving_stream(8, 200, 2000.0, 16, 30)
    rp, lp, wp = bt.bt_serve_replay(ctx.h, opts, arrivals, 0)
    rb, lb, wb = bt.bt_serve_replay(ctx.h, opts, arrivals, 1, max_active=256, n_streams=3)
    assert np.array_equal(rp["value"], rb["value"])
    assert np.all(lp > 0) and np.all(lb > 0)
    print("plain p50 %.2f p99 %.2f ms | batched p50 %.2f p99 %.2f ms" % (
        np.percentile(lp, 50), np.percentile(lp, 99), np.percentile(lb, 50), np.percentile(lb, 99)))


def test_submit_rejects_bad_options(bt, ctx):
    srv = bt.bt_server_start(ctx.h)
    try:
        with pytest.raises(bt.BtError) as e:
            bt.bt_submit(srv, dict(W.single_asian_n20(), S0=-1.0))
        assert e.value.status == bt.BT_EINVAL
    finally:
        bt.bt_server_stop(srv)


def test_mixed_precisions_in_one_server(bt, ctx):
    """FP64 and FP32 requests interleaved: each result is bit-identical to
    pricing it alone at its own precision."""
    opts = _stream(40, 9, 14, 26)
    precs = [bt.BT_PREC_FP64 if i % 3 == 0 else bt.BT_PREC_FP32_COMP for i in range(len(opts))]
    srv = bt.bt_server_start(ctx.h, max_active=16, n_streams=3, max_items_per_launch=200)
    try:
        tickets = [bt.bt_submit(srv, o, p) for o, p in zip(opts, precs)]
        got = [bt.bt_wait(srv, t, 120000) for t in tickets]
    finally:
        bt.bt_server_stop(srv)
    for o, p, g in zip(opts, precs, got):
        assert g["value"] == bt.bt_price_exact(ctx.h, [o], p)[0]["value"], (o, p)
    with pytest.raises(bt.BtError):
        srv2 = bt.bt_server_start(ctx.h)
        try:
            bt.bt_submit(srv2, opts[0], 7)
        finally:
            bt.bt_server_stop(srv2)
