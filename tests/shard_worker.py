"""One rank of a sharded pricing run, for the multi-process tests.

Usage: python tests/shard_worker.py RANK WORLD PORT OUT.json MODE PROVIDER FAIL
  MODE      exact | mc | bench (bench.py's split step: the exchange and the
            rank-order combination of the exact mode's per-option partials)
  PROVIDER  oracle (this rank's part from the CPU oracle) | gpu (from this
            rank's GPU through the C ABI)
  FAIL      none | die (exit before the exchange) | nan (return NaN partials)
Ranks meet over gloo at 127.0.0.1:PORT. Writes {"value": [...], ...} or
{"error": "..."} to OUT.json.
"""
import datetime
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1701_03512_gb300 import workloads as W  # noqa: E402

# several work items per pass at N >= 23 (2^(N-22) items), one below
EXACT_OPTS = [W.opt(N, 100.0, K, 0.05, 0.25, 1.0, pay) for N, K, pay in
              ((16, 95.0, W.ASIAN_ARITH_CALL), (23, 100.0, W.ASIAN_ARITH_PUT), (24, 105.0, W.ASIAN_GEO_CALL),
               (25, 98.0, W.LOOKBACK_FIXED_CALL), (26, 102.0, W.ASIAN_ARITH_CALL), (24, 99.0, W.EURO_PUT))]
MC_OPT = W.opt(48, 100.0, 100.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL)
MC_BITS, MC_R, MC_SEED = 4, 512, 7


def exact_items(o):
    """Work items of the exhaustive pass (FP32_COMP), as the library splits
    them (bt_exact_split, host only): item i covers the path indices
    [i ppi 2^L, (i+1) ppi 2^L), prefix bits first."""
    from paper_1701_03512_gb300 import build as b
    b.build()
    from paper_1701_03512_gb300 import btree as bt
    sp = bt.bt_exact_split(o, bt.BT_PREC_FP32_COMP)
    span = sp["prefixes_per_item"] << sp["L"]
    return [(i * span, min((i + 1) * span, 1 << o["N"])) for i in range(sp["n_items"])]


def oracle_exact_part(rank, world):
    """Items are numbered across the whole batch (option after option: the
    batch has no call/put pair with equal parameters, which would share one
    pass); rank r takes the items whose number is r modulo world."""
    from oracle import py_oracle as O
    out, base = [], 0
    for o in EXACT_OPTS:
        items = exact_items(o)
        s = sum(O.sum_range(o, lo, hi) for i, (lo, hi) in enumerate(items) if (base + i) % world == rank)
        base += len(items)
        out.append(O.discount(o) * s)
    return np.array(out)


def oracle_mc_part(rank, world):
    from oracle import py_oracle as O
    _, _, mean, sv, pr = O.mc(MC_OPT, MC_BITS, MC_R, MC_SEED, 0, False, True)
    disc = O.discount(MC_OPT)
    m = np.arange(1 << MC_BITS) % world == rank
    value = disc * np.sum(pr[m] * mean[m])
    var = disc ** 2 * np.sum(pr[m] ** 2 * sv[m] / MC_R)
    return np.array([[value, var, float(m.sum() * MC_R)]])


def main():
    rank, world, port = int(sys.argv[1]), int(sys.argv[2]), int(sys.argv[3])
    out_path, mode, provider, fail = sys.argv[4], sys.argv[5], sys.argv[6], sys.argv[7]
    import torch.distributed as dist
    from paper_1701_03512_gb300 import sharded as S

    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=datetime.timedelta(seconds=30))
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=30))
    ex = S.Exchange(rank, world, store, timeout_s=3.0)
    ctx = None
    if provider == "gpu":
        from paper_1701_03512_gb300 import btree as bt
        ctx = bt.Context(0)
    if fail == "die":
        os._exit(3)   # leaves between steps, nothing in flight
    res = {}
    try:
        # a failing rank does its share of the work first and then returns NaN, so that it reaches
        # the exchange no earlier than its peers (a peer still computing past the exchange's
        # time limit would be reported missing instead)
        if mode == "bench":
            import bench
            part = oracle_exact_part(rank, world)
            if fail == "nan":
                part = np.full_like(part, np.nan)
            res["value"] = bench.split_combine(ex, part).tolist()
        elif mode == "exact":
            local = oracle_exact_part if provider == "oracle" else None
            if fail == "nan":
                local = lambda r, w: np.full_like(oracle_exact_part(r, w), np.nan)  # noqa: E731
            v = S.price_exact_sharded(ex, EXACT_OPTS, 1, ctx.h if ctx else None, local)
            res["value"] = v.tolist()
        else:
            local = oracle_mc_part if provider == "oracle" else None
            if fail == "nan":
                local = lambda r, w: np.full_like(oracle_mc_part(r, w), np.nan)  # noqa: E731
            v, se, n = S.price_mc_sharded(ex, [MC_OPT], MC_BITS, MC_R, MC_SEED, ctx.h if ctx else None, local)
            res.update(value=v.tolist(), stderr=se.tolist(), samples=n.tolist())
    except S.ShardError as e:
        res["error"] = str(e)
    with open(out_path, "w") as f:
        json.dump(res, f)
    if ctx:
        ctx.close()
    os._exit(0)   # skip process-group teardown, which would wait for a dead peer


if __name__ == "__main__":
    main()
