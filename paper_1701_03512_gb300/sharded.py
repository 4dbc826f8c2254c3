"""One pricing problem split across processes, one GPU each.

The exhaustive sum over 2^N paths and the Partitioned Monte Carlo estimator
both split into independent parts (Section 3: each process takes a block of
the rank bits; Section 4: the strata are those blocks):

  * exact: rank r runs the work items i with i % world == r, items numbered
    across the whole batch (each item is a block of 2^10 prefixes times all
    suffixes of one pass), the round-robin assignment of Section 3, and
    returns per option its discounted partial value;
  * Monte Carlo: rank r runs the strata m with m % world == r and returns
    per option its term of eq. mc12 and its term of the variance.

One exchange per call gathers the per-option partials (a few doubles per
option) from every rank, and every rank combines them in rank order with
Neumaier's compensated sum, so all ranks return the same numbers.

Failure detection is on the host. Before the exchange every rank marks
itself ready in a key-value store and waits, with a time limit, for the
others: a rank that died or never joined is named in a ShardError instead of
hanging the collective. Partials that are not finite are named with the rank
that produced them. No GPU kernel waits on another rank.
"""
from __future__ import annotations

import datetime
import itertools
from typing import Callable, Optional, Sequence

import numpy as np

from . import btree as bt


class ShardError(RuntimeError):
    """A rank is missing or returned unusable partials."""


def neumaier(xs: Sequence[float]) -> float:
    """Compensated sum in the given order."""
    s = 0.0
    c = 0.0
    for x in xs:
        x = float(x)
        t = s + x
        if abs(s) >= abs(x):
            c += (s - t) + x
        else:
            c += (x - t) + s
        s = t
    return s + c


def combine(parts: np.ndarray) -> np.ndarray:
    """parts[world, n]: per-rank partials in rank order -> per-option sums."""
    parts = np.asarray(parts, dtype=np.float64)
    return np.array([neumaier(parts[:, i]) for i in range(parts.shape[1])])


class Exchange:
    """Readiness check in a store, then an all-gather of float64 arrays."""

    _calls = itertools.count()

    def __init__(self, rank: int, world: int, store, timeout_s: float = 60.0, group=None):
        self.rank, self.world, self.store, self.group = rank, world, store, group
        self.timeout = datetime.timedelta(seconds=timeout_s)

    def gather(self, local: np.ndarray, tag: str) -> np.ndarray:
        import torch
        import torch.distributed as dist

        call = "%s/%d" % (tag, next(Exchange._calls))
        self.store.set("%s/ready/%d" % (call, self.rank), "1")
        keys = ["%s/ready/%d" % (call, r) for r in range(self.world)]
        try:
            self.store.wait(keys, self.timeout)
        except Exception as e:  # store timeout: name who is missing
            missing = [r for r, k in enumerate(keys) if not self.store.check([k])]
            raise ShardError("ranks %s did not reach '%s' within %.0f s (%s)"
                             % (missing, call, self.timeout.total_seconds(), type(e).__name__)) from e
        local = np.ascontiguousarray(local, dtype=np.float64)
        dev = "cuda" if dist.get_backend(self.group) == "nccl" else "cpu"
        t = torch.from_numpy(local).to(dev)
        out = [torch.empty_like(t) for _ in range(self.world)]
        dist.all_gather(out, t, group=self.group)
        allp = np.stack([o.cpu().numpy() for o in out])
        bad = [r for r in range(self.world) if not np.all(np.isfinite(allp[r]))]
        if bad:
            raise ShardError("ranks %s returned non-finite partials for '%s'" % (bad, call))
        return allp


# ---------------------------------------------------------------------------
# Local parts on this rank's GPU
# ---------------------------------------------------------------------------
def exact_local(ctx_h, opts, prec: int, rank: int, world: int, stream=None) -> np.ndarray:
    """This rank's discounted partial values, one per option."""
    plan = bt.bt_exact_plan_create(ctx_h, opts, prec)
    try:
        bt.bt_exact_plan_run_shard(plan, rank, world, stream)
        return bt.bt_exact_plan_read(plan, stream)["value"].astype(np.float64)
    finally:
        bt.bt_exact_plan_destroy(plan)


def mc_local(ctx_h, opts, strata_bits: int, samples_per_stratum: int, seed: int, rank: int, world: int,
             stream=None) -> np.ndarray:
    """This rank's (value term, variance term, samples) per option."""
    r = bt.bt_price_mc_shard(ctx_h, opts, strata_bits, samples_per_stratum, seed, rank, world, stream=stream)
    return np.stack([r["value"], r["stderr_mc"] ** 2, r["paths"].astype(np.float64)], axis=1)


# ---------------------------------------------------------------------------
# Sharded calls
# ---------------------------------------------------------------------------
def price_exact_sharded(ex: Exchange, opts, prec: int = bt.BT_PREC_FP32_COMP, ctx_h=None,
                        local: Optional[Callable[[int, int], np.ndarray]] = None) -> np.ndarray:
    """V for every option, summed over all ranks' work items. `local(rank,
    world)` overrides how this rank computes its part (default: its GPU)."""
    part = local(ex.rank, ex.world) if local else exact_local(ctx_h, opts, prec, ex.rank, ex.world)
    allp = ex.gather(np.asarray(part, dtype=np.float64).reshape(len(opts)), "exact")
    return combine(allp)


def price_mc_sharded(ex: Exchange, opts, strata_bits: int, samples_per_stratum: int, seed: int, ctx_h=None,
                     local: Optional[Callable[[int, int], np.ndarray]] = None):
    """(value, stderr, samples) per option of the Partitioned estimator with
    its strata split across ranks (2^strata_bits >= world)."""
    if (1 << strata_bits) < ex.world:
        raise ValueError("%d strata cannot be split across %d ranks" % (1 << strata_bits, ex.world))
    part = local(ex.rank, ex.world) if local else mc_local(ctx_h, opts, strata_bits, samples_per_stratum, seed,
                                                           ex.rank, ex.world)
    allp = ex.gather(np.asarray(part, dtype=np.float64).reshape(len(opts), 3), "mc")
    value = combine(allp[:, :, 0])
    stderr = np.sqrt(combine(allp[:, :, 1]))
    samples = allp[:, :, 2].sum(axis=0)
    return value, stderr, samples
