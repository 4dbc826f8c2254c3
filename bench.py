#!/usr/bin/env python
"""Benchmark of the exhaustive expected value over all 2^N Bernoulli paths.

Workload (one step): the batched exhaustive pass at N=36 -- 64 option sets
drawn from numpy default_rng(0) (S0, K ~ U[80,120], sigma ~ U[0.1,0.5],
rate ~ U[0,0.08], T ~ U[0.25,2]), CRR trees, arithmetic-average Asian call
and put for each set: 128 option-payoffs, each summed over all 2^36 paths,
FP32 path arithmetic with compensation and FP64 reduction. A step runs every
step of the path on the device: tree parameters, suffix and prefix tables,
the path sums and the per-option reduction.

  value  -- payoff-paths per second (128 * 2^36 per step) with the option
            array already in device memory, CUDA events on the launching
            stream, L2 flushed (256 MiB write) between steps;
  e2e    -- the same through bt_price_exact with host arrays (plan creation,
            host-to-device copies, all kernels, device-to-host copy, sync);
  roofline -- the path-sum kernel against the FP32 issue peak
            (n_SM x 128 lanes x max SM clock), counting the algorithmic
            3 ops per payoff-path;
  cpu_baseline -- the CPU oracle (plain enumeration, all host cores) on a
            bounded sample of the same workload.

Two further measurements ride on the same line (rank 0, N=1 only):
  serving -- a Poisson stream of single-option requests (N ~ U{16..34},
            payoff from {arith call, arith put, geo call, lookback call},
            parameters as above, seed 2) replayed through the
            continuous-batching server and as plain one-call-per-request
            pricing; first both capacities (all requests at t=0), then
            p50/p99 latency and throughput at offered loads of 0.5/0.8/0.95
            x the plain capacity, with a check that both modes return
            bit-identical values;
  mc      -- Partitioned Monte Carlo, arithmetic Asian call, N=252,
            2^16 strata x 2^14 Philox samples: samples/s and steps/s against
            the integer/FP32 issue peak;
  greeks  -- the derivative pass over 512 N=28 options (value and four
            Greeks each), host arrays in and out;
  widened -- time-varying trees (FP32, N=32) and the generic FP64 path walk
            on binomial (N=28) and trinomial (N=17) trees.

Multi-GPU (torchrun): the paper's split of one problem (Section 3, eq. f14
and f15) -- every rank holds the same batch, runs the work items i with
i % world == rank (bt_exact_plan_run_shard), and one all-gather of the
per-option partial values (a few doubles per option) is combined in rank
order on every rank; the value is the batch's paths over the slowest rank's
step time (strong scaling). --weak instead prices an independent batch per
rank (seed = rank) with no exchange.

--impl reference times the CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact paths/s at N=36, % FP32 peak; batched-serving p50/p99 ms vs plain"
UNIT = "paths/s"
N_DEFAULT = 36
SETS_DEFAULT = 64
OPS_PER_PATH = 3            # algorithmic: FMA (affine), max(.,0), accumulate
OPS_EXECUTED_PAIR = 6.125   # inner-loop ops per call+put path pair (392 per 64 pairs)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=N_DEFAULT)
    ap.add_argument("--sets", type=int, default=SETS_DEFAULT)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=10000)
    ap.add_argument("--serving-loads", default="0.5,0.8,0.95")
    ap.add_argument("--no-mc", action="store_true")
    ap.add_argument("--no-greeks", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--only", default="",
                    help="comma-separated widened rows (e.g. steps,trinomial_affine): print only those as a JSON "
                         "object and exit (for profiling one kernel)")
    ap.add_argument("--weak", action="store_true",
                    help="N > 1: an independent batch per rank instead of one batch split across the ranks")
    ap.add_argument("--split", action="store_true",
                    help="the split step (shard run, partials read back, rank-order combination) also at N = 1")
    return ap.parse_args()


def workload_config(args, extra=None):
    c = {"workload": "batched exhaustive arithmetic-Asian call+put, N=%d, %d option sets (seed 0), CRR tree"
                     % (args.N, args.sets),
         "N": args.N, "option_sets": args.sets, "payoffs_per_set": 2, "paths_per_payoff": 2 ** args.N,
         "precision": "FP32_COMP (FP32 path math, FP32-pair folds, FP64 reduction)",
         "l2": "flushed between timed steps (256 MiB device write)"}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------------------
# CPU baseline: the oracle, as it stands, on the host cores
# ---------------------------------------------------------------------------
def cpu_oracle_sample(opts, seconds, threads):
    """Times the oracle's plain enumeration (eq. f14 partition over threads)
    on the first paths of the first call/put pair; returns (paths/s, sample)."""
    from oracle import py_oracle as O
    O.lib()
    n = 1 << 20
    pair = opts[:2]
    while True:
        t0 = time.perf_counter()
        for o in pair:
            O.sum_range_mt(o, 0, n, threads)
        dt = time.perf_counter() - t0
        if dt > seconds / 8 or n >= (1 << 34):
            break
        n *= 2
    reps = max(1, int(seconds / max(dt, 1e-3)))
    t0 = time.perf_counter()
    for _ in range(reps):
        for o in pair:
            O.sum_range_mt(o, 0, n, threads)
    dt = time.perf_counter() - t0
    paths = reps * len(pair) * n
    sample = "%d x %d paths (path indices [0, 2^%d)) of the set-0 call and put, %d threads" % (
        reps, n, n.bit_length() - 1, threads)
    cpu_oracle_sample.last_seconds = dt
    return paths / dt, sample


def _mc_oracle_strata(job):
    """Worker of the all-cores MC baseline: the oracle's draws for some strata."""
    o, mb, strata, R, seed = job
    from oracle import py_oracle as O
    for z in strata:
        O.mc_stratum(o, mb, z, R, seed)
    return len(strata) * R


def mc_oracle_all_cores(o, mb, R, seed, threads, strata_per_worker=4):
    """The oracle's Partitioned MC over all host cores: one spawned process per
    core, each drawing whole strata (the paper's strata-to-process mapping);
    returns (samples/s, sample description)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(threads, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_mc_oracle_strata, [(o, mb, [w], 4, seed) for w in range(threads)]))  # start, load
        jobs = [(o, mb, list(range(w * strata_per_worker, (w + 1) * strata_per_worker)), R, seed)
                for w in range(threads)]
        t0 = time.perf_counter()
        n = sum(ex.map(_mc_oracle_strata, jobs))
        dt = time.perf_counter() - t0
    return n / dt, "%d strata x %d samples (strata 0..%d of 2^%d), %d processes" % (
        threads * strata_per_worker, R, threads * strata_per_worker - 1, mb, threads)


def cpu_model():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part", "hardware")):
                v = ln.split(":", 1)[1].strip()
                return {"0xd4f": "Arm Neoverse-V2 (part 0xd4f)"}.get(v, v)
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def physical_gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
    return local_rank


# ---------------------------------------------------------------------------
# Roofline inputs
# ---------------------------------------------------------------------------
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def kernel_source_hash():
    """Hash of the code (comments and blank space removed) the path-sum
    kernel is built from, to tell whether the committed counters still apply."""
    import re
    h = hashlib.sha256()
    for f in ("exact.cu", "exact_common.cuh", "df.cuh", "bt_internal.h"):
        src = open(os.path.join(ROOT, "paper_1701_03512_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(N):
    """DRAM bytes per launch of the path-sum kernel from the committed ncu
    figures (profiles/k_exact32_batched_asian.json), if they were taken on
    the current kernel source; None otherwise."""
    try:
        vals = json.load(open(os.path.join(ROOT, "profiles", "k_exact32_batched_asian.json")))
    except (OSError, ValueError):
        return None
    if vals.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    v = vals.get("dram_bytes_per_launch_N%d" % N)
    return float(v) if isinstance(v, (int, float)) else None


# ---------------------------------------------------------------------------
# Serving: continuous batching vs plain pricing on one arrival stream
# ---------------------------------------------------------------------------
SERVING_CFG = dict(max_active=1024, n_streams=6, max_items_per_launch=4864, device_budget_bytes=8 << 30)


def _lat(lat):
    import numpy as np
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(np.mean(lat)), "max_ms": float(np.max(lat))}


def serving_bench(bt, W, ctx, n_req, loads):
    import numpy as np
    arr1, opts = W.serving_stream(2, n_req, 1.0)     # arrivals at rate 1/s; scaled per load
    paths = float(sum(2.0 ** o["N"] for o in opts))
    zero = np.zeros(n_req)
    bt.bt_serve_replay(ctx.h, opts[:64], zero[:64], 0)          # warm both paths
    bt.bt_serve_replay(ctx.h, opts[:64], zero[:64], 1, **SERVING_CFG)
    rp, _, wall_p = bt.bt_serve_replay(ctx.h, opts, zero, 0)
    rb, _, wall_b = bt.bt_serve_replay(ctx.h, opts, zero, 1, **SERVING_CFG)
    cap_p, cap_b = n_req / wall_p, n_req / wall_b
    out = {"workload": "Poisson stream of %d single-option requests, N~U{16..34}, payoff uniform over "
                       "{arith Asian call, arith Asian put, geometric Asian call, fixed-strike lookback call}, "
                       "parameters drawn as the batched sets (seed 2), FP32_COMP" % n_req,
           "server": dict(SERVING_CFG),
           "plain": "one synchronous bt_price_exact per request, arrival order, same GPU and precision",
           "capacity_rps": {"plain": cap_p, "batched": cap_b},
           "capacity_paths_per_s": {"plain": paths / wall_p, "batched": paths / wall_b},
           "identical_values": bool(np.array_equal(rp["value"], rb["value"])), "loads": []}
    for f in loads:
        lam = f * cap_p
        arr = arr1 / lam
        # three replays per mode, alternating; the median run by p99 is reported (a host-side stall
        # of the replaying process shows up as one run's outlier, in either mode), all p99s beside it
        runs = {"plain": [], "batched": []}
        for _ in range(3):
            rp, lp, wp = bt.bt_serve_replay(ctx.h, opts, arr, 0)
            rb, lb, wb = bt.bt_serve_replay(ctx.h, opts, arr, 1, **SERVING_CFG)
            out["identical_values"] &= bool(np.array_equal(rp["value"], rb["value"]))
            runs["plain"].append(dict(_lat(lp), throughput_rps=n_req / wp))
            runs["batched"].append(dict(_lat(lb), throughput_rps=n_req / wb))
        row = {"load_vs_plain_capacity": f, "arrival_rps": lam}
        for mode, rs in runs.items():
            rs = sorted(rs, key=lambda x: x["p99_ms"])
            row[mode] = dict(rs[1], p99_ms_runs=[x["p99_ms"] for x in runs[mode]])
        out["loads"].append(row)
    main = next((x for x in out["loads"] if abs(x["load_vs_plain_capacity"] - 0.8) < 1e-9), None)
    if main:
        out["at_0.8"] = {"p50_ms": {"plain": main["plain"]["p50_ms"], "batched": main["batched"]["p50_ms"]},
                         "p99_ms": {"plain": main["plain"]["p99_ms"], "batched": main["batched"]["p99_ms"]}}
    return out


# ---------------------------------------------------------------------------
# Monte Carlo: Partitioned estimator throughput
# ---------------------------------------------------------------------------
MC_OPS_PER_STEP = 14   # Philox-4x32-10 per 4 steps: 10 rounds x (2 wide multiplies + 2 three-input xors) = 40
                       # (the key schedule is the same for every thread); + compare, select, multiply, add
MC_IMAD_PER_STEP = 8    # integer multiplies per simulated step (see heavy_pipe_bound)
# Shared-Sample pair (prefix m, suffix i): FADD sign tau_m + sign f_i, FMNMX with 0, FFMA into the sum
# with the folded weight P(D_m) beta_m
SHARED_OPS_PER_PAIR = 3


def mc_bench(bt, W, ctx, sms, fmax, reps=3, with_cpu=True):
    import torch
    N, mb, R = 252, 16, 1 << 14
    o = W.opt(N, 100.0, 100.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL)
    stream = torch.cuda.Stream()
    bt.bt_price_mc(ctx.h, [o], mb, R, 1, stream)
    ts = []
    for i in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = bt.bt_price_mc(ctx.h, [o], mb, R, 2 + i, stream)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    t = statistics.median(ts)
    samples = float(R) * (1 << mb)
    steps = samples * (N - mb)
    # plain MC with the same total number of draws (eq. mc14 comparison)
    plain = bt.bt_price_mc(ctx.h, [o], 0, int(samples), 7, stream)[0]
    peak = sms * 128 * fmax * 1e6
    cpu = None
    if with_cpu:
        from oracle import py_oracle as O
        mb_c, R_c = 4, 256
        t0 = time.perf_counter()
        O.mc(o, mb_c, R_c, 1)
        dt = time.perf_counter() - t0
        cpu = {"samples_per_s": (1 << mb_c) * R_c / dt, "cores": 1, "kind": "oracle",
               "sample": "2^%d strata x %d samples of the same option, one thread" % (mb_c, R_c)}
        threads = cpu_threads()
        v_all, s_all = mc_oracle_all_cores(o, mb, R, 1, threads, strata_per_worker=32)
        cpu["all_cores"] = {"samples_per_s": v_all, "cores": threads, "kind": "oracle", "sample": s_all}
    # the Shared-Sample estimator (the Remark of Section 4): the same R suffixes under every one
    # of the 2^m prefixes, beside the Partitioned estimator with R suffixes per stratum
    shared = None
    try:
        osh = W.opt(64, 100.0, 100.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL)
        msh, rsh = 10, 1 << 24
        bt.bt_price_mc_ex(ctx.h, [osh], msh, rsh, 3, bt.BT_MC_SHARED, stream=stream)   # warm-up, same size
        times = []
        for rep in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rs = bt.bt_price_mc_ex(ctx.h, [osh], msh, rsh, 4, bt.BT_MC_SHARED, stream=stream)[0]
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        tsh = sorted(times)[1]   # median of three calls
        pairs = float(rsh) * (1 << msh)
        # Theorem 1 beside it: both estimators with R = 2^14 suffixes per prefix
        rvs = 1 << 14
        rshs = bt.bt_price_mc_ex(ctx.h, [osh], msh, rvs, 5, bt.BT_MC_SHARED, stream=stream)[0]
        rpart = bt.bt_price_mc_ex(ctx.h, [osh], msh, rvs, 5, bt.BT_MC_PARTITIONED, stream=stream)[0]
        shared = {"workload": "Shared-Sample MC, arithmetic Asian call, N=64, 2^%d prefixes x 2^%d shared suffixes"
                              % (msh, rsh.bit_length() - 1),
                  "ms": 1e3 * tsh, "suffixes_per_s": rsh / tsh, "prefix_suffix_pairs_per_s": pairs / tsh,
                  "ops_per_pair": SHARED_OPS_PER_PAIR,
                  "frac_of_issue_peak": SHARED_OPS_PER_PAIR * pairs / tsh / peak,
                  "value": float(rs["value"]), "stderr": float(rs["stderr_mc"]),
                  "same_R_2^14": {"shared": {"value": float(rshs["value"]), "stderr": float(rshs["stderr_mc"])},
                                  "partitioned": {"value": float(rpart["value"]),
                                                  "stderr": float(rpart["stderr_mc"])}}}
    except Exception as exc:  # keep the rest of the line if this extra entry fails
        shared = {"error": str(exc)}
    # the other stratifications of the MC workload: N = 64 and 252, m = 10, 12, 16
    sweep = []
    for Ns in (64, 252):
        os_ = W.opt(Ns, 100.0, 100.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL)
        for ms, Rs in ((10, 1 << 14), (12, 1 << 12), (16, 1 << 10)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rs = bt.bt_price_mc(ctx.h, [os_], ms, Rs, 20 + ms, stream)[0]
            e1.record(stream)
            e1.synchronize()
            ns = float(Rs) * (1 << ms)
            ps = bt.bt_price_mc(ctx.h, [os_], 0, int(ns), 40 + ms, stream)[0]
            sweep.append({"N": Ns, "m": ms, "R": Rs, "samples_per_s": ns / (e0.elapsed_time(e1) / 1e3),
                          "value": float(rs["value"]), "stderr": float(rs["stderr_mc"]),
                          "plain_stderr_same_draws": float(ps["stderr_mc"]),
                          "variance_ratio": float((ps["stderr_mc"] / rs["stderr_mc"]) ** 2)})
    return {"workload": "Partitioned MC, arithmetic Asian call, N=%d, S0=K=100, rate 0.05, sigma 0.2, T=1, "
                        "2^%d strata x %d samples" % (N, mb, R), "cpu_baseline": cpu, "strata_sweep": sweep,
            "shared_sample": shared,
            "samples_per_s": samples / t, "steps_per_s": steps / t, "ms": 1e3 * t,
            "value": float(r[0]["value"]), "stderr": float(r[0]["stderr_mc"]),
            "plain_mc_same_draws": {"value": float(plain["value"]), "stderr": float(plain["stderr_mc"]),
                                    "variance_ratio": float((plain["stderr_mc"] / r[0]["stderr_mc"]) ** 2)},
            "ops_per_step": MC_OPS_PER_STEP, "frac_of_issue_peak": MC_OPS_PER_STEP * steps / t / peak,
            # the unit that binds: integer multiplies run only on the FMA-heavy pipe (16 lanes per SM
            # sub-partition, 64 per SM); Philox-4x32-10 needs 2 products x (high, low) x 10 rounds per
            # 4 steps, 8 per step once the warp-uniform products of the first rounds are shared
            "heavy_pipe_bound": {"imad_per_step": MC_IMAD_PER_STEP,
                                 "peak_steps_per_s": sms * 64 * fmax * 1e6 / MC_IMAD_PER_STEP,
                                 "frac": steps / t / (sms * 64 * fmax * 1e6 / MC_IMAD_PER_STEP)}}


# ---------------------------------------------------------------------------
# Greeks: one derivative pass over the N=28 Greeks workload
# ---------------------------------------------------------------------------
def greeks_bench(bt, W, ctx, sms, fmax, reps=3, with_cpu=True):
    import numpy as np
    opts = W.greeks_workload(28, 1, 256)
    cpu = {}
    if with_cpu:
        from oracle import py_oracle as O
        oc = dict(opts[0], N=22)
        cpu = {"cpu_baseline": _oracle_rate(lambda: O.greeks_crr(oc), 2.0 ** 22,
                                            "value and four derivatives of set 0's arithmetic Asian call at "
                                            "N=22 (2^22 paths), one thread; unit payoff-paths/s")}
    bt.bt_greeks_exact(ctx.h, opts)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        val, grad = bt.bt_greeks_exact(ctx.h, opts)
        ts.append(time.perf_counter() - t0)
    t = statistics.median(ts)
    paths = float(len(opts)) * 2.0 ** 28
    return {"workload": "value and dV/d(S0, sigma, rate, K), 256 sets (seed 1) x {arithmetic Asian call, "
                        "fixed-strike lookback call}, N=28, FP32_COMP, host arrays in and out",
            "ms": 1e3 * t, "options_per_s": len(opts) / t, "payoff_paths_per_s": paths / t,
            # value (affine FMA, max, accumulate), in-the-money count, df/du accumulate
            "ops_per_payoff_path": 5, "frac_of_issue_peak": 5 * paths / t / (sms * 128 * fmax * 1e6),
            "finite": bool(np.all(np.isfinite(grad))), **cpu}


# ---------------------------------------------------------------------------
# Widened paths: time-varying trees, the generic pass (plug-ins, b-ary trees)
# ---------------------------------------------------------------------------
def _timed(fn, reps=3):
    fn()
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        ts.append(time.perf_counter() - t0)
    return statistics.median(ts)


def _oracle_rate(fn, units, sample):
    """One timed call of the oracle (one host thread) -> its rate in units/s."""
    t0 = time.perf_counter()
    fn()
    dt = time.perf_counter() - t0
    return {"value": units / dt, "cores": 1, "kind": "oracle", "sample": sample}


CLS_OPS_SINGLE = 22   # per (prefix, class): TwoSum tau + f (6), low parts (3), sign select (2),
                      # multiplicity x pair by TwoProd (3), TwoSum into the group sum (8)
CLS_OPS_PAIR = 35     # a call and a put: the 9 ops of tau + f shared, 13 each for select and accumulate


def class_evaluations(bt, o):
    """(prefix, class) evaluations of one option's class pass: 2^P prefixes
    times the distinct suffix classes of its split -- suffixes of one
    up-count with the same key (level sum, end level, max or min level); the
    arithmetic Asian's classes are its suffixes."""
    import numpy as np
    sp = bt.bt_exact_split(o, bt.BT_PREC_FP32_COMP)
    L, P = sp["L"], sp["P"]
    if o["payoff"] in (2, 3):
        return float(2 ** P) * float(2 ** L)
    s = np.arange(1 << L)
    bits = (s[:, None] >> (L - 1 - np.arange(L))[None, :]) & 1
    lvl = np.cumsum(2 * bits - 1, axis=1)
    key = {4: lvl.sum(axis=1), 5: lvl.sum(axis=1), 0: lvl[:, -1], 1: lvl[:, -1],
           6: lvl.max(axis=1), 7: lvl.min(axis=1)}[o["payoff"]]
    classes = len(set(zip(bits.sum(axis=1).tolist(), key.tolist())))
    return float(2 ** P) * classes


def extras_bench(bt, W, ctx, sms, fmax, with_cpu=True, only=None):
    """The widened rows, each timed with host arrays in and out; `only`
    (a set of row names) runs a subset."""
    import numpy as np
    peak = sms * 128 * fmax * 1e6
    if with_cpu:
        from oracle import py_oracle as O

    def steps_row():
        # time-varying trees, FP32: 8 trees at N=32, an arithmetic Asian call and put on each (a pair
        # shares one pass)
        N = 32
        opts, steps = [], []
        for i in range(8):
            st = W.step_factors(900 + i, N, 0.01, 0.05)
            for pay in (W.ASIAN_ARITH_CALL, W.ASIAN_ARITH_PUT):
                opts.append(W.opt(N, 100.0, 90.0 + 5 * (i % 4), 0.03, 0.2, 1.0, pay))
                steps.append(st)
        t = _timed(lambda: bt.bt_price_exact_steps(ctx.h, opts, steps, bt.BT_PREC_FP32_COMP))
        paths = len(opts) * 2.0 ** N
        r = {"workload": "time-varying trees (per-step u_t, d_t, p_t), 8 trees x arithmetic Asian call+put, "
                         "16 x 2^32 payoff-paths, FP32_COMP, host arrays in and out",
             "ms": 1e3 * t, "payoff_paths_per_s": paths / t, "ops_per_payoff_path": 3,
             "frac_of_issue_peak": 3 * paths / t / peak}
        if with_cpu:
            r["cpu_baseline"] = _oracle_rate(
                lambda: O.steps_sum_range(opts[0], steps[0], 0, 1 << 22), float(1 << 22),
                "paths [0, 2^22) of option 0 (arithmetic Asian call), one thread")
        return r

    def generic_binomial_row():
        N2 = 28
        o2 = [W.opt(N2, 100.0, 100.0, 0.05, 0.2, 1.0, pay) for pay in (W.ASIAN_ARITH_CALL, W.LOOKBACK_FIXED_CALL)]
        u, d, p = bt.bt_tree_params(o2[0])
        mv2 = [np.tile([d, u, 1 - p, p], (N2, 1))] * 2
        t = _timed(lambda: bt.bt_price_exact_branching(ctx.h, o2, 2, mv2))
        r = {"workload": "generic pass (FP64 path walk), arithmetic Asian and lookback calls, N=28, 2 x 2^28 paths",
             "ms": 1e3 * t, "payoff_paths_per_s": 2 * 2.0 ** N2 / t}
        if with_cpu:
            o2c = dict(o2[0], N=20)
            r["cpu_baseline"] = _oracle_rate(
                lambda: O.branch_price(o2c, np.tile([d, u, 1 - p, p], (20, 1)), 2, 1), 2.0 ** 20,
                "the arithmetic Asian call at N=20 (2^20 paths) through the b-ary enumeration, one thread")
        return r

    def trinomial_affine_row():
        # trinomial trees through the affine pass (prefix/suffix tables, FP32), N=22: 8 x 3^22 paths
        N4 = 22
        o4 = [W.opt(N4, 100.0, 90.0 + 5 * i, 0.03, 0.2, 1.0, pay)
              for i in range(4) for pay in (W.ASIAN_ARITH_CALL, W.ASIAN_ARITH_PUT)]
        mv4 = [W.branch_moves(800 + i // 2, N4, 3, 0.01, 0.05, 50.0) for i in range(len(o4))]
        t = _timed(lambda: bt.bt_price_exact_moves(ctx.h, o4, 3, mv4, bt.BT_PREC_FP32_COMP))
        paths4 = len(o4) * 3.0 ** N4
        r = {"workload": "4 trinomial trees (per-step moves, probabilities Dirichlet(50)) x arithmetic Asian "
                         "call+put, N=22, 8 x 3^22 payoff-paths, FP32_COMP, host arrays in and out",
             "ms": 1e3 * t, "payoff_paths_per_s": paths4 / t, "frac_of_issue_peak": 3 * paths4 / t / peak}
        if with_cpu:
            o4c = dict(o4[0], N=13)
            mv4c = W.branch_moves(800, 13, 3, 0.01, 0.05, 50.0)
            r["cpu_baseline"] = _oracle_rate(
                lambda: O.branch_price(o4c, mv4c, 3, 1), 3.0 ** 13,
                "the arithmetic Asian call on a trinomial tree at N=13 (3^13 paths), one thread")
        return r

    def generic_trinomial_row():
        N3 = 17
        o3 = [W.opt(N3, 100.0, 100.0, 0.05, 0.2, 1.0, pay) for pay in (W.ASIAN_ARITH_CALL, W.LOOKBACK_FIXED_CALL)]
        mv3 = [W.branch_moves(3, N3, 3), W.branch_moves(4, N3, 3)]
        t = _timed(lambda: bt.bt_price_exact_branching(ctx.h, o3, 3, mv3))
        r = {"workload": "generic pass, trinomial trees, arithmetic Asian and lookback calls, N=17, 2 x 3^17 paths",
             "ms": 1e3 * t, "payoff_paths_per_s": 2 * 3.0 ** N3 / t}
        if with_cpu:
            o3c = dict(o3[0], N=13)
            mv3c = W.branch_moves(3, 13, 3)
            r["cpu_baseline"] = _oracle_rate(
                lambda: O.branch_price(o3c, mv3c, 3, 1), 3.0 ** 13,
                "the arithmetic Asian call on a trinomial tree at N=13 (3^13 paths), one thread")
        return r

    def single_row():
        # the plain single-option case: arithmetic Asian call, N=20 (2^20 paths), FP64, one call with
        # host arrays (its parity against the oracle, <= 1e-12, is asserted by the tests)
        o1 = W.single_asian_n20()
        t1 = _timed(lambda: bt.bt_price_exact(ctx.h, [o1], bt.BT_PREC_FP64), reps=5)
        v1 = float(bt.bt_price_exact(ctx.h, [o1], bt.BT_PREC_FP64)[0]["value"])
        r = {"workload": "arithmetic Asian call, N=20, S0=K=100, rate 0.05, sigma 0.2, T=1, CRR, FP64, one option, "
                         "host arrays in and out", "ms": 1e3 * t1, "value": v1, "paths_per_s": 2.0 ** 20 / t1}
        if with_cpu:
            r["cpu_baseline"] = _oracle_rate(lambda: O.price_exhaustive(o1, 1), 2.0 ** 20,
                                             "the same option, all 2^20 paths, one thread")
        return r

    # The class pass evaluates each (prefix, suffix class) once in FP32 pairs, a class standing for
    # its multiplicity of paths (a regrouping of eq. f14's sum): its work is counted in
    # (prefix, class) evaluations, CLS_OPS_SINGLE counted FP32 ops each (CLS_OPS_PAIR for a
    # call/put pair sharing tau + f); payoff-paths/s is the equivalent count.
    def class_row():
        # recombined classes (geometric, lookback, European) at N=36
        oc = W.batch(36, W.option_sets(0, 64), (W.ASIAN_GEO_CALL, W.LOOKBACK_FIXED_CALL, W.EURO_PUT))
        tc = _timed(lambda: bt.bt_price_exact(ctx.h, oc, bt.BT_PREC_FP32_COMP), reps=2)
        ev = sum(class_evaluations(bt, o) for o in oc)
        return {"workload": "64 sets (seed 0) x {geometric Asian call, fixed-strike lookback call, European put}, "
                            "N=36, FP32_COMP (recombined suffix classes), host arrays in and out",
                "ms": 1e3 * tc, "prefix_class_evaluations_per_s": ev / tc, "ops_per_evaluation": CLS_OPS_SINGLE,
                "frac_of_issue_peak": CLS_OPS_SINGLE * ev / tc / peak,
                "equivalent_payoff_paths_per_s": len(oc) * 2.0 ** 36 / tc}

    def small_arith_row():
        # the small arithmetic Asians (N <= 27), every suffix a class
        oa = W.batched_exact_workload(24, 0, 64)
        ta = _timed(lambda: bt.bt_price_exact(ctx.h, oa, bt.BT_PREC_FP32_COMP), reps=3)
        ev = sum(class_evaluations(bt, o) for o in oa[::2])     # call/put pairs: one evaluation per pair
        return {"workload": "64 sets (seed 0) x arithmetic Asian call+put, N=24, FP32_COMP (each suffix a class, "
                            "a call/put pair per pass), host arrays in and out",
                "ms": 1e3 * ta, "prefix_class_pair_evaluations_per_s": ev / ta,
                "ops_per_pair_evaluation": CLS_OPS_PAIR, "frac_of_issue_peak": CLS_OPS_PAIR * ev / ta / peak,
                "equivalent_payoff_paths_per_s": len(oa) * 2.0 ** 24 / ta}

    def n32_row():
        # the batched workload at N=32 in the all-FP64 kernel (the accuracy reference) beside FP32_COMP
        o32 = W.batched_exact_workload(32, 0, 64)
        t64 = _timed(lambda: bt.bt_price_exact(ctx.h, o32, bt.BT_PREC_FP64), reps=1)
        t32 = _timed(lambda: bt.bt_price_exact(ctx.h, o32, bt.BT_PREC_FP32_COMP), reps=2)
        return {"workload": "batched arithmetic-Asian call+put, N=32, 64 sets (seed 0), host arrays in and out",
                "fp64_s": t64, "fp32_comp_s": t32, "fp64_payoff_paths_per_s": 128 * 2.0 ** 32 / t64,
                "fp32_comp_payoff_paths_per_s": 128 * 2.0 ** 32 / t32}

    def paper_row():
        # the paper's runtime workload (Section 5): a European put, K=10, S0=5,
        # sigma 0.3, rate 0.06, T=1, CRR, N=32; the paper's 64-core Julia run took
        # 13:38 (818 s) and R 2:22:59 (8579 s) on 2x E5-2650v2 nodes
        op = W.paper_runtime_workload(32)
        t_fast = _timed(lambda: bt.bt_price_exact(ctx.h, [op], bt.BT_PREC_FP64))
        u, d, p = bt.bt_tree_params(op)
        mvp = [np.tile([d, u, 1 - p, p], (32, 1))]
        t_walk = _timed(lambda: bt.bt_price_exact_branching(ctx.h, [op], 2, mvp), reps=1)
        return {"workload": "European put, K=10, S0=5, sigma 0.3, rate 0.06, T=1, CRR, N=32 (2^32 paths)",
                "exact_fp64_s": t_fast, "generic_per_path_walk_s": t_walk,
                "paper_context": {"julia_64_cores_s": 818, "r_64_cores_s": 8579,
                                  "hardware": "8 nodes of 2x Intel E5-2650v2 (16 cores each), QDR InfiniBand",
                                  "note": "context, not the target: the paper's workload on the paper's cluster"}}

    rows = (("steps", steps_row), ("generic_binomial", generic_binomial_row),
            ("trinomial_affine", trinomial_affine_row), ("generic_trinomial", generic_trinomial_row),
            ("single_asian_n20_fp64", single_row), ("class_payoffs_n36", class_row),
            ("small_arith_n24_class_pass", small_arith_row), ("batched_n32_fp64_vs_fp32", n32_row),
            ("paper_runtime_workload", paper_row))
    return {name: fn() for name, fn in rows if only is None or name in only}


# ---------------------------------------------------------------------------
# Reference arm: the CPU oracle
# ---------------------------------------------------------------------------
def run_reference(args, rank):
    if rank != 0:
        return
    from paper_1701_03512_gb300 import workloads as W
    opts = W.batched_exact_workload(args.N, 0, args.sets)
    threads = cpu_threads()
    per_step = max(2.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_sample(opts, per_step / 4, threads)
    vals, secs, sample = [], [], ""
    for _ in range(args.steps):
        v, sample = cpu_oracle_sample(opts, per_step, threads)
        vals.append(v)
        secs.append(cpu_oracle_sample.last_seconds)
    value = statistics.median(vals)
    step_paths = float(len(opts)) * 2.0 ** args.N
    # a step here is one bounded sample of the workload (the whole batch would
    # take ms_full_workload at this rate)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
            "ms_full_workload": 1e3 * step_paths / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, {"engine": "CPU oracle (plain C, FP64)",
                                                                   "precision": "FP64 (oracle)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def summary(line):
    """The headline figures of every part in one compact object."""
    def g(d, *ks):
        for k in ks:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d
    out = {"exact_n36_paths_per_s": line["value"], "exact_n36_frac_of_issue_peak": g(line, "roofline", "frac"),
           "e2e_paths_per_s": g(line, "e2e", "value"), "scaling": line["scaling"], "n_gpus": line["n_gpus"]}
    sv = line.get("serving")
    if isinstance(sv, dict):
        out["serving_capacity_rps"] = sv.get("capacity_rps")
        out["serving_identical_values"] = sv.get("identical_values")
        out["serving_p50_p99_ms"] = {
            "%.2f" % r["load_vs_plain_capacity"]: {m: [round(r[m]["p50_ms"], 3), round(r[m]["p99_ms"], 3)]
                                                 for m in ("plain", "batched")} for r in sv.get("loads", [])}
    mc = line.get("mc")
    if isinstance(mc, dict):
        out["mc_n252_samples_per_s"] = mc.get("samples_per_s")
        out["mc_frac_of_issue_peak"] = mc.get("frac_of_issue_peak")
        out["mc_frac_of_heavy_pipe_bound"] = g(mc, "heavy_pipe_bound", "frac")
        out["mc_shared_n64_pairs_per_s"] = g(mc, "shared_sample", "prefix_suffix_pairs_per_s")
        out["mc_shared_frac_of_issue_peak"] = g(mc, "shared_sample", "frac_of_issue_peak")
    gr = line.get("greeks")
    if isinstance(gr, dict):
        out["greeks_n28_ms"] = gr.get("ms")
        out["greeks_frac_of_issue_peak"] = gr.get("frac_of_issue_peak")
    w = line.get("widened")
    if isinstance(w, dict):
        out["steps_n32_payoff_paths_per_s"] = g(w, "steps", "payoff_paths_per_s")
        out["steps_frac_of_issue_peak"] = g(w, "steps", "frac_of_issue_peak")
        out["trinomial_frac_of_issue_peak"] = g(w, "trinomial_affine", "frac_of_issue_peak")
        out["class_pass_n36_evaluations_per_s"] = g(w, "class_payoffs_n36", "prefix_class_evaluations_per_s")
        out["class_pass_n36_frac_of_issue_peak"] = g(w, "class_payoffs_n36", "frac_of_issue_peak")
        out["n32_fp32_comp_payoff_paths_per_s"] = g(w, "batched_n32_fp64_vs_fp32", "fp32_comp_payoff_paths_per_s")
        out["n32_fp64_payoff_paths_per_s"] = g(w, "batched_n32_fp64_vs_fp32", "fp64_payoff_paths_per_s")
    return out


# ---------------------------------------------------------------------------
# The split of one batch across ranks (Section 3, eq. f14/f15)
# ---------------------------------------------------------------------------
def split_combine(ex, local_values):
    """eq. f15 across ranks: every rank's per-option partial values (its work
    items' discounted sums) are gathered and added in rank order with
    Neumaier's compensated sum, so every rank returns the same numbers.
    `ex` is a sharded.Exchange (None for a single rank)."""
    import numpy as np
    from paper_1701_03512_gb300 import sharded as S
    local_values = np.asarray(local_values, dtype=np.float64)
    if ex is None:
        return S.combine(local_values[None, :])
    return S.combine(ex.gather(local_values, "bench-split"))


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import numpy as np
    import torch
    from paper_1701_03512_gb300 import btree as bt
    from paper_1701_03512_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    if args.only:
        ctx = bt.Context(local_rank)
        sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
        fmax = float(measured_peaks().get("sm_max_mhz", 2070.0))
        rows = extras_bench(bt, W, ctx, sms, fmax, with_cpu=False, only=set(args.only.split(",")))
        print(json.dumps(rows), flush=True)
        ctx.close()
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ctx = bt.Context(local_rank)
    split = (world > 1 and not args.weak) or args.split
    ex = None
    if split and world > 1:
        from paper_1701_03512_gb300 import sharded as S
        ex = S.Exchange(rank, world, dist.distributed_c10d._get_default_store(), timeout_s=120.0)
    # split (default): every rank holds the one batch and runs its share of the
    # work items; weak: every rank prices its own batch (seed = rank; rank 0's
    # is the one-GPU workload)
    opts = W.batched_exact_workload(args.N, 0 if split else rank, args.sets)
    plan = bt.bt_exact_plan_create(ctx.h, opts, bt.BT_PREC_FP32_COMP)
    info = bt.bt_exact_plan_info_get(plan)
    step_paths = info["payoff_paths"]            # the batch: every rank's share together when split
    shard, n_shards = (rank, world) if split else (0, 1)
    stream = torch.cuda.Stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        bt.bt_exact_plan_run_shard(plan, shard, n_shards, stream)
        if split:
            split_combine(ex, bt.bt_exact_plan_read(plan, stream)["value"])
    stream.synchronize()

    sampler = ClockSampler(physical_gpu_index(local_rank))
    sampler.start()
    barrier()
    t_wall0 = time.perf_counter()
    step_ms, kern_ms, xchg_ms = [], [], []
    res_split = None
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt.bt_exact_plan_run_shard(plan, shard, n_shards, stream)
        e1.record(stream)
        kern_ms.append(bt.bt_exact_plan_kernel_ms(plan))
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        if split:   # the exchange of eq. f15: read this rank's partials, gather, combine (host clock)
            t0 = time.perf_counter()
            res_split = split_combine(ex, bt.bt_exact_plan_read(plan, stream)["value"])
            xchg_ms.append(1e3 * (time.perf_counter() - t0))
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    res = bt.bt_exact_plan_read(plan, stream)
    vals = res_split if split else res["value"]
    assert np.all(np.isfinite(vals)) and np.all(vals >= 0.0)

    tot_s = (sum(step_ms) + sum(xchg_ms)) / 1e3
    if dist is not None:
        t = torch.tensor([tot_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_s = float(t.item())
    value = (1 if split else world) * step_paths * args.steps / tot_s

    # end to end through the public API with host arrays (split: the sharded
    # call, plan creation and the exchange included)
    e2e = None
    if not args.no_e2e:
        host_opts = bt.options_array(opts)
        if split and ex is not None:
            from paper_1701_03512_gb300 import sharded as S

            def call():
                return S.price_exact_sharded(ex, opts, bt.BT_PREC_FP32_COMP, ctx.h)
        else:
            def call():
                return bt.bt_price_exact(ctx.h, host_opts, bt.BT_PREC_FP32_COMP, stream)["value"]
        call()  # warm
        barrier()
        ts = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            out = call()
            ts.append(time.perf_counter() - t0)
            assert np.all(np.isfinite(out))
        barrier()
        e2e_s = sum(ts)
        if dist is not None:
            t = torch.tensor([e2e_s], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": (1 if split else world) * step_paths * args.steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(info["h2d_bytes"]), "d2h_bytes_per_step": int(info["d2h_bytes"]),
               "ms_per_step": 1e3 * e2e_s / args.steps}

    if rank != 0:
        bt.bt_exact_plan_destroy(plan)
        ctx.close()
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    fmax = float(peaks.get("sm_max_mhz", 2070.0))
    peak_gops = sms * 128 * fmax * 1e6 / 1e9
    kernel_s = statistics.mean(kern_ms) / 1e3
    achieved = OPS_PER_PATH * step_paths / (world if split else 1) / kernel_s / 1e9   # this rank's share
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_gops, "unit": "Gop/s", "frac": achieved / peak_gops,
            "traffic": profiled_traffic(args.N),
            "kernel": "k_exact32", "kernel_ms": 1e3 * kernel_s,
            "ops_per_payoff_path": OPS_PER_PATH, "ops_executed_per_payoff_path": OPS_EXECUTED_PAIR / 2,
            "peak_basis": "%d SMs x 128 FP32 lanes x %.0f MHz (max SM clock, MEASURED_PEAKS.json)" % (sms, fmax)}
    # the same throughput counted as executed: the inner loop's 6.125 instructions per call+put pair
    roof["frac_as_executed"] = roof["frac"] * (OPS_EXECUTED_PAIR / 2) / OPS_PER_PATH
    if clocks.get("sm_mhz"):
        roof["frac_at_measured_clock"] = achieved / (sms * 128 * clocks["sm_mhz"] * 1e6 / 1e9)

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        threads = cpu_threads()
        v, sample = cpu_oracle_sample(opts, args.cpu_seconds, threads)
        v1, sample1 = cpu_oracle_sample(opts, max(2.0, args.cpu_seconds / 4), 1)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
               "one_core": {"value": v1, "sample": sample1}, "cpu": cpu_model()}

    serving = mc = greeks = extras = None
    if world == 1 and not args.no_mc:
        mc = mc_bench(bt, W, ctx, sms, fmax, with_cpu=not args.no_cpu_baseline)
    if world == 1 and not args.no_greeks:
        greeks = greeks_bench(bt, W, ctx, sms, fmax, with_cpu=not args.no_cpu_baseline)
    if world == 1 and not args.no_extras:
        extras = extras_bench(bt, W, ctx, sms, fmax, with_cpu=not args.no_cpu_baseline)
    if world == 1 and not args.no_serving:
        loads = [float(x) for x in args.serving_loads.split(",") if x]
        sctx = bt.Context(local_rank, device_budget_bytes=12 << 30)   # 8 GiB server pool + plain scratch
        serving = serving_bench(bt, W, sctx, args.serving_requests, loads)
        sctx.close()

    if split:
        par = ("split%d: one batch, rank r runs work items i %% %d == r (Section 3), one all-gather of the "
               "per-option partials combined in rank order (eq. f15)" % (world, world))
    elif world > 1:
        par = "dp%d: one batch of option sets per rank (seed = rank), no collective on the data path" % world
    else:
        par = "single GPU"
    extra_cfg = {"parallelism": par, "wall_s_timed": t_wall}
    if split:
        extra_cfg["exchange_ms_per_step"] = statistics.mean(xchg_ms)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak" if (world > 1 and not split) else "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(args, extra_cfg),
            "fp32_peak_frac": roof["frac"], "clocks": clocks, "e2e": e2e,
            # per step: k_params, k_tables, k_class_tables, k_exact32, k_finalize
            "gpu_launches": 5 * args.steps, "roofline": roof, "cpu_baseline": cpu,
            "serving": serving, "mc": mc, "greeks": greeks, "widened": extras}
    line["summary"] = summary(line)   # last, so that a kept tail of the line holds it
    print(json.dumps(line), flush=True)
    bt.bt_exact_plan_destroy(plan)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
