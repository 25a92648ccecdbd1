#!/usr/bin/env python
"""Throughput of the GB300 hash-join engine: (|R| + |S|) tuples per second.

Default workload: the radix-partitioned hash join (PHJ) of |R| = 2^24 and
|S| = 2^28 tuples of (uint32 key, uint32 rid); R keys a seeded permutation of
1..2^24, S keys uniform over [1, 2^25] (about half of S matches).  One step is a
whole join through the C ABI (hj_join): partition R and S, join every partition
pair, materialise the (rid_R, rid_S) pairs.  Inputs (2.28 GB) exceed the 129 MB
L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  At N=1 the default workload's line also carries
("also") summaries of the batched (4096 joins), served (20000 requests) and skewed
64-bit configurations, each run afterwards in a process of its own (--no-extras
skips them).  `--impl reference` times the CPU oracle instead.
Under torchrun every rank joins its own seeded relations (independent problems,
weak scaling, no data-path collective); value = all ranks' tuples / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "(|R|+|S|) tuples/s"
UNIT = "tuples/s"

WORKLOADS = {
    "phj_16m_256m": dict(
        nr=1 << 24, ns=1 << 28, dom=1 << 25, algo=2,
        desc="PHJ radix-partitioned join, |R|=2^24, |S|=2^28 (uint32 key, uint32 rid); R keys a seeded "
             "permutation of 1..2^24, S keys uniform over [1, 2^25] (~50% match); pairs materialised"),
    "phj_8m_128m": dict(
        nr=1 << 23, ns=1 << 27, dom=1 << 24, algo=2,
        desc="PHJ radix-partitioned join, |R|=2^23, |S|=2^27 (uint32 key, uint32 rid); the 2^24 x 2^28 join at "
             "half size (profiling case); R keys a permutation of 1..2^23, S keys uniform over [1, 2^24]"),
    "phj_16m_16m": dict(
        nr=1 << 24, ns=1 << 24, dom=1 << 24, algo=2,
        desc="the paper's default join size, |R| = |S| = 2^24 (uint32 key, uint32 rid); R keys a seeded "
             "permutation of 1..2^24, S keys uniform over them (every S tuple matches once); pairs materialised"),
    "batch_4096": dict(
        kind="batch", njoins=4096, nr=0, ns=0, algo=2,
        desc="4096 independent joins, |R| log-uniform in [2^10, 2^22], |S| = 4|R| (uint32 key, uint32 rid); "
             "R keys a permutation of 1..|R|, S keys uniform over [1, ceil(|R|/0.75)] (75% match); pairs "
             "materialised; one hj_join_batch call (CUDA graph per wave) per step vs one hj_join per join"),
    "serve_20000": dict(
        kind="serve", nreq=20000, nr=0, ns=0, algo=0, budget=120 << 30, load=0.7, sweep=(0.5, 0.9),
        desc="serving: 20000 join requests, Poisson arrivals, |R| log-uniform in [2^12, 2^24], |S| log-uniform "
             "in [|R|, 16|R|] (uint32 key, uint32 rid), R keys a permutation of 1..|R|, S keys uniform over "
             "[1, 2|R|] (50% match), pairs materialised; HBM admission budget 120 GiB"),
    "zipf_4m_64m_t05": dict(
        kind="zipf", nr=1 << 22, ns=1 << 26, ranks=1 << 20, theta_r=0.75, theta_s=0.5, algo=2, width=8, mode=1,
        desc="skewed PHJ, |R|=2^22, |S|=2^26 (uint64 key, uint64 payload); R keys Zipf(0.75), S keys Zipf(0.5) "
             "over the same 2^20 distinct 64-bit keys; count and checksums (about 4.9e9 pairs, not materialised)"),
    "zipf_4m_64m_t10": dict(
        kind="zipf", nr=1 << 22, ns=1 << 26, ranks=1 << 20, theta_r=0.75, theta_s=1.0, algo=2, width=8, mode=1,
        desc="skewed PHJ, |R|=2^22, |S|=2^26 (uint64 key, uint64 payload); R keys Zipf(0.75), S keys Zipf(1.0) "
             "over the same 2^20 distinct 64-bit keys; count and checksums (about 3.1e11 pairs, not materialised)"),
    "zipf_4m_64m_t05_pairs": dict(
        kind="zipf", nr=1 << 22, ns=1 << 26, ranks=1 << 20, theta_r=0.75, theta_s=0.5, algo=2, width=8, mode=2,
        size_hint=True, no_e2e=True, no_cpu=True,
        desc="skewed PHJ, |R|=2^22, |S|=2^26 (uint64 key, uint64 payload); R keys Zipf(0.75), S keys Zipf(0.5) "
             "over the same 2^20 distinct 64-bit keys; every pair materialised (about 4.9e9 pairs, 79 GB; the "
             "pair buffer sized from the warm-up's count)"),
    "sweep_16m": dict(
        kind="sweep", nr=1 << 24, ns=1 << 24, dom=1 << 24, algo=0,
        desc="the paper's sweeps on GB300: |S| = 2^24 with |R| = 2^16 .. 2^24 (R keys a permutation of 1..|R|, "
             "S keys uniform over them: every S tuple matches once), and selectivity 12.5 / 50 / 100 % at "
             "|R| = |S| = 2^24 (S keys uniform over [1, |R| / selectivity]); uint32 key/rid, pairs materialised, "
             "each point autotuned; value = the 2^24 x 2^24 point at 100 %"),
    "outcore_16m_256m": dict(
        kind="outcore", nr=1 << 24, ns=1 << 28, dom=1 << 25, algo=2, budget=1 << 30,
        desc="larger-than-device join from host memory: the 2^24 x 2^28 PHJ workload (uint32 key/rid, ~50% "
             "match) in page-locked host memory, joined through a 1 GiB device budget, pairs copied to host "
             "memory; the value is the library's plan (R kept on the device, S streamed past it in chunks), "
             "and split_ms_per_step times the paper's App. A split of both relations (chunked top-level split "
             "on the device, host partitions, partition pairs joined on the device) on the same call"),
    "heavy_16m_s10": dict(
        kind="heavy", nr=1 << 24, ns=1 << 24, s=0.10, algo=2,
        desc="the paper's low-skew data set at its default size: |R| = |S| = 2^24 (uint32 key, uint32 rid); 10 % of "
             "R's tuples share one key, the other R keys distinct, S keys uniform over R's distinct keys; pairs "
             "materialised"),
    "heavy_16m_s25": dict(
        kind="heavy", nr=1 << 24, ns=1 << 24, s=0.25, algo=2,
        desc="the paper's high-skew data set at its default size: |R| = |S| = 2^24 (uint32 key, uint32 rid); 25 % of "
             "R's tuples share one key, the other R keys distinct, S keys uniform over R's distinct keys; pairs "
             "materialised"),
    "phj_sharded": dict(
        kind="sharded", nr=1 << 24, ns=1 << 28, dom=1 << 25, algo=2,
        desc="one PHJ of |R|=2^24, |S|=2^28 (uint32 key, uint32 rid; the default workload's relations) sharded "
             "over the ranks: each rank holds 1/N of R's and S's rows, splits them by the sharding hash (hj_split), "
             "one all-to-all of R and one of S, a local hj_join, one all-reduce of count and checksums; strong "
             "scaling (the whole job is one join); pairs materialised, left on the rank that found them"),
    "coproc_16m": dict(
        kind="coproc", nr=1 << 24, ns=1 << 24, dom=1 << 24, algo=2, shares=1000,
        desc="CPU/GPU co-processing of the paper's default join, |R| = |S| = 2^24 (uint32 key, uint32 rid; R keys a "
             "permutation of 1..2^24, S keys uniform over them): the PHJ's join step divided between the GPU and "
             "the host cores (hj_join_coproc) at the cost model's share, and the model (Eq. 1-5) checked against "
             "measured times at 1000 seeded random shares (the paper's validation of its model); pairs "
             "materialised"),
    "shj_1m": dict(
        nr=1 << 20, ns=1 << 20, dom=1 << 20, algo=1,
        desc="SHJ, |R|=|S|=2^20 (uint32 key, uint32 rid); R keys a permutation of 1..2^20, S keys drawn "
             "from R's keys (every probe matches once); pairs materialised"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hj", choices=["hj", "reference"])
    ap.add_argument("--workload", default="phj_16m_256m", choices=sorted(WORKLOADS))
    ap.add_argument("--algo", type=int, default=-1, help="0 auto, 1 SHJ, 2 PHJ (default: tuned)")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--radix-bits", type=int, default=0)
    ap.add_argument("--passes", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--plain-steps", type=int, default=2)
    ap.add_argument("--prof-steps", type=int, default=20,
                    help="untimed steps with every launch event-timed, for the per-kernel breakdown")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload at N=1: skip the batched, served and skewed runs added to the line")
    ap.add_argument("--plain-seconds", type=float, default=20.0,
                    help="serving: bound on the one-hj_join-per-request comparison run")
    ap.add_argument("--no-sweep", action="store_true", help="serving: skip the offered-load sweep")
    ap.add_argument("--serve-workers", type=int, default=4, help="serving: worker threads (streams)")
    ap.add_argument("--serve-wave-tuples", type=int, default=0, help="serving: tuples per wave (0: the default)")
    ap.add_argument("--scatter", default="auto", choices=["auto", "region", "ring"],
                    help="padded-pass scatter at 2^9..2^11 digits (hj_debug_scatter): auto, or force one kernel")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------- ranks


def ranks_max(x: float, ws: int, dev=None) -> float:
    """Max over ranks of a local measurement (one all-reduce of a scalar; the join
    itself exchanges nothing between ranks)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(units_per_rank_step: int, steps: int, ws: int, ms_max: float) -> float:
    """Whole-job throughput of independent per-rank problems: the units every rank
    processed over the slowest rank's time."""
    return units_per_rank_step * steps * ws / (ms_max / 1000.0)


# ------------------------------------------------------------------- peaks, clocks


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------- roofline


def kernel_bytes(name: str, wl: dict, w: int, passes: int, pairs: int) -> float:
    """Algorithmic bytes one step moves in all launches of kernel `name`."""
    n = wl["nr"] + wl["ns"]
    tb = 2 * w
    if name == "partition_scatter":      # read + write every tuple, each pass
        return 2.0 * tb * n * passes
    if name == "partition_hist":         # read every tuple, each pass
        return 1.0 * tb * n * passes
    if name == "partition_join":         # read both partitioned relations, write the pairs
        return tb * n + tb * pairs
    if name == "table_build":
        return tb * wl["nr"]
    if name == "table_probe":
        return tb * wl["ns"] + tb * pairs
    return 0.0


def traffic_record(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the
    kernel source is unchanged since it was captured (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)[workload][kernel]
        src = os.path.join(ROOT, "paper_1307_1955_gb300", "csrc", rec["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        return rec["bytes_per_launch"] if h == rec["source_sha"] else None
    except Exception:
        return None


# ------------------------------------------------------------------- CPU oracle


class OneCore:
    """Run the single-threaded oracle pinned to one host core (Linux affinity),
    restoring the process's affinity afterwards; records the host's core count."""

    def __enter__(self):
        self.saved = None
        try:
            self.saved = os.sched_getaffinity(0)
            os.sched_setaffinity(0, {max(self.saved)})
        except (AttributeError, OSError):
            pass
        return self

    def __exit__(self, *exc):
        if self.saved:
            try:
                os.sched_setaffinity(0, self.saved)
            except OSError:
                pass


def host_cores() -> int:
    return os.cpu_count() or 0


def oracle_rate(R_np, S_np, mode=2):
    """Run the oracle's hash join once (pairs materialised), or its per-key
    aggregation in the count modes; return (tuples, seconds, pairs)."""
    import oracle

    with OneCore():
        t0 = time.perf_counter()
        if mode == 2:
            rr, ss = oracle.hash_join(R_np, S_np, cap_hint=len(S_np))
            m = len(rr)
        else:
            m = oracle.join_aggregate(R_np, S_np)[0]
        dt = time.perf_counter() - t0
    return len(R_np) + len(S_np), dt, m


def make_inputs(wl, rank, device):
    from paper_1307_1955_gb300 import workload as W

    if wl.get("kind") == "zipf":
        return W.zipf_pair(wl["nr"], wl["ns"], wl["theta_r"], wl["theta_s"], wl["ranks"], W.DEFAULT_SEED, device,
                           ids=(3, int(wl["theta_s"] * 10), rank))

    if wl.get("kind") == "heavy":
        return W.heavy_hitter(wl["nr"], wl["ns"], wl["s"], W.DEFAULT_SEED, device, ids=(66, int(wl["s"] * 100), rank))
    return W.unique_and_uniform(wl["nr"], wl["ns"], wl["dom"], W.DEFAULT_SEED, device, ids=(2, rank))


def cpu_sample(wl, R, S, target_s: float):
    """Oracle on a bounded sample: all of R and a prefix of S sized to about target_s."""
    from paper_1307_1955_gb300 import workload as W

    mode = wl.get("mode", 2)
    Rn = W.to_numpy_u(R)
    ns0 = min(len(S), 1 << 20)
    n, dt, _ = oracle_rate(Rn, W.to_numpy_u(S[:ns0]), mode)
    # time per S tuple beyond the build, from one calibration run
    rate = max(n / dt, 1.0)
    want = int(min(len(S), max(ns0, rate * target_s - len(Rn))))
    Ss = W.to_numpy_u(S[:want])
    n, dt, m = oracle_rate(Rn, Ss, mode)
    what = f"{m} pairs materialised" if mode == 2 else f"{m} pairs counted by per-key aggregation"
    return {"value": n / dt, "unit": UNIT, "cores": 1, "host_cores": host_cores(), "kind": "oracle",
            "sample": f"all |R|={len(Rn)} tuples, first {want} of |S|={len(S)} tuples "
                      f"({what}), single-threaded C oracle, {dt:.1f} s"}


# ------------------------------------------------------------------- arms


def run_reference(args, wl, ws, rank):
    """The CPU oracle on the machine's host cores, one bounded sample per step."""
    if rank != 0:
        return
    import torch

    from paper_1307_1955_gb300 import workload as W
    import oracle

    oracle.build()
    total = args.steps + args.warmup
    per_step = max(0.05, min(20.0, 150.0 / max(total, 1)))
    if wl.get("kind") in ("batch", "serve"):
        run_reference_batch(args, wl, ws, per_step)
        return
    if wl.get("kind") in ("zipf", "heavy"):
        run_reference_prefix(args, wl, ws, per_step)
        return
    # Scale the workload down (|S| / |R| and the key-domain ratio kept) so that one
    # step takes about per_step seconds: time the oracle at 1/256 and extrapolate.
    cal = 256
    R, S = W.unique_and_uniform(wl["nr"] // cal, wl["ns"] // cal, wl["dom"] // cal, W.DEFAULT_SEED, "cpu",
                                ids=(2, 0))
    _, dt_cal, _ = oracle_rate(W.to_numpy_u(R), W.to_numpy_u(S))
    scale = 1
    while dt_cal * cal / scale > per_step and scale < (1 << 14):
        scale *= 2
    R, S = W.unique_and_uniform(wl["nr"] // scale, wl["ns"] // scale, wl["dom"] // scale, W.DEFAULT_SEED, "cpu",
                                ids=(2, 0))
    Rn, Sn = W.to_numpy_u(R), W.to_numpy_u(S)
    for _ in range(args.warmup):
        oracle_rate(Rn, Sn)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_rate(Rn, Sn)
    dt = time.perf_counter() - t0
    value = (len(Rn) + len(Sn)) * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * dt / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": wl["desc"], "sample_scale": f"1/{scale} of |R| and |S|"},
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": 1, "host_cores": host_cores(),
                         "sample": f"|R|={len(Rn)}, |S|={len(Sn)} (the workload scaled by 1/{scale}), "
                                   f"single-threaded C oracle hash join, pairs materialised"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_prefix(args, wl, ws, per_step):
    """Oracle on the workload's own relations: all of R and the prefix of S whose
    oracle time is about per_step seconds (count modes: per-key aggregation)."""
    from paper_1307_1955_gb300 import workload as W

    mode = wl.get("mode", 2)
    R, S = make_inputs(wl, 0, "cpu")
    Rn = W.to_numpy_u(R)
    ns0 = min(len(S), 1 << 20)
    n, dt, _ = oracle_rate(Rn, W.to_numpy_u(S[:ns0]), mode)
    want = int(min(len(S), max(ns0, max(n / dt, 1.0) * per_step - len(Rn))))
    Sn = W.to_numpy_u(S[:want])
    for _ in range(args.warmup):
        oracle_rate(Rn, Sn, mode)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_rate(Rn, Sn, mode)
    dt = time.perf_counter() - t0
    value = (len(Rn) + len(Sn)) * args.steps / dt
    sample = (f"all |R|={len(Rn)} tuples and the first {want} of |S|={len(S)} tuples, single-threaded C oracle, "
              + ("pairs materialised" if mode == 2 else "count and checksums by per-key aggregation"))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * dt / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32" if wl.get("width", 4) == 4 else "u64",
        "data": "synthetic", "config": {"workload": wl["desc"], "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": 1, "host_cores": host_cores(), "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_batch(args, wl, ws, per_step):
    """Oracle on the batch's (or the request stream's) joins in order: each step
    joins the first joins whose oracle time adds up to about per_step seconds."""
    from paper_1307_1955_gb300 import workload as W

    if wl.get("kind") == "serve":
        specs = W.serving_specs(wl["nreq"], W.DEFAULT_SEED, 1.0)
        gen_ids = lambda j: (5, j)  # noqa: E731
    else:
        specs = W.batched_specs(wl["njoins"], W.DEFAULT_SEED)
        gen_ids = lambda j: (4, j)  # noqa: E731
    sample, acc = [], 0.0
    for j, sp in enumerate(specs):
        R, S = W.unique_and_uniform(sp.n_r, sp.n_s, sp.s_domain, W.DEFAULT_SEED, "cpu", ids=gen_ids(j))
        sample.append((W.to_numpy_u(R), W.to_numpy_u(S)))
        acc += oracle_rate(*sample[-1])[1]
        if acc >= per_step:
            break
    tuples = sum(len(r) + len(s) for r, s in sample)
    for _ in range(args.warmup):
        for r, s in sample[:1]:
            oracle_rate(r, s)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for r, s in sample:
            oracle_rate(r, s)
    dt = time.perf_counter() - t0
    value = tuples * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * dt / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": wl["desc"], "sample": f"the first {len(sample)} of {len(specs)} joins"},
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": 1, "host_cores": host_cores(),
                         "sample": f"the first {len(sample)} joins of the batch ({tuples} tuples), "
                                   f"single-threaded C oracle hash join, pairs materialised"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def force_scatter(hj, ctx, kind: str):
    """Make the context's padded passes take one scatter kernel (measurement only;
    results are identical either way)."""
    if kind != "auto":
        code = {"region": hj.HJ_SCATTER_REGION, "ring": hj.HJ_SCATTER_RING}[kind]
        assert hj.load_library().hj_debug_scatter(ctx.handle, code) == hj.HJ_OK


def run_hj(args, wl, ws, rank, local):
    import torch
    import torch.distributed as dist

    import __graft_entry__

    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    from paper_1307_1955_gb300 import hj

    dev = torch.device("cuda", local)
    R, S = make_inputs(wl, rank, dev)
    stream = torch.cuda.current_stream(dev)
    ctx = hj.Context(local, stream=stream)
    force_scatter(hj, ctx, args.scatter)
    mode = wl.get("mode", hj.HJ_MATERIALIZE)
    w = wl.get("width", 4)
    kw = dict(algo=wl["algo"] if args.algo < 0 else args.algo, radix_bits=args.radix_bits, passes=args.passes,
              mode=mode)
    tuned = None
    if args.algo < 0 and args.radix_bits == 0 and args.passes == 0 and not args.no_tune:
        # the autotuner times the cost model's cheapest plans on these relations
        # (untimed); the timed joins then run its pick through HJ_ALGO_AUTO
        tuned = hj.hj_tune(ctx, R, S, mode=mode)
        kw = dict(algo=hj.HJ_ALGO_AUTO, mode=mode)

    def step():
        res = hj.hj_join(ctx, R, S, **kw)
        info = (res.count, res.radix_bits, res.passes, res.algo)
        res.free()
        return info

    for _ in range(args.warmup):
        info = step()
    if wl.get("size_hint"):
        # a caller that knows its output size passes it: one join per step, no rerun
        kw["out_capacity"] = info[0]
    torch.cuda.synchronize()
    # per-kernel breakdown from a profiled pass outside the timed region (events
    # around every launch); the timed region brackets the dominant kernel only
    prof_n = max(1, min(args.steps, args.prof_steps))
    hj.prof_reset(ctx)
    hj.prof_only(ctx, None)
    hj.prof_enable(ctx, True)
    for _ in range(prof_n):
        step()
    prof_all = hj.prof_read(ctx)
    hj.prof_enable(ctx, False)
    dom_name = max(prof_all.items(), key=lambda kv: kv[1][1])[0]
    sampler = ClockSampler(local)
    if not args.no_clocks:
        sampler.start()
        time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    hj.prof_reset(ctx)
    hj.prof_only(ctx, dom_name)
    hj.prof_enable(ctx, True)
    l0 = hj.launch_count(ctx)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        info = step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches = hj.launch_count(ctx) - l0
    ms = ev0.elapsed_time(ev1)
    prof = hj.prof_read(ctx)
    hj.prof_enable(ctx, False)
    hj.prof_only(ctx, None)
    clocks = sampler.stop() if not args.no_clocks else None
    ms = ranks_max(ms, ws, dev)
    count, bits, passes, algo = info
    value = weak_value(wl["nr"] + wl["ns"], args.steps, ws, ms)

    # roofline of the dominant kernel (algorithmic bytes / its event-timed duration)
    peak, peak_kind = measured_peak()
    out_pairs = count if mode == hj.HJ_MATERIALIZE else 0
    dom_launches, dom_ms = prof.get(dom_name, (0, 0.0))
    g = max(passes, 1) if algo == 2 else 0
    bytes_k = kernel_bytes(dom_name, wl, w, g, out_pairs) * args.steps
    achieved = bytes_k / (dom_ms / 1000.0) / 1e9 if dom_ms > 0 else 0.0
    per_launch_bytes = bytes_k / max(dom_launches, 1)
    roofline = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind,
                "bytes_per_launch": per_launch_bytes, "launches": dom_launches,
                "avg_launch_ms": dom_ms / max(dom_launches, 1),
                "traffic": traffic_record(dom_name, args.workload)}
    # whole-join roofline: (2g + 1) w (|R| + |S|) + o M bytes per step (PHJ), w (|R|+|S|) + o M (SHJ)
    n, tb = wl["nr"] + wl["ns"], 2 * w
    join_bytes = ((2 * g + 1) * tb * n if algo == 2 else tb * n) + tb * out_pairs
    join_bytes_g1 = 3 * tb * n + tb * out_pairs if algo == 2 else join_bytes
    step_s = ms / 1000.0 / args.steps
    join_roof = {"bytes_per_step": join_bytes, "achieved_gbs": join_bytes / step_s / 1e9,
                 "frac": join_bytes / step_s / 1e9 / peak, "frac_vs_g1": join_bytes_g1 / step_s / 1e9 / peak}
    if bytes_k == 0:
        # the dominant kernel has no per-launch byte count of its own (the key-list
        # fallback: its rows are however many partitions overflowed): the whole join
        # against its algorithmic bytes stands for it
        roofline = {"bound": "hbm", "kernel": f"whole join (all kernels; dominant: {dom_name})",
                    "achieved": join_roof["achieved_gbs"], "peak": peak, "unit": "GB/s", "frac": join_roof["frac"],
                    "peak_kind": peak_kind, "bytes_per_launch": join_bytes, "launches": args.steps,
                    "avg_launch_ms": ms / args.steps, "traffic": None}
    kernels = {k: {"launches": v[0], "ms": v[1], "share": v[1] / sum(x[1] for x in prof_all.values()),
                   "steps": prof_n}
               for k, v in sorted(prof_all.items(), key=lambda kv: -kv[1][1])}

    # end to end through hj_join_host: host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e and not wl.get("no_e2e"):
        Rh = R.cpu().pin_memory()
        Sh = S.cpu().pin_memory()
        out = (torch.empty((max(wl["ns"], count) + (1 << 20), 2), dtype=R.dtype).pin_memory()
               if mode == hj.HJ_MATERIALIZE else None)
        res = hj.hj_join_host(ctx, Rh, Sh, out, **kw)
        m = res.count
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            res = hj.hj_join_host(ctx, Rh, Sh, out, **kw)
        torch.cuda.synchronize()
        dt = ranks_max(time.perf_counter() - t0, ws, dev)
        e2e = {"value": weak_value(wl["nr"] + wl["ns"], args.e2e_steps, ws, dt * 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": tb * (wl["nr"] + wl["ns"]),
               "d2h_bytes_per_step": (tb * m if mode == hj.HJ_MATERIALIZE else 0) + 24,
               "api": "hj_join_host", "steps": args.e2e_steps}
        del Rh, Sh, out

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and not wl.get("no_cpu"):
        # (not for the materialised skewed join: the oracle's pairs for even a 2^20-row
        # sample of S -- about 8e7 -- would take most of the sample's time budget)
        cpu = cpu_sample(wl, R, S, target_s=15.0)

    also = None
    if ws == 1 and not args.no_extras and args.workload == "phj_16m_256m":
        # the other configurations, each in its own process once this one's memory is free
        ctx.close()
        del R, S
        torch.cuda.empty_cache()
        also = run_extras()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32" if w == 4 else "u64", "data": "synthetic",
            "config": {"workload": wl["desc"], "algo": {1: "SHJ", 2: "PHJ"}[algo], "radix_bits": bits,
                       "mode": {0: "count", 1: "count+checksum", 2: "pairs materialised"}[mode],
                       "passes": passes, "plan": "hj_tune" if tuned else "forced", "scatter": args.scatter,
                       "tuned": tuned, "pairs_per_step": count, "parallelism": f"replicas x{ws}",
                       "l2": f"inputs {tb * n / 1e9:.2f} GB per step exceed the 129 MB L2; no flush"
                       if tb * n > 129e6 else "inputs smaller than L2; warm L2 across steps"},
            "roofline": roofline, "join_roofline": join_roof, "kernels": kernels,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        }
        if also is not None:
            line["also"] = also
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def batch_inputs(wl, rank, dev):
    from paper_1307_1955_gb300 import workload as W

    seed = W.DEFAULT_SEED + rank
    specs = W.batched_specs(wl["njoins"], seed)
    R_all, S_all, rs, ss = W.batched_relations(specs, seed, dev)
    Rs = [R_all[rs[j]:rs[j] + sp.n_r] for j, sp in enumerate(specs)]
    Ss = [S_all[ss[j]:ss[j] + sp.n_s] for j, sp in enumerate(specs)]
    return specs, R_all, S_all, Rs, Ss


def batch_cpu_sample(Rs, Ss, target_s: float):
    """The oracle over the batch's joins in order until about target_s seconds."""
    from paper_1307_1955_gb300 import workload as W

    tuples, dt, k, pairs = 0, 0.0, 0, 0
    while k < len(Rs) and dt < target_s:
        n, t, m = oracle_rate(W.to_numpy_u(Rs[k]), W.to_numpy_u(Ss[k]))
        tuples += n
        dt += t
        pairs += m
        k += 1
    return {"value": tuples / dt, "unit": UNIT, "cores": 1, "host_cores": host_cores(), "kind": "oracle",
            "sample": f"the first {k} of {len(Rs)} joins ({tuples} tuples, {pairs} pairs materialised), "
                      f"single-threaded C oracle, {dt:.1f} s"}


def run_batch(args, wl, ws, rank, local):
    """Config of many uneven joins: hj_join_batch (one persistent join launch per wave,
    CUDA graph) against one hj_join call per join, on the same resident inputs."""
    import torch
    import torch.distributed as dist

    import __graft_entry__

    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    from paper_1307_1955_gb300 import hj

    dev = torch.device("cuda", local)
    specs, R_all, S_all, Rs, Ss = batch_inputs(wl, rank, dev)
    torch.cuda.synchronize()
    tuples_step = sum(sp.n_r + sp.n_s for sp in specs)
    stream = torch.cuda.current_stream(dev)
    ctx = hj.Context(local, stream=stream)
    ra, sa = hj.rel_array(Rs), hj.rel_array(Ss)
    n = len(specs)

    def batched(graph=True):
        outs = hj.hj_join_batch(ctx, ra, sa, graph=graph, raw=True)
        counts = [outs[j].count for j in range(n)]
        hj.hj_results_free(ctx, outs, n)
        return counts

    def plain():
        for j in range(n):
            hj.hj_join(ctx, Rs[j], Ss[j]).free()

    def timed(fn, steps):
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return ranks_max(e0.elapsed_time(e1), ws, dev), out

    for _ in range(args.warmup):
        counts = batched()
    sampler = ClockSampler(local)
    if not args.no_clocks:
        sampler.start()
        time.sleep(0.3)
    l0 = hj.launch_count(ctx)
    ms, counts = timed(batched, args.steps)
    launches = hj.launch_count(ctx) - l0
    clocks = sampler.stop() if not args.no_clocks else None
    pairs = sum(counts)
    value = weak_value(tuples_step, args.steps, ws, ms)

    # the same joins one hj_join call at a time
    plain()
    psteps = max(1, min(args.steps, args.plain_steps))
    pms, _ = timed(plain, psteps)
    plain_value = weak_value(tuples_step, psteps, ws, pms)

    # kernel times from one profiled step without the graph (events are not captured)
    hj.prof_reset(ctx)
    hj.prof_enable(ctx, True)
    batched(graph=False)
    torch.cuda.synchronize()
    prof = hj.prof_read(ctx)
    hj.prof_enable(ctx, False)
    peak, peak_kind = measured_peak()
    dom_name, (dom_launches, dom_ms) = max(prof.items(), key=lambda kv: kv[1][1])
    wl1 = {"nr": sum(sp.n_r for sp in specs), "ns": sum(sp.n_s for sp in specs)}
    bytes_k = kernel_bytes(dom_name, wl1, 4, 1, pairs)
    achieved = bytes_k / (dom_ms / 1000.0) / 1e9 if dom_ms > 0 else 0.0
    roofline = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind, "bytes_per_launch": bytes_k / max(dom_launches, 1),
                "launches": dom_launches, "avg_launch_ms": dom_ms / max(dom_launches, 1),
                "traffic": traffic_record(dom_name, args.workload)}
    join_bytes = 3 * 8 * tuples_step + 8 * pairs
    step_s = ms / 1000.0 / args.steps
    join_roof = {"bytes_per_step": join_bytes, "achieved_gbs": join_bytes / step_s / 1e9,
                 "frac": join_bytes / step_s / 1e9 / peak}
    kernels = {k: {"launches": v[0], "ms": v[1], "share": v[1] / sum(x[1] for x in prof.values())}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = batch_cpu_sample(Rs, Ss, 12.0)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": wl["desc"], "joins": n, "tuples_per_step": tuples_step,
                       "pairs_per_step": pairs, "parallelism": f"replicas x{ws}",
                       "l2": f"inputs {8 * tuples_step / 1e9:.1f} GB per step exceed the 129 MB L2; no flush"},
            "plain": {"value": plain_value, "unit": UNIT, "ms_per_step": pms / psteps, "steps": psteps,
                      "api": "hj_join once per join"},
            "batched_vs_plain": value / plain_value,
            "roofline": roofline, "join_roofline": join_roof, "kernels": kernels,
            "cpu_baseline": cpu, "e2e": None, "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def run_sharded(args, wl, ws, rank, local):
    """One join whose rows are spread over the ranks (paper_1307_1955_gb300.dist):
    split, all-to-all, local join, all-reduce per step; value = the whole join's
    tuples over the slowest rank's time (strong scaling)."""
    import torch
    import torch.distributed as dist

    import __graft_entry__

    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    from paper_1307_1955_gb300 import dist as D
    from paper_1307_1955_gb300 import hj
    from paper_1307_1955_gb300 import workload as W

    dev = torch.device("cuda", local)
    # the default workload's relations; this rank keeps its share of the rows
    R, S = W.unique_and_uniform(wl["nr"], wl["ns"], wl["dom"], W.DEFAULT_SEED, dev, ids=(2, 0))
    r0, r1 = wl["nr"] * rank // ws, wl["nr"] * (rank + 1) // ws
    s0, s1 = wl["ns"] * rank // ws, wl["ns"] * (rank + 1) // ws
    R, S = R[r0:r1].clone(), S[s0:s1].clone()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream(dev)
    ctx = hj.Context(local, stream=stream)

    def step():
        res = D.shard_join(ctx, R, S, mode=hj.HJ_MATERIALIZE, checksum=False)
        res.local.free()
        return res

    for _ in range(args.warmup):
        res = step()
    sampler = ClockSampler(local)
    if not args.no_clocks:
        sampler.start()
        time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = hj.launch_count(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        res = step()
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches = hj.launch_count(ctx) - l0
    clocks = sampler.stop() if not args.no_clocks else None
    ms = ranks_max(e0.elapsed_time(e1), ws, dev)
    n = wl["nr"] + wl["ns"]
    value = n * args.steps / (ms / 1000.0)
    # one profiled step for the per-kernel times of this rank
    hj.prof_reset(ctx)
    hj.prof_enable(ctx, True)
    step()
    prof = hj.prof_read(ctx)
    hj.prof_enable(ctx, False)
    peak, peak_kind = measured_peak()
    dom_name, (dom_launches, dom_ms) = max(prof.items(), key=lambda kv: kv[1][1])
    tb = 8
    join_bytes = 3 * tb * n + tb * res.count
    step_s = ms / 1000.0 / args.steps
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": wl["desc"], "pairs_per_step": res.count, "parallelism": f"sharded x{ws}",
                       "rows_per_rank": [r1 - r0, s1 - s0], "received_rows_rank0": list(res.received),
                       "l2": "inputs far larger than the 129 MB L2; no flush"},
            "join_roofline": {"bytes_per_step": join_bytes, "achieved_gbs": join_bytes / step_s / 1e9,
                              "frac": join_bytes / step_s / 1e9 / peak / ws, "peak_per_gpu": peak},
            "roofline": None,
            "kernels_rank0": {k: {"launches": v[0], "ms": v[1]} for k, v in
                              sorted(prof.items(), key=lambda kv: -kv[1][1])},
            "dominant_kernel_rank0": dom_name,
            "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def deciles(pts):
    """Mean and max |relative error| of the model's two predictions per tenth of
    the CPU share range."""
    out = []
    for b in range(10):
        q = [p for p in pts if b / 10 <= p["share"] < (b + 1) / 10 or (b == 9 and p["share"] == 1.0)]
        if q:
            out.append({"share": [b / 10, (b + 1) / 10], "n": len(q),
                        "mean_abs_rel_err": sum(abs(p["rel_err"]) for p in q) / len(q),
                        "max_abs_rel_err": max(abs(p["rel_err"]) for p in q),
                        "mean_abs_rel_err_whole_wait": sum(abs(p["rel_err_whole_wait"]) for p in q) / len(q),
                        "mean_abs_rel_err_handoff": sum(abs(p["rel_err_handoff"]) for p in q) / len(q)})
    return out


def run_coproc(args, wl, ws, rank, local):
    """hj_join_coproc on the paper's default join: per-item costs calibrated at CPU
    shares 0 and 1, then the cost model's predicted time (hj_coproc_time, steps
    partition + join, the partition step on the GPU) against the measured time at
    seeded random shares; the value is the throughput at the model's own share."""
    import torch

    import __graft_entry__

    torch.cuda.set_device(local)
    if rank == 0:
        __graft_entry__.build()
    from paper_1307_1955_gb300 import hj
    from paper_1307_1955_gb300 import workload as W

    dev = torch.device("cuda", local)
    R, S = W.unique_and_uniform(wl["nr"], wl["ns"], wl["dom"], W.DEFAULT_SEED, dev, ids=(67, rank))
    torch.cuda.synchronize()
    ctx = hj.Context(local)
    N = wl["nr"] + wl["ns"]

    def run(share):
        res, t = hj.hj_join_coproc(ctx, R, S, share)
        cnt = res.count
        res.free()
        return t, cnt

    for _ in range(max(1, args.warmup)):
        run(0.0)
    run(1.0)
    # calibration: GPU per-item costs at share 0, CPU and copy costs at share 1 (medians of 3)
    t0 = [run(0.0)[0] for _ in range(3)]
    t1 = [run(1.0)[0] for _ in range(3)]
    med = lambda xs: statistics.median(xs)
    g1 = med([t["partition_gpu"] for t in t0]) / N
    g2 = med([t["join_gpu"] for t in t0]) / N
    c2 = med([t["join_cpu"] for t in t1]) / N
    xf = med([t["copy_to_host"] for t in t1]) / N
    cpu_s, gpu_s, x = [1.0, c2], [g1, g2], [float(N), float(N)]
    ratios_best, t_best = hj.hj_coproc_ratios(x, cpu_s, gpu_s, xfer_s=xf, delta=0.02)

    def whole_wait(r):
        _, _, pg = hj.hj_coproc_time(x, cpu_s, gpu_s, [0.0, r], xfer_s=xf)
        return max(pg, g1 * N + r * N * (xf + c2))

    # a fixed host hand-off for any CPU share (the copy thread's start, the
    # partition offsets' read-back, the final merge), which Eq. 1-5 have no term
    # for: fitted at one more share, 0.03, kept out of the checked shares
    F = max(0.0, med([run(0.03)[0]["total"] for _ in range(3)]) - whole_wait(0.03))
    # the model against measured times at seeded random shares (and a few small ones)
    import random
    rnd = random.Random(1307)
    shares = sorted([0.005, 0.01, 0.02, 0.05] + [rnd.random() for _ in range(wl["shares"])])
    # Eq. 4 lets the CPU start step 2 once the GPU has produced its share of step 1
    # (r x T1); here the partition pass hands over every partition at its end, so the
    # CPU waits all of T1: the second prediction uses that wait
    pts, errs, errs_adj, errs_h = [], [], [], []
    for r in shares:
        meas = run(r)[0]["total"]
        pred, _, _ = hj.hj_coproc_time(x, cpu_s, gpu_s, [0.0, r], xfer_s=xf)
        pred_adj = whole_wait(r)
        pred_h = pred_adj + (F if r > 0 else 0.0)
        err, err_adj, err_h = (pred - meas) / meas, (pred_adj - meas) / meas, (pred_h - meas) / meas
        errs.append(abs(err))
        errs_adj.append(abs(err_adj))
        errs_h.append(abs(err_h))
        pts.append({"share": r, "measured_s": meas, "predicted_s": pred, "rel_err": err,
                    "predicted_whole_wait_s": pred_adj, "rel_err_whole_wait": err_adj,
                    "predicted_handoff_s": pred_h, "rel_err_handoff": err_h})
    # timed: the model's share
    share = ratios_best[1]
    sampler = ClockSampler(local)
    if not args.no_clocks:
        sampler.start()
        time.sleep(0.3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        tt, cnt = run(share)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop() if not args.no_clocks else None
    value = N * args.steps / (ms / 1000.0)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": wl["desc"], "cpu_share": share, "pairs_per_step": cnt,
                       "host_cores": host_cores(), "parallelism": f"replicas x{ws}",
                       "l2": "inputs 268 MB per step exceed the 129 MB L2; no flush"},
            "model": {"per_item_s": {"partition_gpu": g1, "join_gpu": g2, "join_cpu": c2, "copy_to_host": xf},
                      "best_shares": ratios_best, "best_predicted_s": t_best,
                      "mean_abs_rel_err": sum(errs) / len(errs), "max_abs_rel_err": max(errs),
                      "mean_abs_rel_err_whole_wait": sum(errs_adj) / len(errs_adj),
                      "max_abs_rel_err_whole_wait": max(errs_adj),
                      "handoff_s": F, "mean_abs_rel_err_handoff": sum(errs_h) / len(errs_h),
                      "max_abs_rel_err_handoff": max(errs_h),
                      "points_n": len(pts),
                      "by_share_decile": deciles(pts),
                      "points_sample": pts[:: max(1, len(pts) // 24)],
                      "measured_best": min(pts, key=lambda q: q["measured_s"])},
            "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    ctx.close()


def serve_pool(wl, rank, dev, pool_bytes: float):
    """Request sizes and arrival order of the whole stream, and the device inputs of
    its first K requests (K as large as pool_bytes allows); request i is served
    with the inputs and sizes of pool entry i mod K."""
    from paper_1307_1955_gb300 import workload as W

    seed = W.DEFAULT_SEED + rank
    specs = W.serving_specs(wl["nreq"], seed, 1.0)
    k, acc = 0, 0
    while k < len(specs) and acc + 8 * (specs[k].n_r + specs[k].n_s) <= pool_bytes:
        acc += 8 * (specs[k].n_r + specs[k].n_s)
        k += 1
    pool = specs[:k]
    R_all, S_all, rs, ss = W.batched_relations(pool, seed, dev, ids=(5,))
    reqs = [(R_all[rs[j]:rs[j] + sp.n_r], S_all[ss[j]:ss[j] + sp.n_s]) for j, sp in enumerate(pool)]
    return specs, pool, reqs, (R_all, S_all)


def run_serve(args, wl, ws, rank, local):
    """Serving: the request stream through hj_server (continuous batching over
    several streams, HBM admission budget) -- saturated, then Poisson arrivals at a
    fraction of the saturated rate (p50/p99 latency) -- against one hj_join call per
    request on one stream."""
    import torch
    import torch.distributed as dist

    import __graft_entry__

    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    from paper_1307_1955_gb300 import hj

    dev = torch.device("cuda", local)
    specs, pool, reqs, keep = serve_pool(wl, rank, dev, 40e9)
    K, n = len(pool), len(specs)
    order = [i % K for i in range(n)]
    tuples = [pool[j].n_r + pool[j].n_s for j in order]
    total = sum(tuples)
    ctx = hj.Context(local)
    # expected count of every pool entry: the same request alone
    want = []
    for R, S in reqs:
        res = hj.hj_join(ctx, R, S)
        want.append(res.count)
        res.free()
    torch.cuda.synchronize()

    def stream(srv, arrivals=None):
        """Submit requests (at their arrival times if given) from a client thread,
        collect them here; returns (makespan s, latencies s, mismatches)."""
        ids = [None] * n
        posted = [threading.Event() for _ in range(n)]

        def client():
            t0 = time.perf_counter()
            for i in range(n):
                if arrivals is not None:
                    d = arrivals[i] - (time.perf_counter() - t0)
                    if d > 0:
                        time.sleep(d)
                R, S = reqs[order[i]]
                ids[i] = srv.submit(R, S, sync=False)  # inputs were synchronised before the run
                posted[i].set()

        th = threading.Thread(target=client)
        lat, bad, first, last = [], 0, None, 0.0
        th.start()
        for i in range(n):
            posted[i].wait()
            res, t = srv.wait(ids[i], 600.0)
            bad += res.count != want[order[i]]
            res.free()
            lat.append(t.done - t.submit)
            first = t.submit if first is None else min(first, t.submit)
            last = max(last, t.done)
        th.join()
        return last - first, lat, bad

    def pct(xs, q):
        xs = sorted(xs)
        return xs[min(len(xs) - 1, int(math.ceil(q * len(xs))) - 1)]

    with hj.Server(ctx, budget=wl["budget"], workers=args.serve_workers, wave_tuples=args.serve_wave_tuples) as srv:
        # warm-up: the first requests of the stream
        for _ in range(args.warmup):
            for R, S in reqs[:min(K, 64)]:
                srv.wait(srv.submit(R, S, sync=False))[0].free()
        sampler = ClockSampler(local)
        if not args.no_clocks:
            sampler.start()
            time.sleep(0.3)
        l0 = srv.stats()["launches"]
        span, lat_sat, bad_sat = stream(srv)
        launches = srv.stats()["launches"] - l0
        clocks = sampler.stop() if not args.no_clocks else None
        sat = total / span
        # Poisson arrivals at `load` x the saturated request rate
        rate = wl["load"] * sat / (total / n)
        arrivals = [sp.arrival_s / rate for sp in specs]
        span_l, lat_l, bad_l = stream(srv, arrivals)
        # the same stream at lighter and heavier offered loads
        sweep = []
        for ld in (() if args.no_sweep else wl.get("sweep", ())):
            r_ = ld * sat / (total / n)
            span_x, lat_x, bad_x = stream(srv, [sp.arrival_s / r_ for sp in specs])
            sweep.append({"load": ld, "offered_req_per_s": r_, "tuples_per_s": total / span_x, "span_s": span_x,
                          "p50_ms": 1000 * pct(lat_x, 0.5), "p99_ms": 1000 * pct(lat_x, 0.99), "mismatches": bad_x})
        st = srv.stats()
    # one hj_join per request, one stream, same requests (bounded to ~20 s)
    t0 = time.perf_counter()
    done_t = 0
    for i in range(n):
        R, S = reqs[order[i]]
        hj.hj_join(ctx, R, S).free()
        done_t += tuples[i]
        if time.perf_counter() - t0 > args.plain_seconds:
            break
    torch.cuda.synchronize()
    plain = done_t / (time.perf_counter() - t0)
    peak, peak_kind = measured_peak()
    pairs = sum(want[j] for j in order)
    alg = 3 * 8 * total + 8 * pairs
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle over the stream's requests in order, about 12 s of work
        cpu = batch_cpu_sample([reqs[j][0] for j in order[:K]], [reqs[j][1] for j in order[:K]], 12.0)
    if rank == 0:
        line = {
            "metric": METRIC, "value": sat, "unit": UNIT, "n_gpus": ws, "steps": 1, "warmup": args.warmup,
            "ms_per_step": span * 1000.0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": wl["desc"], "requests": n, "distinct_inputs": K,
                       "inputs": f"request i uses the seeded inputs and sizes of request i mod {K} of the stream "
                                 f"(device-resident, generated before the run)",
                       "tuples": total, "pairs": pairs, "workers": args.serve_workers,
                       "wave_tuples": args.serve_wave_tuples or "default (2^26)", "budget_bytes": wl["budget"],
                       "parallelism": f"replicas x{ws}", "l2": "inputs far larger than the 129 MB L2; no flush"},
            "saturated": {"tuples_per_s": sat, "span_s": span, "p50_ms": 1000 * pct(lat_sat, 0.5),
                          "p99_ms": 1000 * pct(lat_sat, 0.99), "mismatches": bad_sat},
            "at_load": {"load": wl["load"], "offered_req_per_s": rate, "tuples_per_s": total / span_l,
                        "span_s": span_l, "p50_ms": 1000 * pct(lat_l, 0.5), "p99_ms": 1000 * pct(lat_l, 0.99),
                        "mismatches": bad_l},
            "load_sweep": sweep,
            "plain": {"value": plain, "unit": UNIT, "api": "hj_join once per request, one stream"},
            "served_vs_plain": sat / plain,
            "server": st,
            "roofline": {"bound": "hbm", "kernel": "whole join (all kernels)", "achieved": alg / span / 1e9,
                         "peak": peak, "unit": "GB/s", "frac": alg / span / 1e9 / peak, "peak_kind": peak_kind,
                         "traffic": None},
            "cpu_baseline": cpu, "e2e": None, "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    del keep
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def run_sweep(args, wl, ws, rank, local):
    """Throughput of the join over the paper's size and selectivity sweeps (each
    point autotuned, inputs resident, CUDA events around the timed joins)."""
    import torch

    import __graft_entry__

    torch.cuda.set_device(local)
    if rank == 0:
        __graft_entry__.build()
    from paper_1307_1955_gb300 import hj
    from paper_1307_1955_gb300 import workload as W

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = hj.Context(local, stream=stream)
    ns = wl["ns"]
    points = [(1 << lg, ns, 1 << lg, "size") for lg in (16, 18, 20, 22, 24)]
    points += [(wl["nr"], ns, int(wl["nr"] / sel), f"selectivity {sel:g}") for sel in (0.125, 0.5)]
    out, launches = [], 0
    steps = max(1, min(args.steps, 20))
    for nr, nsp, dom, kind in points:
        R, S = W.unique_and_uniform(nr, nsp, dom, W.DEFAULT_SEED + rank, dev, ids=(6, nr, dom))
        plan = hj.hj_tune(ctx, R, S)
        for _ in range(args.warmup):
            hj.hj_join(ctx, R, S).free()
        torch.cuda.synchronize()
        l0 = hj.launch_count(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            res = hj.hj_join(ctx, R, S)
            m = res.count
            res.free()
        e1.record(stream)
        torch.cuda.synchronize()
        launches += hj.launch_count(ctx) - l0
        ms = e0.elapsed_time(e1) / steps
        out.append({"sweep": kind, "nr": nr, "ns": nsp, "selectivity": round(min(1.0, nr / dom), 4), "pairs": m,
                    "algo": {1: "SHJ", 2: "PHJ"}[plan["algo"]], "radix_bits": plan["radix_bits"],
                    "passes": plan["passes"], "ms": ms, "tuples_per_s": (nr + nsp) / (ms / 1000.0)})
        del R, S
    head = [p for p in out if p["nr"] == wl["nr"] and p["selectivity"] == 1.0][0]
    if rank == 0:
        line = {
            "metric": METRIC, "value": head["tuples_per_s"], "unit": UNIT, "n_gpus": ws, "steps": steps,
            "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": wl["desc"], "parallelism": f"replicas x{ws}",
                       "l2": "the larger points exceed the 129 MB L2; no flush"},
            "points": out, "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    ctx.close()


def run_outcore(args, wl, ws, rank, local):
    """hj_join_host_large on pinned host relations with a device budget far below
    their size; the whole call (copies both ways, partitioning, joins) is timed."""
    import torch

    import __graft_entry__

    torch.cuda.set_device(local)
    if rank == 0:
        __graft_entry__.build()
    from paper_1307_1955_gb300 import hj
    from paper_1307_1955_gb300 import workload as W

    dev = torch.device("cuda", local)
    R, S = make_inputs(wl, rank, dev)
    Rh, Sh = R.cpu().pin_memory(), S.cpu().pin_memory()
    del R, S
    ctx = hj.Context(local)
    out = torch.empty((wl["ns"] + (1 << 20), 2), dtype=torch.int32).pin_memory()
    for _ in range(args.warmup):
        res = hj.hj_join_host_large(ctx, Rh, Sh, out, device_bytes=wl["budget"])
    steps = max(1, min(args.steps, 5))
    l0 = hj.launch_count(ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        res = hj.hj_join_host_large(ctx, Rh, Sh, out, device_bytes=wl["budget"])
    torch.cuda.synchronize()
    dt = ranks_max(time.perf_counter() - t0, ws, dev)
    value = weak_value(wl["nr"] + wl["ns"], steps, ws, dt * 1000.0)
    launches = hj.launch_count(ctx) - l0
    plan = {"passes": res.passes, "radix_bits": res.radix_bits,
            "kind": "R resident, S streamed" if res.passes == 1 else "split (App. A)"}
    # the paper's split of both relations through the same budget, forced
    lib = hj.load_library()
    lib.hj_debug_outcore(ctx.handle, hj.HJ_OUTCORE_SPLIT)
    res_split = hj.hj_join_host_large(ctx, Rh, Sh, out, device_bytes=wl["budget"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        res_split = hj.hj_join_host_large(ctx, Rh, Sh, out, device_bytes=wl["budget"])
    torch.cuda.synchronize()
    split_ms = ranks_max(time.perf_counter() - t0, ws, dev) * 1000.0 / steps
    lib.hj_debug_outcore(ctx.handle, hj.HJ_OUTCORE_AUTO)
    if res_split.count != res.count:
        raise RuntimeError(f"split plan counted {res_split.count} pairs, the streamed plan {res.count}")
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_sample(wl, Rh, Sh, target_s=12.0)
    if rank == 0:
        tb = 8
        # every tuple crosses the link once when R stays on the device, R + S in and
        # R + S home again before the second crossing in when both are split
        if res.passes == 1:
            h2d, d2h = tb * (wl["nr"] + wl["ns"]), tb * res.count
        else:
            h2d, d2h = 2 * tb * (wl["nr"] + wl["ns"]), tb * (wl["nr"] + wl["ns"]) + tb * res.count
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": steps, "warmup": args.warmup,
            "ms_per_step": dt * 1000.0 / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": wl["desc"], "device_bytes": wl["budget"], "plan": plan,
                       "pairs_per_step": res.count, "parallelism": f"replicas x{ws}",
                       "l2": "host-resident inputs of 2.28 GB; no flush"},
            "host_traffic_per_step": {"h2d_bytes": h2d, "d2h_bytes": d2h},
            "split_ms_per_step": split_ms,
            "split_top_bits": res_split.radix_bits,
            "split_host_traffic_per_step": {"h2d_bytes": 2 * tb * (wl["nr"] + wl["ns"]),
                                            "d2h_bytes": tb * (wl["nr"] + wl["ns"]) + tb * res.count},
            "roofline": None, "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "api": "hj_join_host_large"},
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    ctx.close()


# Other configurations, measured after the default workload's line is computed (N=1 only), each in a
# process of its own so that the previous run's device memory is gone: the batched joins, the served
# request stream and the skewed 64-bit joins.  Their summaries ride on the default line ("also").
EXTRAS = (
    ("batched", ["--workload", "batch_4096", "--steps", "5", "--warmup", "2", "--plain-steps", "1"]),
    ("served", ["--workload", "serve_20000", "--warmup", "1", "--plain-seconds", "8", "--no-sweep"]),
    ("skewed_u64_theta_0.5", ["--workload", "zipf_4m_64m_t05", "--steps", "10", "--warmup", "3", "--no-e2e"]),
    ("skewed_u64_theta_1.0", ["--workload", "zipf_4m_64m_t10", "--steps", "10", "--warmup", "3", "--no-e2e"]),
)


def run_extras() -> dict:
    """Run every EXTRAS configuration through this script and keep a summary of its
    JSON line (throughput, its comparison, latency and roofline figures)."""
    out = {}
    for name, extra in EXTRAS:
        cmd = [sys.executable, os.path.abspath(__file__), *extra, "--no-cpu-baseline", "--no-clocks", "--no-extras"]
        t0 = time.perf_counter()
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
            lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
            if r.returncode != 0 or not lines:
                out[name] = {"error": f"exit {r.returncode}: {(r.stderr or r.stdout)[-300:]}"}
                continue
            d = json.loads(lines[-1])
        except Exception as e:  # a failed extra leaves the default line intact
            out[name] = {"error": repr(e)[:300]}
            continue
        rec = {"value": d["value"], "unit": d["unit"], "ms_per_step": d["ms_per_step"], "steps": d["steps"],
               "workload": d["config"]["workload"], "wall_s": round(time.perf_counter() - t0, 1),
               "cmd": "python bench.py " + " ".join(extra)}
        if "roofline" in d and d["roofline"]:
            rec["roofline_frac"] = d["roofline"].get("frac")
            rec["roofline_kernel"] = d["roofline"].get("kernel")
        if "join_roofline" in d:
            rec["join_roofline_frac"] = d["join_roofline"].get("frac")
        if "batched_vs_plain" in d:
            rec.update(plain_value=d["plain"]["value"], batched_vs_plain=d["batched_vs_plain"],
                       joins=d["config"]["joins"], pairs_per_step=d["config"]["pairs_per_step"])
        if "served_vs_plain" in d:
            rec.update(plain_value=d["plain"]["value"], served_vs_plain=d["served_vs_plain"],
                       requests=d["config"]["requests"], saturated=d["saturated"], at_load=d["at_load"])
        if d.get("config", {}).get("mode"):
            rec["mode"] = d["config"]["mode"]
            rec["pairs_per_step"] = d["config"].get("pairs_per_step")
        out[name] = rec
    return out


def main():
    args = parse()
    ws, rank, local = dist_env()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl, ws, rank)
    elif wl.get("kind") == "serve":
        run_serve(args, wl, ws, rank, local)
    elif wl.get("kind") == "sweep":
        run_sweep(args, wl, ws, rank, local)
    elif wl.get("kind") == "outcore":
        run_outcore(args, wl, ws, rank, local)
    elif wl.get("kind") == "batch":
        run_batch(args, wl, ws, rank, local)
    elif wl.get("kind") == "sharded":
        run_sharded(args, wl, ws, rank, local)
    elif wl.get("kind") == "coproc":
        run_coproc(args, wl, ws, rank, local)
    else:
        run_hj(args, wl, ws, rank, local)


if __name__ == "__main__":
    main()
