#!/usr/bin/env python
"""Benchmark of the matrix-profile sweep (distance-matrix cells per second).

Workload (default): the pure-Euclidean matrix profile (AAMP, Algorithm 1) of
a float32 random walk of n = 2^20 samples with 20 Gaussian bumps, m = 256,
exclusion zone m / 4 = 64: N = 1,048,321 windows and 549,420,844,896 cells
(unordered pairs with |i - j| > 64).  A step is one full mp_aamp call on
device-resident T: conversion, diagonal sweep, FP64 polish, P and I.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank computes its own
series (seed + rank): weak scaling, no collective on the data path; with
--shard the ranks split one series' diagonals (Algorithm 1's k loop) and
merge the partial profiles with two MIN all-reduces: strong scaling.
--impl reference times the FP64 CPU oracle (Algorithm 1, OpenMP over the
host cores) on a bounded diagonal range of the same series.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1901_05708_gb300 import workloads as W  # noqa: E402

METRIC = "distance-matrix cells/s (GCells/s) at 1 GB300 + % FP32 roofline, FP32 vs FP64 sweep"
UNIT = "GCells/s"
FP32_INSTR_PER_CELL = 4          # minimum FP32-pipe instructions per cell (Lemma 1 update)
FP32_LANES_PER_SM = 128
CSRC = os.path.join(ROOT, "paper_1901_05708_gb300", "csrc")
# the sources that make up each workload's sweep kernel (their hash names the kernel version)
SWEEP_SOURCES = {
    "euclid": ["mp_device.cuh", "mp_sweep2.cuh", "k_sweep2.cu", "k_sweep2_tall.cu"],
    "pnorm": ["mp_device.cuh", "mp_sweep2.cuh", "k_sweep2_p13.cu", "mp_sweep_z2.cuh", "k_sweepz.cu"],
    "znorm": ["mp_device.cuh", "mp_sweep2.cuh", "mp_sweep_z2.cuh", "k_sweepz.cu"],
}


def kernel_version(dist_name: str) -> str:
    """Hash of the sources of the sweep kernel a workload runs."""
    import hashlib
    h = hashlib.sha1()
    for f in SWEEP_SOURCES[dist_name]:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def sweep_dram_bytes(workload: str, n: int, version: str):
    """DRAM bytes (read + write) of one sweep launch from the committed ncu
    summaries under profiles/: a line
      dram_bytes_per_launch: workload=<name> n=<n> kernel=<version> bytes=<B>
    recorded for this workload, size and kernel version; None when the kernel
    has changed since its last capture."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for line in f:
                line = line.strip().strip("`")
                if not line.startswith("dram_bytes_per_launch:"):
                    continue
                kv = dict(x.split("=", 1) for x in line.split(":", 1)[1].split())
                if kv.get("workload") == workload and int(kv.get("n", -1)) == n and kv.get("kernel") == version:
                    return int(kv["bytes"])
    return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples taken while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(series: W.Series, target_s: float = 12.0):
    """Time the FP64 oracle (Algorithm 1, all host cores) on a diagonal range
    of the series sized to take about target_s seconds."""
    import oracle
    oracle.build()
    T = series.T.astype(np.float64)
    k0 = series.excl + 1

    def sweep(k_range):
        if series.dist == W.EUCLID:
            return oracle.aamp(T, series.m, series.excl, k_range=k_range)
        if series.dist == W.PNORM:
            return oracle.pnorm(T, series.m, series.excl, series.p, k_range=k_range)
        return oracle.acamp_centred(T, series.m, series.excl, k_range=k_range)

    # calibrate on a short range, then grow the range until the run takes at
    # least half the target (thread start-up makes short calibrations pessimistic)
    K = min(256, max(1, series.N - k0))
    while True:
        t0 = time.perf_counter()
        ref = sweep((k0, k0 + K))
        dt = time.perf_counter() - t0
        if dt >= 0.5 * target_s or K >= series.N - k0:
            break
        K = int(min(series.N - k0, max(2 * K, K * target_s / max(dt, 1e-3))))
    cells = sum(series.N - k for k in range(k0, k0 + K))
    return {"value": cells / dt / 1e9, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{series.name}: diagonals {k0}..{k0 + K - 1} ({cells:.3e} cells) in {dt:.2f} s",
            "cpu": cpu_model(), "seconds": dt, "cells": cells, "k_range": (k0, k0 + K), "ref": ref}


def slice_error(torch, mp, series: W.Series, T, dname: str, cb: dict) -> dict:
    """The FP32 profile of the oracle's timed diagonal slice, raw (polish off)
    and polished, against the oracle's FP64 partial profile of the same slice,
    over every row the slice reaches: the largest relative error of P (with
    the oracle's P at that row), the largest error in units of the FP32
    acceptance bound 1e-5 P_ref + atol (atol = 1e-5 m^(1/p) sd(diff T) for
    the pure and p-norm distances, 1e-5 sqrt(m) for the z-normalised one; at
    most 1 is within it), and the rows whose index differs (a near-tie can
    legitimately differ)."""
    Pr, Ir = cb["ref"]
    fin = np.isfinite(Pr) & (Pr > 0)
    rtol = 1e-5
    if series.dist == W.ZNORM:
        atol = rtol * math.sqrt(series.m)
    else:
        atol = rtol * series.m ** (1.0 / series.p) * float(np.std(np.diff(series.T.astype(np.float64))))
    out = {"diagonals": list(cb["k_range"]), "rows": int(fin.sum())}
    for polish in (False, True):
        P, I = mp.profile(T, series.m, series.excl, dname, series.p, k_range=cb["k_range"], polish=polish)
        torch.cuda.synchronize()
        mp.sync_status()
        P, I = P.cpu().numpy()[fin], I.cpu().numpy()[fin]
        key = "polished" if polish else "raw"
        if P.size:
            err = np.abs(P - Pr[fin])
            w = int(np.argmax(err / Pr[fin]))
            out[f"{key}_max_rel_err"] = float(err[w] / Pr[fin][w])
            out[f"{key}_max_rel_err_at_P"] = float(Pr[fin][w])
            out[f"{key}_max_over_bound"] = float(np.max(err / (rtol * Pr[fin] + atol)))
        if polish:
            out["index_mismatch"] = int(np.sum(I != Ir[fin]))
    return out


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    if args.workload == "batch_4096":
        b = W.batch_4096()
        series = max(b.series, key=lambda x: x.n)  # the oracle's sample: the longest series
        config = batch_config(b)
    else:
        make, desc, _ = WORKLOADS[args.workload]
        series = make(1, args.n)
        config = workload_config(series, desc)
    runs = []
    for _ in range(max(0, args.warmup_ref)):
        oracle_sample(series, target_s=2.0)
    for _ in range(args.steps):
        runs.append(oracle_sample(series, target_s=args.ref_seconds))
    cells = sum(r["cells"] for r in runs)
    secs = sum(r["seconds"] for r in runs)
    value = cells / secs / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, len(runs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(config, precision="fp64 CPU oracle (OpenMP over diagonals)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": runs[0]["cores"], "kind": "oracle",
                             "sample": runs[0]["sample"], "cpu": runs[0]["cpu"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


WORKLOADS = {
    # name: (series factory, description, FP32-pipe instructions per cell at minimum)
    "aamp_1m": (lambda seed, n: W.aamp_1m(seed=seed, n=n),
                "AAMP pure Euclidean, float32 random walk + 20 Gaussian bumps", 4),
    "acamp_1m": (lambda seed, n: W.acamp_1m(seed=seed + 2, n=n),
                 "ACAMP z-normalised, float32 random walk + N(0, 0.01)", 4),
    "pnorm_p1": (lambda seed, n: W.pnorm_262k(1.0, seed=seed + 1, n=min(n, 1 << 18)),
                 "p-norm p = 1, float32 sine + motifs + flat run", 4),
    "pnorm_p3": (lambda seed, n: W.pnorm_262k(3.0, seed=seed + 1, n=min(n, 1 << 18)),
                 "p-norm p = 3, float32 sine + motifs + flat run", 6),
    "aamp_small": (lambda seed, n: W.aamp_small(seed=seed - 1),
                   "AAMP pure Euclidean, float64 random walk, n = 10,000", 4),
}
# the paper's timing data (Sec. 5.1): i.i.d. uniform series, n = 2^18, m from 2^8 to 2^16
for _lg in (8, 10, 12, 14, 16):
    WORKLOADS[f"uniform_m{1 << _lg}"] = (
        (lambda lg: lambda seed, n: W.Series(f"uniform_n262144_m{1 << lg}", W.uniform(1 << 18, seed + 4), 1 << lg,
                                             W.excl_zone(1 << lg), W.EUCLID))(_lg),
        f"AAMP pure Euclidean, i.i.d. uniform values, n = 2^18, m = 2^{_lg}", 4)


# the paper's other timing shape (Sec. 5.1): i.i.d. uniform series, m = 2^8, n from 2^14 to 2^20, both distances
for _lg in range(14, 21):
    WORKLOADS[f"s1_aamp_n{1 << _lg}"] = (
        (lambda lg: lambda seed, n: W.Series(f"uniform_n{1 << lg}_m256", W.uniform(1 << lg, seed + 4), 256,
                                             W.excl_zone(256), W.EUCLID))(_lg),
        f"AAMP pure Euclidean, i.i.d. uniform values, n = 2^{_lg}, m = 256", 4)
    WORKLOADS[f"s1_acamp_n{1 << _lg}"] = (
        (lambda lg: lambda seed, n: W.Series(f"uniform_n{1 << lg}_m256", W.uniform(1 << lg, seed + 4), 256,
                                             W.excl_zone(256), W.ZNORM))(_lg),
        f"ACAMP z-normalised, i.i.d. uniform values, n = 2^{_lg}, m = 256", 4)


def workload_config(series: W.Series, desc: str = WORKLOADS["aamp_1m"][1], precision: str = "fp32") -> dict:
    prec = ("fp32 sweep (re-anchored / compensated), fp64 polish" if precision == "fp32"
            else "fp64 sweep, fp64 polish")
    return {"workload": f"{series.name} ({desc})",
            "n": series.n, "m": series.m, "excl": series.excl, "N": series.N,
            "cells_per_step": series.cells, "precision": prec,
            "l2": "flushed before every timed step (512 MiB write)"}


def batch_config(b: W.Batch) -> dict:
    ns = np.array([x.n for x in b.series])
    return {"workload": f"{b.name} (4,096 float32 random walks, m in {{32, 64, 128}}, "
                        f"half Euclidean / half z-normalised, one graph launch)",
            "series": len(b.series), "samples": int(ns.sum()), "cells_per_step": int(b.cells),
            "precision": "fp32 sweep (re-anchored / compensated), fp64 polish",
            "l2": "inputs (553 MB) and outputs larger than L2; L2 flushed before every timed step"}


def bench_batch(args, torch, mp, lib, dev, stream, rank, ws):
    """The 4,096-series batch: one mp_batch_run (one graph launch) per step."""
    b = W.batch_4096(seed=4 + rank)
    plan = mp.BatchPlan([x.n for x in b.series], [x.m for x in b.series], [x.dist for x in b.series],
                        [x.excl for x in b.series])
    T_host = torch.from_numpy(np.concatenate([x.T for x in b.series]).astype(np.float32)).pin_memory()
    T = T_host.to(dev)
    P = torch.empty(plan.windows, dtype=torch.float64, device=dev)
    I = torch.empty(plan.windows, dtype=torch.int64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        plan.run(T, out=(P, I))
    torch.cuda.synchronize()
    mp.sync_status()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = lib.mp_launch_count()
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        ev[k][0].record(stream)
        plan.run(T, out=(P, I))
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = lib.mp_launch_count() - launches0
    clk = clocks.stop()
    mp.sync_status()
    step_ms = [a.elapsed_time(c) for a, c in ev]
    total_ms = float(sum(step_ms))
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    cells = b.cells
    value = ws * cells * args.steps / (total_ms * 1e-3) / 1e9

    # end to end: host series in, host profiles out
    P_host = torch.empty(plan.windows, dtype=torch.float64).pin_memory()
    I_host = torch.empty(plan.windows, dtype=torch.int64).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(e2e_steps):
        T.copy_(T_host, non_blocking=True)
        plan.run(T, out=(P, I))
        P_host.copy_(P, non_blocking=True)
        I_host.copy_(I, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_value = ws * cells / (e2e_ms * 1e-3) / 1e9

    pk, src = peaks()
    f_max = float(pk.get("sm_max_mhz", 2070.0)) * 1e6
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_cells = sms * FP32_LANES_PER_SM * f_max / FP32_INSTR_PER_CELL / 1e9
    achieved = cells / (total_ms / args.steps * 1e-3) / 1e9
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_cells, "unit": UNIT,
            "frac": achieved / peak_cells, "traffic": None,
            "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {f_max/1e6:.0f} MHz "
                           f"({src} sm_max_mhz) / {FP32_INSTR_PER_CELL} FP32 instructions per cell",
            "kernel": "whole batch graph (statistics, persistent sweeps, finalize): a lower bound "
                      "for the sweep kernels", "kernel_ms": total_ms / args.steps,
            "tiles": plan.tiles}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": batch_config(b), "roofline": roof, "clocks": clk, "gpu_launches": int(launches),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(T_host.numel() * 4),
                    "d2h_bytes_per_step": int(plan.windows * 16), "ms_per_step": e2e_ms}}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        longest = max(b.series, key=lambda x: x.n)
        cb = oracle_sample(longest, target_s=args.ref_seconds)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "cpu")}
    elif rank == 0:
        line["cpu_baseline"] = None
    plan.close()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--warmup-ref", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--workload", default="aamp_1m", choices=sorted(WORKLOADS) + ["batch_4096"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--k-range", type=int, nargs=2, default=None,
                    help="sweep only diagonals [k0, k1) (for timing the FP64 sweep on a slice)")
    ap.add_argument("--shard", action="store_true",
                    help="split one series' diagonals over the ranks and merge (strong scaling); "
                         "default: every rank its own series (weak scaling)")
    ap.add_argument("--tile-rows", type=int, default=0,
                    help="mp_options.tile_rows of the FP32 sweep (0: the library's choice)")
    ap.add_argument("--fp64-diagonals", type=int, default=8192,
                    help="also time the FP64 sweep on this many diagonals (0: skip)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_1901_05708_gb300 import mp

    ws, rank, local = dist_env()
    if args.gpus != ws:
        raise SystemExit(f"--gpus {args.gpus} but {ws} ranks: launch N > 1 with torch.distributed.run "
                         f"--nproc-per-node N (one rank per GPU)")
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = mp.load()

    if args.workload == "batch_4096":
        line = bench_batch(args, torch, mp, lib, dev, torch.cuda.current_stream(dev), rank, ws)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if ws > 1:
            dist.destroy_process_group()
        return
    make, desc, instr_per_cell = WORKLOADS[args.workload]
    shard_range = None
    if args.shard:  # one series, its diagonals split over the ranks (strong scaling)
        from paper_1901_05708_gb300 import shard as SH
        series = make(1, args.n)
        shard_range = SH.diagonal_ranges(series.excl + 1, series.N, ws)[rank]
    else:           # every rank its own series (weak scaling)
        series = make(1 + rank, args.n)
    dname = {W.EUCLID: "euclid", W.PNORM: "pnorm", W.ZNORM: "znorm"}[series.dist]
    T_host = torch.from_numpy(series.T).pin_memory()
    T = T_host.to(dev)
    N = series.N
    P = torch.empty(N, dtype=torch.float64, device=dev)
    I = torch.empty(N, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    kw = {"precision": args.precision}
    if args.tile_rows:
        kw["tile_rows"] = args.tile_rows
    if args.k_range:
        kw["k_range"] = tuple(args.k_range)
    if shard_range is not None:
        kw["k_range"] = shard_range

    def step(Tin=None):
        mp.profile(T if Tin is None else Tin, series.m, series.excl, dname, series.p, out=(P, I), **kw)
        if shard_range is not None and ws > 1:  # the one exchange: two MIN all-reduces of the partial profiles
            Pm, Im = SH.allreduce_merge(P, I)
            P.copy_(Pm)
            I.copy_(Im)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    mp.sync_status()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sw = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for a, b in sw:  # create the CUDA events now (torch makes them on first record)
        a.record(stream)
        b.record(stream)
    clocks = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = lib.mp_launch_count()
    for k in range(args.steps):
        flush.fill_(k & 0xff)  # L2 flush, outside the timed events
        lib.mp_set_sweep_events(ctypes_event(sw[k][0]), ctypes_event(sw[k][1]))
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    lib.mp_set_sweep_events(None, None)
    torch.cuda.synchronize()
    launches = lib.mp_launch_count() - launches0
    clk = clocks.stop()
    mp.sync_status()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    sweep_ms = [a.elapsed_time(b) for a, b in sw]
    total_ms = float(sum(step_ms))
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()

    cells = series.cells
    if args.k_range:
        lo, hi = max(args.k_range[0], series.excl + 1), min(args.k_range[1], series.N)
        cells = sum(series.N - k for k in range(lo, hi))
    job_cells = cells if shard_range is not None else ws * cells  # cells of the whole job per step
    if shard_range is not None:  # this rank's own diagonals (for its sweep kernel's roofline)
        lo, hi = shard_range
        cells = (hi - lo) * (2 * series.N - lo - hi + 1) // 2
    value = job_cells * args.steps / (total_ms * 1e-3) / 1e9

    # ---- end to end through the public API with host buffers -------------------
    P_host = torch.empty(N, dtype=torch.float64).pin_memory()
    I_host = torch.empty(N, dtype=torch.int64).pin_memory()
    T_dev2 = torch.empty_like(T)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(e2e_steps):
        T_dev2.copy_(T_host, non_blocking=True)
        step(T_dev2)
        P_host.copy_(P, non_blocking=True)
        I_host.copy_(I, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_value = job_cells / (e2e_ms * 1e-3) / 1e9

    # ---- the FP64 sweep on a slice of the same diagonals (kernel events only) ----------
    fp64 = None
    if args.precision == "fp32" and not args.k_range and shard_range is None and args.fp64_diagonals > 0:
        k0 = series.excl + 1
        k1 = min(series.N, k0 + args.fp64_diagonals)
        kw64 = {"precision": "fp64", "k_range": (k0, k1)}
        mp.profile(T, series.m, series.excl, dname, series.p, out=(P, I), **kw64)  # warm-up
        ms64 = []
        for k in range(2):
            flush.fill_(k & 0xff)
            lib.mp_set_sweep_events(ctypes_event(sw[k][0]), ctypes_event(sw[k][1]))
            mp.profile(T, series.m, series.excl, dname, series.p, out=(P, I), **kw64)
            lib.mp_set_sweep_events(None, None)
            torch.cuda.synchronize()
            ms64.append(sw[k][0].elapsed_time(sw[k][1]))
        mp.sync_status()
        cells64 = sum(series.N - k for k in range(k0, k1))
        g64 = cells64 / (float(np.mean(ms64)) * 1e-3) / 1e9
        fp64 = {"value": g64, "unit": UNIT, "diagonals": [k0, k1], "cells": cells64,
                "kernel_ms": float(np.mean(ms64)),
                "what": "FP64 sweep kernel alone (no re-anchoring needed), same series, first diagonals"}

    # ---- roofline of the dominant kernel (the diagonal sweep) ------------------------
    pk, src = peaks()
    f_max = float(pk.get("sm_max_mhz", 2070.0)) * 1e6
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_cells = sms * FP32_LANES_PER_SM * f_max / instr_per_cell / 1e9
    sweep_avg_ms = float(np.mean(sweep_ms))
    achieved = cells / (sweep_avg_ms * 1e-3) / 1e9
    version = kernel_version(dname)
    traffic = None if args.k_range else sweep_dram_bytes(args.workload, args.n, version)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_cells, "unit": UNIT,
            "frac": achieved / peak_cells, "traffic": traffic,
            "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {f_max/1e6:.0f} MHz "
                           f"({src} sm_max_mhz) / {instr_per_cell} FP32 instructions per cell",
            "kernel": "diagonal sweep (a3-a5)", "kernel_ms": sweep_avg_ms, "kernel_version": version}
    if traffic is not None:
        algo = {"euclid": "the series and the keys once: 4n + 8N bytes",
                "pnorm": "the series and the keys once: 4n + 8N bytes",
                "znorm": "the series, the FP32 operands (df, dg, inv, float-float means) and the keys once: "
                         "4n + 28N bytes"}
        roof["traffic_note"] = ("bytes per launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum) of this "
                                "kernel version; algorithmic: " + algo[dname])
    if series.dist == W.EUCLID and series.p == 2.0:
        # the FLOP convention: 6 flops per cell (2 FADD, 2 FMUL, 2 FADD for s += e^2 - f^2) against
        # 2 flops per lane per cycle; its ceiling is 6 / (2 x 4) = 0.75 by construction
        roof["flop_convention"] = {"flops_per_cell": 6, "ceiling": 0.75,
                                   "frac": achieved * 6 / (sms * FP32_LANES_PER_SM * 2 * f_max / 1e9)}
    if clk.get("sm_mhz"):
        roof["frac_at_measured_clock"] = achieved / (sms * FP32_LANES_PER_SM * clk["sm_mhz"] * 1e6
                                                     / instr_per_cell / 1e9)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if shard_range is not None else "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic", "config": workload_config(series, desc, args.precision), "roofline": roof,
            "clocks": clk,
            "gpu_launches": int(launches),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(T_host.numel() * T_host.element_size()),
                    "d2h_bytes_per_step": int(N * 16), "ms_per_step": e2e_ms}}
    if args.k_range:
        line["config"]["k_range"] = list(args.k_range)
    if args.tile_rows:
        line["config"]["tile_rows"] = args.tile_rows
    if shard_range is not None:
        line["config"]["parallelism"] = f"diagonal ranges over {ws} ranks, merged by two MIN all-reduces"
        line["config"]["rank0_diagonals"] = list(shard_range)
    if fp64 is not None:
        fp64["fp32_over_fp64"] = achieved / fp64["value"]
        line["fp64_sweep"] = fp64
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb = oracle_sample(series, target_s=args.ref_seconds)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "cpu")}
        if args.precision == "fp32" and not args.k_range:
            # outside the timed regions: the FP32 path's error on the oracle's own slice
            line["cpu_baseline"]["fp32_error_on_sample"] = slice_error(torch, mp, series, T, dname, cb)
    elif rank == 0:
        line["cpu_baseline"] = None  # timed on rank 0 at N = 1 only
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def ctypes_event(e):
    """The cudaEvent_t handle of a (recorded) torch.cuda.Event as a void*."""
    import ctypes
    h = getattr(e, "cuda_event", 0)
    if not h:
        raise RuntimeError("torch.cuda.Event has no CUDA handle yet")
    return ctypes.c_void_p(h)


if __name__ == "__main__":
    main()
