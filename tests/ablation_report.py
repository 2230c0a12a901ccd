#!/usr/bin/env python
"""Precision / speed ablation of the z-normalised sweep's forms (needs a GPU).

On the C4 generator (random walk + N(0, 0.01)) at n = 2^18, m = 512: the
sweep kernel's time (CUDA events around it) and the raw sweep value's error
(polish off) against the FP64 oracle's brute force on seeded rows, for
  - the centred covariance in the FP32 fast kernel (the product),
  - the centred covariance in the FP32 and FP64 plain sweeps,
  - Algorithm 2's raw sums (MP_VARIANT_ZRAW) in FP32 and FP64,
  - Sec. 4.3's F comparison on the raw sums (MP_VARIANT_ZF) in FP32 and FP64.

    python tests/ablation_report.py [--n 262144] [--rows 64]

Prints one JSON line per form and a markdown table.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1901_05708_gb300 import workloads as W  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1 << 18)
    ap.add_argument("--rows", type=int, default=64)
    args = ap.parse_args()
    import torch
    from paper_1901_05708_gb300 import mp
    lib = mp.load()
    s = W.acamp_1m(n=args.n)
    rows = np.sort(np.random.default_rng(13).choice(s.N, args.rows, replace=False))
    Pr, Ir, _ = oracle.brute_rows(s.T, s.m, s.excl, rows, "znorm")
    T = torch.from_numpy(s.T).cuda()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream()
    e0.record(st)
    e1.record(st)
    forms = [("centred, FP32 fast kernel (the product)", "fp32", 0, False),
             ("centred, FP32 plain sweep", "fp32", 0, True),
             ("raw sums, FP32 plain sweep", "fp32", mp.MP_VARIANT_ZRAW, False),
             ("F comparison, FP32 plain sweep", "fp32", mp.MP_VARIANT_ZF, False),
             ("centred, FP64 plain sweep", "fp64", 0, False),
             ("raw sums, FP64 plain sweep", "fp64", mp.MP_VARIANT_ZRAW, False),
             ("F comparison, FP64 plain sweep", "fp64", mp.MP_VARIANT_ZF, False)]
    out = []
    for name, prec, variant, generic in forms:
        if generic:
            os.environ["MP_FORCE_GENERIC"] = "1"
        try:
            mp.acamp(T, s.m, s.excl, precision=prec, variant=variant, polish=False)  # warm-up
            lib.mp_set_sweep_events(ctypes.c_void_p(e0.cuda_event), ctypes.c_void_p(e1.cuda_event))
            P, I = mp.acamp(T, s.m, s.excl, precision=prec, variant=variant, polish=False)
            lib.mp_set_sweep_events(None, None)
            torch.cuda.synchronize()
            mp.sync_status()
        finally:
            os.environ.pop("MP_FORCE_GENERIC", None)
        ms = e0.elapsed_time(e1)
        P, I = P.cpu().numpy()[rows], I.cpu().numpy()[rows]
        rel = np.abs(P - Pr) / Pr
        r = {"form": name, "gcells": s.cells / (ms * 1e-3) / 1e9, "sweep_ms": ms,
             "max_rel_err": float(rel.max()), "median_rel_err": float(np.median(rel)),
             "i_mismatch": int(np.sum(I != Ir)), "rows": int(rows.size)}
        out.append(r)
        print(json.dumps(r), flush=True)
    print(f"\n| sweep (n = {args.n}, m = {s.m}) | Gcells/s | max / median relative error of P (raw) | "
          f"I != oracle (of {rows.size}) |")
    print("|---|---|---|---|")
    for r in out:
        print(f"| {r['form']} | {r['gcells']:,.1f} | {r['max_rel_err']:.1e} / {r['median_rel_err']:.1e} | "
              f"{r['i_mismatch']} |")


if __name__ == "__main__":
    main()
