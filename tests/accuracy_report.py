#!/usr/bin/env python
"""Per-workload error of the GPU profile against the FP64 oracle (needs a GPU).

For each workload configuration: the maximum relative error of P on the
checked rows for the FP32 sweep's raw value (polish off) and for the polished
profile (the default), the same for the FP64 sweep (on a diagonal slice for
the million-point series), and the number of rows whose index differs from the
oracle's.  Rows: every row of the 10,000-point series, seeded samples of rows
(brute force of the whole row) for the others, as in tests/test_gpu_configs.py.

    python tests/accuracy_report.py [--rows 48] [--json out.json]

Prints a markdown table; the test-suite asserts the same quantities against
the tolerances, this script only reports them.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import oracle  # noqa: E402
from paper_1901_05708_gb300 import workloads as W  # noqa: E402
from test_gpu_configs import sample_rows, slice_brute  # noqa: E402

NAMES = {W.EUCLID: "euclid", W.PNORM: "pnorm", W.ZNORM: "znorm"}


def rel_err(P, rows, ref):
    fin = np.isfinite(ref) & (ref > 0)
    if not fin.any():
        return 0.0
    return float(np.max(np.abs(P[rows][fin] - ref[fin]) / ref[fin]))


def run(mp, torch, s, **kw):
    T = torch.from_numpy(np.ascontiguousarray(s.T)).cuda()
    P, I = mp.profile(T, s.m, s.excl, NAMES[s.dist], s.p, **kw)
    torch.cuda.synchronize()
    mp.sync_status()
    return P.cpu().numpy(), I.cpu().numpy()


def report(nrows: int):
    import torch
    from paper_1901_05708_gb300 import mp
    mp.load()
    configs = [("C1 aamp_small", W.aamp_small(), None),
               ("C2 aamp_1m", W.aamp_1m(), 2000),
               ("C3 pnorm p=1", W.pnorm_262k(1.0), 2000),
               ("C3 pnorm p=3", W.pnorm_262k(3.0), 2000),
               ("C4 acamp_1m", W.acamp_1m(), 600)]
    out = []
    for name, s, kslice in configs:
        dist = NAMES[s.dist]
        rows = np.arange(s.N) if s.N <= 10_000 else sample_rows(s.N, nrows, 13)
        Pr, Ir, _ = oracle.brute_rows(s.T, s.m, s.excl, rows, dist, s.p)
        row = {"config": name, "rows": int(rows.size)}
        for polish in (False, True):
            P, I = run(mp, torch, s, polish=polish)
            row[f"fp32_{'polished' if polish else 'raw'}"] = rel_err(P, rows, Pr)
            row["fp32_i_mismatch"] = int(np.sum(I[rows] != Ir))
        if kslice is None:
            k_range, ref = None, (Pr, Ir)
        else:
            k0 = s.excl + 1
            k_range = (k0, k0 + kslice)
            ref = slice_brute(s.T, s.m, s.excl, rows, k0, k0 + kslice, dist, s.p)
        row["fp64_slice"] = None if k_range is None else list(k_range)
        for polish in (False, True):
            kw = {"precision": "fp64", "polish": polish}
            if k_range is not None:
                kw["k_range"] = k_range
            P, I = run(mp, torch, s, **kw)
            row[f"fp64_{'polished' if polish else 'raw'}"] = rel_err(P, rows, ref[0])
            row["fp64_i_mismatch"] = int(np.sum(I[rows] != ref[1]))
        out.append(row)
        print(json.dumps(row), flush=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rows", type=int, default=48)
    ap.add_argument("--json", default=None)
    args = ap.parse_args()
    out = report(args.rows)
    print("\n| Config | rows | FP32 raw / polished | I != oracle | FP64 raw / polished | I != oracle | FP64 diagonals |")
    print("|---|---|---|---|---|---|---|")
    for r in out:
        sl = "all" if r["fp64_slice"] is None else f"{r['fp64_slice'][0]}..{r['fp64_slice'][1] - 1}"
        print(f"| {r['config']} | {r['rows']} | {r['fp32_raw']:.1e} / {r['fp32_polished']:.1e} | "
              f"{r['fp32_i_mismatch']} | {r['fp64_raw']:.1e} / {r['fp64_polished']:.1e} | {r['fp64_i_mismatch']} | {sl} |")
    if args.json:
        with open(args.json, "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
