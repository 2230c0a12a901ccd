"""Parity on the five workload configurations, at full size.

Rows are checked against the FP64 oracle: every row for the 10,000-point
series, seeded samples of rows (brute force of the whole row, plus the
runner-up) for the million-point series.  The calls are the ones bench.py
times (same entry points, same default options)."""
import numpy as np
import pytest

import oracle
from paper_1901_05708_gb300 import workloads as W

import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL32, RTOL64 = 1e-5, 1e-12


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_05708_gb300 import mp as lib
    lib.load()
    return lib


def run(mp, s, **kw):
    T = torch.from_numpy(np.ascontiguousarray(s.T)).cuda()
    dist = {W.EUCLID: "euclid", W.PNORM: "pnorm", W.ZNORM: "znorm"}[s.dist]
    P, I = mp.profile(T, s.m, s.excl, dist, s.p, **kw)
    torch.cuda.synchronize()
    mp.sync_status()
    return P.cpu().numpy(), I.cpu().numpy(), dist


def sample_rows(N, count, seed, extra=()):
    rng = np.random.default_rng(seed)
    rows = set(rng.choice(N, count, replace=False).tolist())
    rows.update(int(r) for r in extra if 0 <= r < N)
    rows.update((0, N - 1))
    return np.array(sorted(rows), dtype=np.int64)


def slice_brute(T, m, excl, rows, k0, k1, dist, p=2.0):
    """Brute force of rows over the diagonals k0 <= |i - j| < k1 only (the
    profile of a diagonal range): best value, its index with the paper's tie
    rule, and the runner-up outside the winner's zone."""
    T = np.asarray(T, np.float64)
    N = T.size - m + 1
    Pr, Ir, P2 = [], [], []
    for i in rows:
        ks = np.arange(max(k0, excl + 1), k1)
        js = np.concatenate([i - ks, i + ks])
        side = np.concatenate([np.zeros(ks.size, int), np.ones(ks.size, int)])
        kk = np.concatenate([ks, ks])
        ok = (js >= 0) & (js < N)
        js, side, kk = js[ok], side[ok], kk[ok]
        if js.size == 0:
            Pr.append(np.inf), Ir.append(-1), P2.append(np.inf)
            continue
        d = oracle.pair_dist(T, m, np.full(js.size, i), js, dist, p)
        order = np.lexsort((side, kk, d))  # value, then smaller k, then the left neighbour
        w = order[0]
        Pr.append(d[w]), Ir.append(js[w])
        far = np.abs(js - js[w]) > excl
        P2.append(d[far].min() if far.any() else np.inf)
    return np.array(Pr), np.array(Ir, np.int64), np.array(P2)


def raw_error(P, rows, ref, s=None, p=2.0):
    """Max relative error of P on rows against the reference values (rows with
    a finite reference); for a raw FP32 pure / p-norm value of series s, P
    below the score's resolution (S_ATOL^(1/p), see tests/parity.py) is
    measured against that resolution instead of itself."""
    fin = np.isfinite(ref)
    floor = 1e-300
    if s is not None and s.dist != W.ZNORM:
        pp = 2.0 if s.dist == W.EUCLID else p
        floor = (RTOL32 * s.m * np.std(np.diff(np.asarray(s.T, np.float64))) ** pp) ** (1.0 / pp)
    den = np.maximum(ref[fin], floor)
    return float(np.max(np.abs(P[rows][fin] - ref[fin]) / den)) if fin.any() else 0.0


def test_aamp_small_all_rows(mp):
    """10,000-point float64 random walk, m = 100: every row, FP32 and FP64
    sweeps, polished (the default) and the sweeps' own raw values."""
    s = W.aamp_small()
    rows = np.arange(s.N)
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, "euclid")
    for prec, rtol in (("fp32", RTOL32), ("fp64", RTOL64)):
        for polish in (True, False):
            P, I, dist = run(mp, s, precision=prec, polish=polish)
            st = parity.check(s.T, s.m, s.excl, dist, 2.0, P, I, rtol, rows=rows, P_ref=ref[0], I_ref=ref[1],
                              P2=ref[2], label=f"aamp_small {prec} polish={polish}")
            assert st["rows"] == s.N and raw_error(P, rows, ref[0], s if prec == "fp32" else None) < rtol


def test_aamp_1m_sampled_rows(mp):
    """n = 2^20 random walk with bumps, m = 256: sampled rows and the bump centres."""
    s = W.aamp_1m()
    rows = sample_rows(s.N, 96, 11, extra=np.asarray(s.info["bump_centres"], int) - s.m // 2)
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, "euclid")
    P, I, dist = run(mp, s, polish=False)  # the FP32 sweep's own value
    parity.check(s.T, s.m, s.excl, dist, 2.0, P, I, RTOL32, rows=rows, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                 label="aamp_1m raw", raw_fp32=True)
    assert raw_error(P, rows, ref[0], s) < RTOL32
    P, I, dist = run(mp, s)
    parity.check(s.T, s.m, s.excl, dist, 2.0, P, I, RTOL32, rows=rows, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                 label="aamp_1m")
    # properties that hold on every row: a valid neighbour outside the zone, P = d(i, I[i])
    x = np.arange(s.N)
    assert np.all(I >= 0) and np.all(np.abs(I - x) > s.excl)
    pick = np.random.default_rng(5).choice(s.N, 2000, replace=False)
    d = oracle.pair_dist(s.T, s.m, pick, I[pick], "euclid")
    np.testing.assert_allclose(P[pick], d, rtol=1e-12)


@pytest.mark.parametrize("p", [1.0, 3.0])
def test_pnorm_262k_sampled_rows(mp, p):
    """n = 2^18 sine + motifs + flat run, m = 128, p = 1 and 3."""
    s = W.pnorm_262k(p)
    fa, fl = s.info["flat"]
    extra = list(s.info["motif_starts"]) + [fa, fa + fl // 2, fa + fl - s.m]
    rows = sample_rows(s.N, 64, 12, extra=extra)
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, "pnorm", p)
    P, I, dist = run(mp, s, polish=False)  # raw: near P = 0 (the flat run) the score's resolution applies
    parity.check(s.T, s.m, s.excl, dist, p, P, I, RTOL32, rows=rows, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                 label=f"pnorm p={p} raw", raw_fp32=True)
    # (no separate relative bound: near the flat run the raw value's error is the
    # score's absolute resolution, which rule (i) of the raw check above states)
    P, I, dist = run(mp, s)
    parity.check(s.T, s.m, s.excl, dist, p, P, I, RTOL32, rows=rows, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                 label=f"pnorm p={p}")
    # every planted copy finds another copy (their windows are near-identical)
    starts = np.asarray(s.info["motif_starts"])
    for st in starts:
        assert np.min(np.abs(starts - I[st])) <= s.excl


def test_acamp_1m_sampled_rows(mp):
    """n = 2^20 random walk + N(0, 0.01), m = 512, z-normalised."""
    s = W.acamp_1m()
    rows = sample_rows(s.N, 48, 13)
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, "znorm")
    P, I, dist = run(mp, s, polish=False)  # raw: the kernel's stated q resolution applies
    parity.check(s.T, s.m, s.excl, dist, 2.0, P, I, RTOL32, rows=rows, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                 label="acamp_1m raw", raw_fp32=True)
    assert raw_error(P, rows, ref[0]) < RTOL32
    P, I, dist = run(mp, s)
    parity.check(s.T, s.m, s.excl, dist, 2.0, P, I, RTOL32, rows=rows, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                 label="acamp_1m")


@pytest.mark.parametrize("dist,k1", [("euclid", 2_000), ("znorm", 600)])
def test_fp64_sweep_at_scale(mp, dist, k1):
    """The FP64 sweep on the million-point series, on the first diagonals (the
    slice bench.py times): sampled rows against brute force over the same
    diagonals, polished P and the raw FP64 sweep value at the FP64 bar."""
    s = W.aamp_1m() if dist == "euclid" else W.acamp_1m()
    k0 = s.excl + 1
    k1 = k0 + k1
    rows = sample_rows(s.N, 40, 14)
    ref = slice_brute(s.T, s.m, s.excl, rows, k0, k1, dist)
    T = torch.from_numpy(s.T).cuda()
    for polish, rtol in ((True, RTOL64), (False, RTOL64)):
        P, I = mp.profile(T, s.m, s.excl, dist, 2.0, precision="fp64", polish=polish, k_range=(k0, k1))
        torch.cuda.synchronize()
        mp.sync_status()
        P, I = P.cpu().numpy(), I.cpu().numpy()
        parity.check(s.T, s.m, s.excl, dist, 2.0, P, I, rtol, rows=rows, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                     label=f"fp64 slice {dist} polish={polish}")
