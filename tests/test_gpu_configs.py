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


def test_aamp_small_all_rows(mp):
    """10,000-point float64 random walk, m = 100: every row, FP32 and FP64 sweeps."""
    s = W.aamp_small()
    rows = np.arange(s.N)
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, "euclid")
    for prec, rtol in (("fp32", RTOL32), ("fp64", RTOL64)):
        P, I, dist = run(mp, s, precision=prec)
        st = parity.check(s.T, s.m, s.excl, dist, 2.0, P, I, rtol, rows=rows, P_ref=ref[0], I_ref=ref[1],
                          P2=ref[2], label=f"aamp_small {prec}")
        assert st["rows"] == s.N


def test_aamp_1m_sampled_rows(mp):
    """n = 2^20 random walk with bumps, m = 256: sampled rows and the bump centres."""
    s = W.aamp_1m()
    rows = sample_rows(s.N, 96, 11, extra=np.asarray(s.info["bump_centres"], int) - s.m // 2)
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, "euclid")
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
    P, I, dist = run(mp, s)
    parity.check(s.T, s.m, s.excl, dist, 2.0, P, I, RTOL32, rows=rows, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                 label="acamp_1m")
