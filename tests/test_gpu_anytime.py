"""Anytime runs (mp_anytime_*): tiles in a seeded random order.

Partial profiles are made of exact cells, only tighten and stay above the
complete profile, up to the FP32 sweep's resolution (candidates closer than it
may be ordered either way: parity rule iii); the complete run equals the
batch path's profile of the series bit for bit (same tiles, only the order
differs); a checkpoint taken halfway and restored into a fresh run finishes to
the same profile."""
import numpy as np
import pytest

import oracle
import parity
from paper_1901_05708_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_05708_gb300 import mp as lib
    lib.load()
    return lib


def fp32_tol(s, dist, p, P):
    """The FP32 sweep's ordering resolution at P, for comparing partial
    profiles with each other: rtol 1e-5, the absolute floor and, for
    z-normalised rows, the FP32 resolution of q (candidates closer than this
    may be ordered either way, so a later partial profile may hold a neighbour
    that much farther).  The finished profile is checked against the oracle
    with the contract's rules."""
    rtol = 1e-5
    Pf = np.where(np.isfinite(P), P, 0.0)
    tol = rtol * Pf + parity.atol_for(s.T, s.m, dist, p, rtol)
    if dist == "znorm":
        tol = tol + np.sqrt(Pf ** 2 + 2 * s.m * parity.Q_ATOL_Z32) - Pf
    return tol


def reference(mp, s, dist, p):
    plan = mp.BatchPlan([s.n], [s.m], [dist], [s.excl], p=p)
    P, I = plan.run(torch.from_numpy(s.T).cuda())
    torch.cuda.synchronize()
    plan.close()
    return P.cpu().numpy(), I.cpu().numpy()


@pytest.mark.parametrize("dist,p,m", [("euclid", 2.0, 64), ("euclid", 2.0, 40), ("znorm", 2.0, 48),
                                      ("pnorm", 1.0, 32), ("pnorm", 2.5, 20)])
def test_partial_profiles_tighten_to_the_full_one(mp, dist, p, m):
    s = W.small("motif", 60_000, m, 17, dtype=np.float32)
    Pref, Iref = reference(mp, s, dist, p)
    a = mp.Anytime(torch.from_numpy(s.T).cuda(), s.m, s.excl, dist, p, seed=7)
    total = a.tiles_total
    assert total > 4
    prev = np.full(s.N, np.inf)
    T64 = s.T.astype(np.float64)
    for step in range(4):
        a.run(max(1, total // 4) if step < 3 else total)  # the last call takes what is left
        P, I = a.read()
        torch.cuda.synchronize()
        P, I = P.cpu().numpy(), I.cpu().numpy()
        assert np.all(P <= prev + fp32_tol(s, dist, p, prev))  # never loosens (beyond FP32 near-ties)
        has = I >= 0
        assert np.all(np.abs(I[has] - np.arange(s.N)[has]) > s.excl)
        pick = np.nonzero(has)[0][:: max(1, has.sum() // 300)]
        d = oracle.pair_dist(T64, s.m, pick, I[pick], dist, p)
        np.testing.assert_allclose(P[pick], d, rtol=1e-12)  # exact cells (polished)
        assert np.all(P[has] >= Pref[has] - fp32_tol(s, dist, p, Pref)[has])  # upper bounds of the full profile
        prev = P
    assert a.tiles_done == total
    np.testing.assert_array_equal(I, Iref)
    np.testing.assert_array_equal(P, Pref)
    a.close()
    # the finished profile against the oracle's brute force (the contract's rules)
    rows = np.unique(np.concatenate([np.random.default_rng(5).choice(s.N, 200, replace=False), [0, s.N - 1]]))
    ref = oracle.brute_rows(T64, s.m, s.excl, rows, dist, p)
    parity.check(T64, s.m, s.excl, dist, p, P, I, 1e-5, rows=rows, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                 label=f"anytime {dist} p={p}")


def test_checkpoint_and_restore(mp):
    s = W.small("walk", 50_000, 32, 23, dtype=np.float32)
    T = torch.from_numpy(s.T).cuda()
    a = mp.Anytime(T, s.m, s.excl, "euclid", seed=99)
    total = a.tiles_total
    a.run(total // 2)
    blob = a.checkpoint()
    Ph, Ih = a.read()
    a.run(total)
    Pfull, Ifull = a.read()
    torch.cuda.synchronize()
    a.close()
    b = mp.Anytime(T, s.m, s.excl, "euclid", seed=99)
    b.restore(blob)
    assert b.tiles_done == total // 2
    P2, I2 = b.read()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(P2.cpu().numpy(), Ph.cpu().numpy())
    b.run(total)
    P3, I3 = b.read()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(P3.cpu().numpy(), Pfull.cpu().numpy())
    np.testing.assert_array_equal(I3.cpu().numpy(), Ifull.cpu().numpy())
    c = mp.Anytime(T, s.m, s.excl, "euclid", seed=100)  # another seed: the checkpoint does not fit
    with pytest.raises(mp.MPError):
        c.restore(blob)
    b.close()
    c.close()
