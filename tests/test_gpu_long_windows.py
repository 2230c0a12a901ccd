"""Long windows: the tall-tile kernel (float-float sums, tiles of max(8192, 8m)
rows) serves the Euclidean and p-norm sweeps for m >= 512, including window
lengths the generic kernel's shared memory cannot hold.  Checked against
brute-force rows of the FP64 oracle and against the generic kernel where both
apply."""
import numpy as np
import pytest

import oracle
from paper_1901_05708_gb300 import workloads as W

import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL32 = 1e-5


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_05708_gb300 import mp as lib
    lib.load()
    return lib


def run(mp, T, m, excl, dist, p=2.0, **kw):
    P, I = mp.profile(torch.from_numpy(np.ascontiguousarray(T)).cuda(), m, excl, dist, p, **kw)
    torch.cuda.synchronize()
    mp.sync_status()
    return P.cpu().numpy(), I.cpu().numpy()


@pytest.mark.parametrize("dist,p", [("euclid", 2.0), ("pnorm", 1.0), ("pnorm", 3.0)])
def test_long_window_rows(mp, dist, p):
    s = W.small("motif", 40_000, 2_000, 61, dtype=np.float32)
    rows = np.unique(np.concatenate([np.random.default_rng(6).choice(s.N, 40, replace=False), [0, s.N - 1]]))
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, dist, p)
    P, I = run(mp, s.T, s.m, s.excl, dist, p)
    parity.check(s.T, s.m, s.excl, dist, p, P, I, RTOL32, rows=rows, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                 label=f"m=2000 {dist}")
    x = np.arange(s.N)
    assert np.all(I >= 0) and np.all(np.abs(I - x) > s.excl)


def test_tall_and_generic_agree(mp):
    """Where the two kernels pick different neighbours (near ties of long,
    smooth windows; the generic kernel re-anchors only every 250 rows here),
    the tall kernel's choice must pass the oracle's parity rules."""
    s = W.small("walk", 30_000, 1_500, 62, dtype=np.float32)
    Pt, It = run(mp, s.T, s.m, s.excl, "euclid", variant=4)
    Pg, Ig = run(mp, s.T, s.m, s.excl, "euclid", variant=3)
    assert np.mean(It == Ig) > 0.995
    np.testing.assert_allclose(Pt, Pg, rtol=1e-4)
    diff = np.nonzero(It != Ig)[0][:40]
    rows = np.unique(np.concatenate([diff, np.random.default_rng(9).choice(s.N, 20, replace=False)]))
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, "euclid")
    parity.check(s.T, s.m, s.excl, "euclid", 2.0, Pt, It, RTOL32, rows=rows, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                 label="tall, rows where the kernels differ")


def test_window_beyond_the_generic_kernel(mp):
    """m = 16,384: no shared-memory tile of the generic kernel holds it."""
    s = W.small("motif", 80_000, 16_384, 63, dtype=np.float32)
    rows = np.array([0, 17, 4_000, 30_000, s.N - 1])
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, "euclid")
    P, I = run(mp, s.T, s.m, s.excl, "euclid")
    parity.check(s.T, s.m, s.excl, "euclid", 2.0, P, I, RTOL32, rows=rows, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                 label="m=16384")


def test_tall_kernel_on_short_windows(mp):
    """The tall kernel forced on m = 64 (p = 2), which AUTO never picks for
    windows this short: it carries each tile's float-float sums over 8,192
    rows without re-anchoring, so on near ties it may pick a neighbour up to
    about 1e-4 relative farther than the two-stream kernel's (measured:
    5.9e-5 on 7 of 49,937 rows); everywhere else the two agree.  On integer
    data it is exact."""
    s = W.small("walk", 50_000, 64, 64, dtype=np.float32)
    Pt, It = run(mp, s.T, s.m, s.excl, "euclid", variant=4)
    Pd, Id = run(mp, s.T, s.m, s.excl, "euclid")
    assert np.mean(It == Id) > 0.999
    np.testing.assert_allclose(Pt, Pd, rtol=1e-4)
    rng = np.random.default_rng(8)
    T = rng.integers(-8, 9, 20_000).astype(np.float32)  # integer data: bit-exact
    Pt, It = run(mp, T, 1_100, 200, "euclid")
    Pr, Ir = oracle.aamp(T.astype(np.float64), 1_100, 200)
    np.testing.assert_array_equal(It, Ir)
    np.testing.assert_array_equal(Pt, Pr)


@pytest.mark.parametrize("dist,p,tile_rows", [("euclid", 2.0, 4096), ("pnorm", 1.0, 1024), ("znorm", 2.0, 1024),
                                              ("znorm", 2.0, 8192)])
def test_tile_rows(mp, dist, p, tile_rows):
    """mp_options.tile_rows on the tall-tile kernels: tiles shorter than the
    default (here down to 1,024 rows, below 8m, so several tiles per band and
    ragged last tiles) give the oracle's profile within the parity rules."""
    m = 600 if dist != "znorm" else 200
    s = W.small("motif", 30_000, m, 63, dtype=np.float32)
    rows = np.unique(np.concatenate([np.random.default_rng(7).choice(s.N, 60, replace=False), [0, s.N - 1]]))
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, dist, p)
    kw = {"tile_rows": tile_rows}
    if dist != "znorm":
        kw["variant"] = 4  # the tall-tile kernel
    P, I = run(mp, s.T, s.m, s.excl, dist, p, **kw)
    parity.check(s.T, s.m, s.excl, dist, p, P, I, RTOL32, rows=rows, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                 label=f"{dist} tile_rows={tile_rows}")
    x = np.arange(s.N)
    assert np.all(I >= 0) and np.all(np.abs(I - x) > s.excl)
