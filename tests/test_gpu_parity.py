"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle."""
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


def run(mp, T, m, excl, dist, p=2.0, **kw):
    Tt = torch.from_numpy(np.ascontiguousarray(T)).cuda()
    P, I = mp.profile(Tt, m, excl, dist, p, **kw)
    torch.cuda.synchronize()
    mp.sync_status()
    return P.cpu().numpy(), I.cpu().numpy()


DISTS = [("euclid", 2.0), ("pnorm", 1.0), ("pnorm", 3.0), ("pnorm", 2.5), ("znorm", 2.0)]


@pytest.mark.parametrize("dist,p", DISTS)
@pytest.mark.parametrize("n,m,seed", [(40, 3, 0), (300, 8, 1), (700, 32, 2), (2600, 5, 3)])
def test_small_all_rows(mp, dist, p, n, m, seed):
    s = W.small("walk", n, m, seed, dtype=np.float32)
    for excl in (0, s.excl):
        P, I = run(mp, s.T, m, excl, dist, p)
        parity.check(s.T, m, excl, dist, p, P, I, RTOL32, label=f"{dist} p={p} n={n} m={m} excl={excl}")


@pytest.mark.parametrize("dist,p", DISTS)
def test_multi_band_ragged(mp, dist, p):
    """n = 6,000, m = 24: several diagonal bands and row tiles with ragged
    triangle edges; every row is checked against brute force."""
    s = W.small("motif", 6000, 24, 11, dtype=np.float32)
    P, I = run(mp, s.T, s.m, s.excl, dist, p)
    parity.check(s.T, s.m, s.excl, dist, p, P, I, RTOL32, label=f"{dist} p={p}")


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("dist,p", [("euclid", 2.0), ("pnorm", 1.0), ("pnorm", 3.0)])
def test_integer_series_bit_exact(mp, seed, dist, p):
    """Integer data: every FP32 intermediate is an exact integer, so P equals
    the oracle bit for bit and I follows the paper's tie-break exactly."""
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(100, 5000))
    m = int(rng.integers(1, 40))
    T = rng.integers(-8, 9, n).astype(np.float32)
    for excl in (0, max(1, m // 4)):
        Pr, Ir = oracle.brute(T, m, excl, dist, p)
        P, I = run(mp, T, m, excl, dist, p)
        np.testing.assert_array_equal(I, Ir)
        if p == 3.0:   # the final cube root is CUDA's pow on one side, libm's on the other
            np.testing.assert_allclose(P, Pr, rtol=4e-16)
        else:
            np.testing.assert_array_equal(P, Pr)
        P, I = run(mp, T, m, excl, dist, p, polish=False)   # raw sweep value
        np.testing.assert_array_equal(I, Ir)
        np.testing.assert_allclose(P, Pr, rtol=1e-6)


@pytest.mark.parametrize("dist,p", [("euclid", 2.0), ("pnorm", 1.0), ("pnorm", 3.0), ("znorm", 2.0)])
def test_fp64_sweep(mp, dist, p):
    """The FP64 sweep: polished P at the FP64 bar (1e-12); the raw FP64 sweep
    value too, except for p = 3, whose running sum of cubes |e|^3 - |f|^3
    cancels more between re-anchors (every 256 rows): its raw value is held to
    1e-10 (measured 2.7e-11 on this series); the polished value meets 1e-12."""
    s = W.small("walk", 3000, 20, 21)
    P, I = run(mp, s.T, s.m, s.excl, dist, p, precision="fp64")
    parity.check(s.T, s.m, s.excl, dist, p, P, I, RTOL64, label=f"fp64 {dist}")
    P, I = run(mp, s.T, s.m, s.excl, dist, p, precision="fp64", polish=False)
    parity.check(s.T, s.m, s.excl, dist, p, P, I, 1e-10 if p == 3.0 else RTOL64, label=f"fp64 raw {dist} p={p}")


def test_float64_input(mp):
    """FP64 input on the FP32 path: the hi/lo split keeps differences exact."""
    s = W.small("walk", 4000, 50, 31)
    T = s.T * 10.0 + 300.0
    for dist, p in (("euclid", 2.0), ("pnorm", 1.0), ("znorm", 2.0)):
        P, I = run(mp, T, s.m, s.excl, dist, p)
        parity.check(T, s.m, s.excl, dist, p, P, I, RTOL32, label=f"f64 input {dist}")


def test_edge_cases(mp):
    T = W.small("walk", 64, 4, 41, dtype=np.float32).T
    # no valid pair: N - 1 <= excl
    P, I = run(mp, T, 4, 61, "euclid")
    assert np.all(np.isinf(P)) and np.all(I == -1)
    # m = n: one window
    P, I = run(mp, T, 64, 0, "euclid")
    assert P.shape == (1,) and np.isinf(P[0]) and I[0] == -1
    # m = 1 and excl = 0 (the paper's own exclusion rule)
    for dist, p in (("euclid", 2.0), ("pnorm", 1.0)):
        P, I = run(mp, T, 1, 0, dist, p)
        parity.check(T, 1, 0, dist, p, P, I, RTOL32, label="m=1")
    # a single valid diagonal
    P, I = run(mp, T, 4, 59, "euclid")
    parity.check(T, 4, 59, "euclid", 2.0, P, I, RTOL32, label="one diagonal")


def test_flat_run_znorm(mp):
    s = W.small("flat", 3000, 32, 51, dtype=np.float32)
    mu, S, flat = oracle.window_stats(s.T, 32)
    assert flat.sum() > 0
    P, I = run(mp, s.T, 32, 8, "znorm")
    assert np.all(np.isinf(P[flat])) and np.all(I[flat] == -1)
    assert not np.any(flat[I[I >= 0]])
    parity.check(s.T, 32, 8, "znorm", 2.0, P, I, RTOL32, label="flat z")
    Pe, Ie = run(mp, s.T, 32, 8, "euclid")
    parity.check(s.T, 32, 8, "euclid", 2.0, Pe, Ie, RTOL32, label="flat euclid")


def test_diagonal_ranges_merge(mp):
    """Disjoint diagonal ranges merged with the tie rule equal the full run."""
    T = W.small("int", 5000, 9, 61, dtype=np.float32).T
    N = T.size - 9 + 1
    Pf, If = run(mp, T, 9, 2, "euclid")
    best = np.full(N, np.inf)
    bkey = np.full(N, np.iinfo(np.int64).max)
    x = np.arange(N)
    for r in ((0, 700), (700, 2100), (2100, N)):
        P, I = run(mp, T, 9, 2, "euclid", k_range=r)
        key = np.where(I >= 0, 2 * np.abs(I - x) + (I > x), np.iinfo(np.int64).max)
        take = (P < best) | ((P == best) & (key < bkey))
        best = np.where(take, P, best)
        bkey = np.where(take, key, bkey)
    Irec = np.where(bkey == np.iinfo(np.int64).max, -1, np.where(bkey & 1, x + (bkey >> 1), x - (bkey >> 1)))
    np.testing.assert_array_equal(best, Pf)
    np.testing.assert_array_equal(Irec, If)


def test_repeatable(mp):
    s = W.small("walk", 5000, 16, 71, dtype=np.float32)
    a = run(mp, s.T, s.m, s.excl, "euclid", polish=False)
    b = run(mp, s.T, s.m, s.excl, "euclid", polish=False)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_invalid_arguments(mp):
    Tt = torch.zeros(100, device="cuda")
    with pytest.raises(mp.MPError) as e:
        mp.aamp(Tt, 101, 0)
    assert e.value.status == mp.MP_ERR_INVALID_ARG
    with pytest.raises(mp.MPError):
        mp.pnorm(Tt, 10, 0, 0.5)
    with pytest.raises(mp.MPError):
        mp.aamp(Tt, 10, -1)
    with pytest.raises(mp.MPError):
        mp.acamp(Tt, 1, 0)
    # a rejected call launches nothing and leaves the outputs as they were
    P = torch.full((91,), 7.5, dtype=torch.float64, device="cuda")
    I = torch.full((91,), 3, dtype=torch.int64, device="cuda")
    lib = mp.load()
    n0 = lib.mp_launch_count()
    for bad in (dict(excl=-1), dict(variant=9), dict(precision="fp64", variant=mp.MP_VARIANT_FAST)):
        kw = dict(excl=2)
        kw.update(bad)
        with pytest.raises(mp.MPError):
            mp.aamp(Tt, 10, kw.pop("excl"), out=(P, I), **kw)
    torch.cuda.synchronize()
    assert lib.mp_launch_count() == n0
    assert torch.all(P == 7.5) and torch.all(I == 3)


@pytest.mark.parametrize("m", [32, 64, 96])
def test_integer_fast_path_bit_exact(mp, m):
    """The two-stream kernel (m a multiple of 32, FP32 input) on integer data,
    for p = 2, 1 and 3 (for p = 3 also the tall-tile kernel, its default):
    every term and partial sum is an integer below 2^24, so P and I equal the
    oracle exactly, ties included."""
    rng = np.random.default_rng(900 + m)
    T = rng.integers(-8, 9, 7000).astype(np.float32)
    for dist, p, variant in (("euclid", 2.0, 0), ("pnorm", 1.0, 0), ("pnorm", 3.0, mp.MP_VARIANT_FAST),
                             ("pnorm", 3.0, 0)):
        for excl in (0, m // 4):
            Pr, Ir = oracle.brute(T, m, excl, dist, p)
            P, I = run(mp, T, m, excl, dist, p, variant=variant)
            np.testing.assert_array_equal(I, Ir, err_msg=f"{dist} p={p} excl={excl} variant={variant}")
            if p == 3.0:  # the final cube root: CUDA's and the C library's pow may differ by an ulp
                np.testing.assert_allclose(P, Pr, rtol=4e-16, atol=0)
            else:
                np.testing.assert_array_equal(P, Pr, err_msg=f"{dist} p={p} excl={excl}")


@pytest.mark.parametrize("excl", [0, 8])
def test_integer_long_series_bit_exact(mp, excl):
    """Long series (N >= 200,000) take the Euclidean kernel with the per-block
    filter; on integer data every FP32 value is exact, so P and I must equal
    the FP64 oracle's (Algorithm 1) everywhere, ties included."""
    rng = np.random.default_rng(77 + excl)
    T = rng.integers(-8, 9, 210_000).astype(np.float32)
    m = 32
    Pr, Ir = oracle.aamp(T.astype(np.float64), m, excl)
    P, I = run(mp, T, m, excl, "euclid")
    np.testing.assert_array_equal(I, Ir)
    np.testing.assert_array_equal(P, Pr)


@pytest.mark.parametrize("tile_rows", [4096, 6144, 16384])
def test_two_stream_tall_tiles_bit_exact(mp, tile_rows):
    """Tall tiles of the two-stream kernel (mp_options.tile_rows, a multiple of
    2,048): each stream walks several staged sub-tiles, carrying its sums and
    the ring of block sums from one to the next, and the last tile of each
    band is ragged.  On integer data every FP32 value is exact, so P and I
    equal the FP64 oracle (Algorithms 1 and 3) for p = 2 with and without the
    block filter, p = 1 and p = 3."""
    rng = np.random.default_rng(910 + tile_rows)
    T = rng.integers(-8, 9, 30_000).astype(np.float32)
    m, excl = 64, 16
    T64 = T.astype(np.float64)
    cases = (("euclid", 2.0, mp.MP_VARIANT_FAST_FILTER), ("euclid", 2.0, mp.MP_VARIANT_FAST),
             ("pnorm", 1.0, mp.MP_VARIANT_FAST), ("pnorm", 3.0, mp.MP_VARIANT_FAST))
    for dist, p, variant in cases:
        Pr, Ir = oracle.aamp(T64, m, excl) if dist == "euclid" else oracle.pnorm(T64, m, excl, p)
        P, I = run(mp, T, m, excl, dist, p, variant=variant, tile_rows=tile_rows)
        np.testing.assert_array_equal(I, Ir, err_msg=f"{dist} p={p} variant={variant}")
        if p == 3.0:  # the final cube root: CUDA's and the C library's pow may differ by an ulp
            np.testing.assert_allclose(P, Pr, rtol=4e-16, atol=0)
        else:
            np.testing.assert_array_equal(P, Pr, err_msg=f"{dist} p={p} variant={variant}")


@pytest.mark.parametrize("dist,p", [("euclid", 2.0), ("pnorm", 1.0), ("pnorm", 3.0)])
def test_two_stream_tall_tiles_walk(mp, dist, p):
    """A random walk with a planted motif through 8,192-row tiles of the
    two-stream kernel (4 sub-tiles of 768 rows per stream): every row passes
    the parity rules against brute force."""
    s = W.small("motif", 20_000, 128, 912, dtype=np.float32)
    P, I = run(mp, s.T, s.m, s.excl, dist, p, variant=mp.MP_VARIANT_FAST, tile_rows=8192)
    parity.check(s.T, s.m, s.excl, dist, p, P, I, RTOL32, label=f"tall two-stream {dist} p={p}")


def test_long_walk_filter_kernel(mp):
    """A 300,000-point random walk with a planted motif (filter kernel): sampled
    rows by brute force, the motif rows included."""
    s = W.small("motif", 300_000, 64, 83, dtype=np.float32)
    rows = np.unique(np.concatenate([np.random.default_rng(2).choice(s.N, 300, replace=False), [0, s.N - 1]]))
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, "euclid")
    P, I = run(mp, s.T, s.m, s.excl, "euclid")
    parity.check(s.T, s.m, s.excl, "euclid", 2.0, P, I, RTOL32, rows=rows, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                 label="long walk")
    x = np.arange(s.N)
    assert np.all(I >= 0) and np.all(np.abs(I - x) > s.excl)


def test_long_znorm_filter_kernel(mp):
    """A 250,000-point walk with a flat run (z-normalised, filter kernel): the
    flat rows get no neighbour and are nobody's neighbour; sampled rows, the
    flat run's edges included, match brute force."""
    s = W.small("flat", 250_000, 64, 85, dtype=np.float32)
    mu, S, flat = oracle.window_stats(s.T, s.m)
    assert flat.sum() > 0
    fr = np.nonzero(flat)[0]
    extra = [fr[0] - 1, fr[0], fr[-1], fr[-1] + 1]
    rows = np.unique(np.concatenate([np.random.default_rng(4).choice(s.N, 250, replace=False), extra]))
    rows = rows[(rows >= 0) & (rows < s.N)]
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, "znorm")
    P, I = run(mp, s.T, s.m, s.excl, "znorm")
    assert np.all(np.isinf(P[flat])) and np.all(I[flat] == -1)
    assert not np.any(flat[I[I >= 0]])
    parity.check(s.T, s.m, s.excl, "znorm", 2.0, P, I, RTOL32, rows=rows, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                 label="long z")


@pytest.mark.parametrize("dist,p", [("euclid", 2.0), ("pnorm", 1.0), ("pnorm", 3.0)])
def test_fast_and_generic_kernels_agree(mp, monkeypatch, dist, p):
    """The default FP32 kernel (two-stream; tall-tile for p = 3) and the
    generic one against the oracle on a series with many bands and row tiles
    (n = 40,000, m = 64)."""
    s = W.small("motif", 40_000, 64, 81, dtype=np.float32)
    rows = np.random.default_rng(1).choice(s.N, 400, replace=False)
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, dist, p)
    P1, I1 = run(mp, s.T, s.m, s.excl, dist, p)
    monkeypatch.setenv("MP_FORCE_GENERIC", "1")
    P2, I2 = run(mp, s.T, s.m, s.excl, dist, p)
    for P, I, lab in ((P1, I1, "fast"), (P2, I2, "generic")):
        parity.check(s.T, s.m, s.excl, dist, p, P, I, RTOL32, rows=rows,
                     P_ref=ref[0], I_ref=ref[1], P2=ref[2], label=lab)
    agree = np.mean(I1 == I2)
    assert agree > 0.999, agree


@pytest.mark.parametrize("kind,m,dist,seed", [("uniform", 32, "euclid", 91), ("uniform", 48, "znorm", 92),
                                              ("flat", 64, "znorm", 93)])
def test_block_filters_are_exact(mp, kind, m, dist, seed):
    """The block filters only skip blocks whose candidates cannot pass: forced on
    and off they give the same profile bit for bit.  On i.i.d. uniform data the
    distances are tightly spread, so the bounds fail often and many blocks are
    replayed; the flat run gives the z-normalised filter NaN rows and columns."""
    s = W.small(kind, 230_000, m, seed, dtype=np.float32)
    Pf, If = run(mp, s.T, s.m, s.excl, dist, variant=mp.MP_VARIANT_FAST_FILTER)
    Pn, In = run(mp, s.T, s.m, s.excl, dist, variant=mp.MP_VARIANT_FAST)
    np.testing.assert_array_equal(If, In)
    np.testing.assert_array_equal(Pf, Pn)
    rows = np.random.default_rng(seed).choice(s.N, 120, replace=False)
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, dist)
    parity.check(s.T, s.m, s.excl, dist, 2.0, Pf, If, RTOL32, rows=rows, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                 label=f"filter {kind} {dist}")


def test_raw_sum_ablation(mp):
    """MP_VARIANT_ZRAW, Algorithm 2's raw-sum form: in FP64 it meets the FP64
    bar on a stationary series (mean small against the spread, so the
    numerator C - A_i A_j / m barely cancels); in FP32 it returns exact
    distances (polished) at valid neighbours close to the best; it exists only
    for the z-normalised distance."""
    s = W.small("uniform", 3000, 32, 95, dtype=np.float32)
    ref = oracle.brute_rows(s.T, s.m, s.excl, np.arange(s.N), "znorm")
    P, I = run(mp, s.T, s.m, s.excl, "znorm", precision="fp64", variant=mp.MP_VARIANT_ZRAW)
    parity.check(s.T, s.m, s.excl, "znorm", 2.0, P, I, RTOL64, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                 label="raw sums fp64")
    P, I = run(mp, s.T, s.m, s.excl, "znorm", variant=mp.MP_VARIANT_ZRAW)
    assert np.all(np.abs(I - np.arange(s.N)) > s.excl)
    d = oracle.pair_dist(s.T.astype(np.float64), s.m, np.arange(s.N), I, "znorm", 2.0)
    np.testing.assert_allclose(P, d, rtol=1e-12)
    assert np.all(P <= ref[0] * (1 + 1e-3))
    with pytest.raises(mp.MPError):
        run(mp, s.T, s.m, s.excl, "euclid", variant=mp.MP_VARIANT_ZRAW)


def test_f_comparison_ablation(mp):
    """MP_VARIANT_ZF, Sec. 4.3's comparison of candidates through
    F = (A_i A_j - m C)|A_i A_j - m C| / (S_i S_j) on the raw sums, with the
    winner's DZ^2 = 2m + 2 sign(F) sqrt(|F|): in FP64 it meets the FP64 bar
    (polished, and the raw value converted from F) on a stationary series; in
    FP32 it returns exact distances (polished) at valid neighbours close to the
    best; it exists only for the z-normalised distance."""
    s = W.small("uniform", 3000, 32, 96, dtype=np.float32)
    ref = oracle.brute_rows(s.T, s.m, s.excl, np.arange(s.N), "znorm")
    for polish in (True, False):
        P, I = run(mp, s.T, s.m, s.excl, "znorm", precision="fp64", variant=mp.MP_VARIANT_ZF, polish=polish)
        parity.check(s.T, s.m, s.excl, "znorm", 2.0, P, I, RTOL64, P_ref=ref[0], I_ref=ref[1], P2=ref[2],
                     label=f"F comparison fp64 polish={polish}")
    P, I = run(mp, s.T, s.m, s.excl, "znorm", variant=mp.MP_VARIANT_ZF)
    assert np.all(np.abs(I - np.arange(s.N)) > s.excl)
    d = oracle.pair_dist(s.T.astype(np.float64), s.m, np.arange(s.N), I, "znorm", 2.0)
    np.testing.assert_allclose(P, d, rtol=1e-12)
    assert np.all(P <= ref[0] * (1 + 1e-3))
    # flat windows: no neighbour, never a neighbour (as every z-normalised kernel)
    f = W.small("flat", 3000, 32, 51, dtype=np.float32)
    mu, S, flat = oracle.window_stats(f.T, 32)
    for prec in ("fp32", "fp64"):
        P, I = run(mp, f.T, 32, 8, "znorm", precision=prec, variant=mp.MP_VARIANT_ZF)
        assert np.all(np.isinf(P[flat])) and np.all(I[flat] == -1)
        assert not np.any(flat[I[I >= 0]])
    with pytest.raises(mp.MPError):
        run(mp, s.T, s.m, s.excl, "euclid", variant=mp.MP_VARIANT_ZF)
