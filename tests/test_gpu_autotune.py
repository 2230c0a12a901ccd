"""Autotuning (mp_autotune): candidates are timed, the choice is one of them,
results with the chosen kernel pass parity, and the cache answers a second
call without timing."""
import numpy as np
import pytest

import oracle
from paper_1901_05708_gb300 import workloads as W

import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_05708_gb300 import mp as lib
    lib.load()
    return lib


@pytest.mark.parametrize("dist,p,m", [("euclid", 2.0, 64), ("pnorm", 1.0, 64), ("euclid", 2.0, 48)])
def test_autotune_choice_and_parity(mp, dist, p, m, tmp_path):
    s = W.small("motif", 220_000, m, 41, dtype=np.float32)
    T = torch.from_numpy(s.T).cuda()
    kw, times = mp.autotune(T, s.m, s.excl, dist, p, force=True)
    fast = (2 if dist == "euclid" else 1) if m % 32 == 0 else 0
    assert len(times) >= fast + 2 and all(t > 0 for t in times), times  # fast kernels, 2 generic intervals
    assert kw["variant"] in (1, 2, 3, 4)
    kw2, times2 = mp.autotune(T, s.m, s.excl, dist, p)  # cached
    assert kw2 == kw and times2 == []
    P, I = mp.profile(T, s.m, s.excl, dist, p, **kw)
    torch.cuda.synchronize()
    rows = np.random.default_rng(3).choice(s.N, 200, replace=False)
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, dist, p)
    parity.check(s.T, s.m, s.excl, dist, p, P.cpu().numpy(), I.cpu().numpy(), 1e-5, rows=rows, P_ref=ref[0],
                 I_ref=ref[1], P2=ref[2], label=f"tuned {kw}")
    path = str(tmp_path / "tune.txt")
    mp.autotune_cache_save(path)
    assert mp.autotune_cache_size() >= 1
    mp.autotune_cache_load(path)


def test_forced_variants_agree(mp):
    s = W.small("walk", 210_000, 64, 43, dtype=np.float32)
    T = torch.from_numpy(s.T).cuda()
    out = []
    for v in (1, 2, 3):
        P, I = mp.aamp(T, s.m, s.excl, variant=v)
        torch.cuda.synchronize()
        out.append((P.cpu().numpy(), I.cpu().numpy()))
    np.testing.assert_array_equal(out[0][1], out[1][1])  # same tiles and values: filter or not
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert np.mean(out[0][1] == out[2][1]) > 0.999
    with pytest.raises(mp.MPError):
        mp.pnorm(T, s.m, s.excl, 3.0, variant=1)  # the filter is for p = 2
    with pytest.raises(mp.MPError):
        mp.acamp(T, s.m, s.excl, variant=3)


def test_autotune_znorm_filter_choice(mp):
    """For the z-normalised distance the candidates are its kernel with and
    without the block filter; the choice runs and matches the oracle."""
    s = W.small("walk", 210_000, 64, 44, dtype=np.float32)
    T = torch.from_numpy(s.T).cuda()
    kw, times = mp.autotune(T, s.m, s.excl, "znorm", force=True)
    assert kw["variant"] in (mp.MP_VARIANT_FAST_FILTER, mp.MP_VARIANT_FAST, mp.MP_VARIANT_FAST_FILTER_BOUND)
    assert kw["tile_rows"] in (0, 16384, 4096)
    # filter on / off x 3 tile heights, and the bound filter
    assert len(times) == 7 and all(t > 0 for t in times), times
    P, I = mp.acamp(T, s.m, s.excl, **kw)
    torch.cuda.synchronize()
    rows = np.random.default_rng(5).choice(s.N, 150, replace=False)
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, "znorm")
    parity.check(s.T, s.m, s.excl, "znorm", 2.0, P.cpu().numpy(), I.cpu().numpy(), 1e-5, rows=rows,
                 P_ref=ref[0], I_ref=ref[1], P2=ref[2], label=f"tuned z {kw}")
    with pytest.raises(mp.MPError):
        mp.acamp(T, s.m, s.excl, variant=mp.MP_VARIANT_TALL)


def _cache_key(mp, N, m, dist_code, dtype=0, p=2.0):
    """The autotuning cache key of a problem class (device name, dist, dtype,
    m, floor(log2 N), p), as the library writes it."""
    name = torch.cuda.get_device_name().replace(" ", "_").replace("|", "_")
    return f"{name}|{dist_code}|{dtype}|{m}|{N.bit_length() - 1}|{p:.6g}"


def test_cached_tile_rows_in_calls_and_batches(mp, tmp_path):
    """A cached choice with a tile height (here loaded from a cache file:
    the z-normalised kernel without its filter at 4,096 rows per tile) is
    what MP_VARIANT_CACHED runs, in a single call and for the z-normalised
    series of a batch plan: bit for bit the explicit options' result, which
    passes the parity rules; without a cache entry CACHED is AUTO."""
    s = W.small("walk", 60_000, 64, 45, dtype=np.float32)
    e = W.small("walk", 30_000, 64, 46, dtype=np.float32)  # a Euclidean series in the same batch
    T = torch.from_numpy(s.T).cuda()
    path = tmp_path / "cache.txt"
    path.write_text(f"{_cache_key(mp, s.N, s.m, mp.MP_DIST_ZNORM)} {mp.MP_VARIANT_FAST} 0 1.0 4096\n")
    mp.autotune_cache_load(str(path))
    Pc, Ic = mp.acamp(T, s.m, s.excl, variant=mp.MP_VARIANT_CACHED)
    Pe, Ie = mp.acamp(T, s.m, s.excl, variant=mp.MP_VARIANT_FAST, tile_rows=4096)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Pc.cpu().numpy(), Pe.cpu().numpy())
    np.testing.assert_array_equal(Ic.cpu().numpy(), Ie.cpu().numpy())
    rows = np.random.default_rng(6).choice(s.N, 150, replace=False)
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, "znorm")
    parity.check(s.T, s.m, s.excl, "znorm", 2.0, Pc.cpu().numpy(), Ic.cpu().numpy(), 1e-5, rows=rows,
                 P_ref=ref[0], I_ref=ref[1], P2=ref[2], label="cached tile rows")
    plan = mp.BatchPlan([e.n, s.n], [e.m, s.m], ["euclid", "znorm"], [e.excl, s.excl],
                        variant=mp.MP_VARIANT_CACHED)
    P, I = plan.run(torch.from_numpy(np.concatenate([e.T, s.T])).cuda())
    torch.cuda.synchronize()
    o = plan.out_offsets
    np.testing.assert_array_equal(P.cpu().numpy()[o[1]:o[2]], Pe.cpu().numpy())
    np.testing.assert_array_equal(I.cpu().numpy()[o[1]:o[2]], Ie.cpu().numpy())
    plan.close()
    # another problem class has no entry: CACHED runs as AUTO
    u = W.small("walk", 20_000, 40, 47, dtype=np.float32)
    Tu = torch.from_numpy(u.T).cuda()
    a1 = mp.acamp(Tu, u.m, u.excl, variant=mp.MP_VARIANT_CACHED)
    a0 = mp.acamp(Tu, u.m, u.excl)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a1[0].cpu().numpy(), a0[0].cpu().numpy())
    with pytest.raises(mp.MPError):
        mp.aamp(Tu, u.m, u.excl, tile_rows=4096)  # m = 40: the generic kernel, whose tiles are fixed


@pytest.mark.parametrize("kind", ["flat", "uniform"])
def test_bound_filter_is_bit_identical(mp, kind):
    """MP_VARIANT_FAST_FILTER_BOUND only changes which blocks the z-normalised
    filter skips: its profile equals the exact filter's and the unfiltered
    kernel's bit for bit (flat windows included)."""
    s = W.small(kind, 210_000, 64, 48, dtype=np.float32)  # a random walk with a flat run, or i.i.d. values
    T = torch.from_numpy(s.T).cuda()
    out = []
    for v in (mp.MP_VARIANT_FAST_FILTER_BOUND, mp.MP_VARIANT_FAST_FILTER, mp.MP_VARIANT_FAST):
        P, I = mp.acamp(T, s.m, s.excl, variant=v)
        torch.cuda.synchronize()
        out.append((P.cpu().numpy(), I.cpu().numpy()))
    for P, I in out[1:]:
        np.testing.assert_array_equal(out[0][0], P)
        np.testing.assert_array_equal(out[0][1], I)
    with pytest.raises(mp.MPError):
        mp.aamp(T, s.m, s.excl, variant=mp.MP_VARIANT_FAST_FILTER_BOUND)
