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
    assert kw["variant"] in (mp.MP_VARIANT_FAST_FILTER, mp.MP_VARIANT_FAST)
    assert len(times) == 2 and all(t > 0 for t in times), times
    P, I = mp.acamp(T, s.m, s.excl, **kw)
    torch.cuda.synchronize()
    rows = np.random.default_rng(5).choice(s.N, 150, replace=False)
    ref = oracle.brute_rows(s.T, s.m, s.excl, rows, "znorm")
    parity.check(s.T, s.m, s.excl, "znorm", 2.0, P.cpu().numpy(), I.cpu().numpy(), 1e-5, rows=rows,
                 P_ref=ref[0], I_ref=ref[1], P2=ref[2], label=f"tuned z {kw}")
    with pytest.raises(mp.MPError):
        mp.acamp(T, s.m, s.excl, variant=mp.MP_VARIANT_TALL)
