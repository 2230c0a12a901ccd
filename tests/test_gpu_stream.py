"""Streaming append (mp_stream_*): after appending samples one by one and in
chunks, the profile equals the profile of the whole series.

References: the FP64 oracle's brute force of the whole series (P to 1e-12,
I exact where unique), and, on integer data (every value exact), bit-for-bit
equality with Algorithm 1 on the whole series, ties included."""
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


def grow(mp, T, n0, chunks, m, excl, dist, p=2.0, **kw):
    T = np.asarray(T)
    st = mp.StreamProfile(torch.from_numpy(T[:n0].copy()).cuda(), m, excl, dist, p, n_max=T.size, **kw)
    at = n0
    for c in chunks:
        st.append(torch.from_numpy(T[at:at + c].copy()).cuda())
        at += c
    assert at == T.size
    P, I = st.read()
    torch.cuda.synchronize()
    mp.sync_status()
    st.close()
    return P.cpu().numpy(), I.cpu().numpy()


@pytest.mark.parametrize("dist,p", [("euclid", 2.0), ("pnorm", 1.0), ("pnorm", 3.0), ("znorm", 2.0)])
def test_append_equals_whole_series(mp, dist, p):
    s = W.small("motif", 2400, 24, 31, dtype=np.float32)
    P, I = grow(mp, s.T, 1500, [1, 1, 7, 100, 391, 400], s.m, s.excl, dist, p)
    assert P.shape == (s.N,)
    parity.check(s.T, s.m, s.excl, dist, p, P, I, 1e-12, label=f"stream {dist} p={p}")


def test_append_integer_bit_exact(mp):
    rng = np.random.default_rng(5)
    T = rng.integers(-8, 9, 3000).astype(np.float32)
    for excl in (0, 4):
        P, I = grow(mp, T, 800, [1, 3, 96, 1100, 1000], 16, excl, "euclid")
        Pr, Ir = oracle.aamp(T.astype(np.float64), 16, excl)
        np.testing.assert_array_equal(I, Ir)
        np.testing.assert_array_equal(P, Pr)


def test_append_with_frequent_reanchor_and_flat_run(mp):
    s = W.small("flat", 2000, 32, 51, dtype=np.float32)
    P, I = grow(mp, s.T, 1200, [200] * 4, s.m, 8, "znorm", reanchor=50)
    parity.check(s.T, s.m, 8, "znorm", 2.0, P, I, 1e-12, label="stream flat z")


def test_capacity_is_enforced(mp):
    T = torch.zeros(500, dtype=torch.float32, device="cuda")
    st = mp.StreamProfile(T[:400], 16, 4, n_max=450)
    with pytest.raises(mp.MPError) as e:
        st.append(T[:60])
    assert e.value.status == mp.MP_ERR_UNSUPPORTED
    assert st.windows == 400 - 16 + 1
    st.append(T[:50])
    assert st.windows == 450 - 16 + 1
    st.close()
