"""mp_aamp_noalloc: the Euclidean profile for callers that cannot allocate
device memory (a host framework that owns every allocation, or a service that
forbids allocation after start-up).  It runs on a static scratch array inside
the library instead of a caller workspace, and must give what mp_aamp gives.

Named test_zz_* so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

from paper_1901_05708_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL32 = 1e-5


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_05708_gb300 import mp
    L = mp.load()
    vp = ctypes.c_void_p
    L.mp_aamp_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                  vp, vp, ctypes.POINTER(mp.Options), vp]
    L.mp_aamp_noalloc.restype = ctypes.c_int
    return L


def _noalloc(lib, T, m, excl, **kw):
    from paper_1901_05708_gb300 import mp
    N = T.numel() - m + 1
    P = torch.full((N,), -1.0, dtype=torch.float64, device=T.device)
    I = torch.full((N,), -7, dtype=torch.int64, device=T.device)
    opt = mp.options(**kw)
    stream = torch.cuda.current_stream(T.device)
    st = lib.mp_aamp_noalloc(ctypes.c_void_p(T.data_ptr()), mp.MP_F32, T.numel(), m, excl,
                             ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(I.data_ptr()),
                             ctypes.byref(opt), ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, lib.mp_last_error()
    torch.cuda.synchronize()
    return P.cpu().numpy(), I.cpu().numpy()


def test_noalloc_matches_workspace_entry_point(lib):
    from paper_1901_05708_gb300 import mp
    for seed, n, m in ((3, 20_000, 64), (4, 9_000, 40)):
        s = W.small("motif", n, m, seed, dtype=np.float32)
        T = torch.from_numpy(s.T).cuda()
        Pw, Iw = mp.aamp(T, s.m, s.excl)
        torch.cuda.synchronize()
        Pw, Iw = Pw.cpu().numpy(), Iw.cpu().numpy()
        for _ in range(2):  # two calls in a row share the scratch
            P, I = _noalloc(lib, T, s.m, s.excl)
            np.testing.assert_allclose(P, Pw, rtol=RTOL32, atol=0)
            np.testing.assert_array_equal(I, Iw)


@pytest.mark.parametrize("n,m,kw", [
    (300_000, 256, {}),                        # long series: the kernel with the block filter
    (3_000, 20, {"precision": "fp64"}),        # the FP64 sweep (128-bit keys)
    (20_000, 64, {"k_range": (500, 7_000)}),   # a diagonal range
])
def test_noalloc_other_kernels(lib, n, m, kw):
    """The scratch also serves the filtered kernel of long series, the FP64
    sweep and diagonal ranges: two calls in a row equal mp_aamp's result."""
    from paper_1901_05708_gb300 import mp
    s = W.small("motif", n, m, 17, dtype=np.float32)
    T = torch.from_numpy(s.T).cuda()
    Pw, Iw = mp.aamp(T, s.m, s.excl, **kw)
    torch.cuda.synchronize()
    Pw, Iw = Pw.cpu().numpy(), Iw.cpu().numpy()
    rtol = 1e-12 if kw.get("precision") == "fp64" else RTOL32
    for _ in range(2):
        P, I = _noalloc(lib, T, s.m, s.excl, **kw)
        np.testing.assert_allclose(P, Pw, rtol=rtol, atol=0)
        np.testing.assert_array_equal(I, Iw)


def test_noalloc_checks_arguments_first(lib):
    """Bad arguments get mp_aamp's status (MP_ERR_INVALID_ARG) before any
    scratch lookup, and nothing is written."""
    from paper_1901_05708_gb300 import mp
    T = torch.zeros(100, dtype=torch.float32, device="cuda")
    P = torch.full((91,), -1.0, dtype=torch.float64, device="cuda")
    I = torch.full((91,), -7, dtype=torch.int64, device="cuda")
    for args in ((ctypes.c_void_p(0), mp.MP_F32, 100, 10), (ctypes.c_void_p(T.data_ptr()), 7, 100, 10),
                 (ctypes.c_void_p(T.data_ptr()), mp.MP_F32, 100, 0)):
        st = lib.mp_aamp_noalloc(*args, 2, ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(I.data_ptr()), None,
                                 ctypes.c_void_p(0))
        assert st == mp.MP_ERR_INVALID_ARG, lib.mp_last_error()
    torch.cuda.synchronize()
    assert torch.all(P == -1.0) and torch.all(I == -7)


def test_noalloc_rejects_oversized_problem(lib):
    from paper_1901_05708_gb300 import mp
    n = 3_000_000  # workspace well above the 32 MiB scratch
    assert mp.workspace_size(mp.MP_DIST_EUCLID, mp.MP_F32, n, 256) > 32 << 20
    T = torch.zeros(n, dtype=torch.float32, device="cuda")
    P = torch.empty(n, dtype=torch.float64, device="cuda")
    I = torch.empty(n, dtype=torch.int64, device="cuda")
    st = lib.mp_aamp_noalloc(ctypes.c_void_p(T.data_ptr()), mp.MP_F32, n, 256, 64,
                             ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(I.data_ptr()), None,
                             ctypes.c_void_p(0))
    assert st == mp.MP_ERR_UNSUPPORTED
    assert b"scratch" in lib.mp_last_error()
