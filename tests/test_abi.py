"""The C ABI library builds, loads and exports what include/mp.h declares; the
host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_1901_05708_gb300 import build as B
from paper_1901_05708_gb300 import mp

HEADER = os.path.join(B.ROOT, "include", "mp.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return mp.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mp_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_function(lib):
    names = declared_functions()
    assert "mp_aamp" in names and "mp_acamp" in names and "mp_pnorm" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(mp.EXPORTS) <= set(names)


def test_options_and_strings(lib):
    o = mp.Options()
    lib.mp_options_default(ctypes.byref(o))
    assert o.struct_size == ctypes.sizeof(mp.Options)
    assert o.precision == mp.MP_PREC_FP32 and o.polish == 1 and o.k_end == 0
    assert lib.mp_status_string(0) == b"MP_OK"
    assert lib.mp_status_string(3) == b"MP_ERR_WORKSPACE"
    assert lib.mp_version().count(b".") == 2


def test_workspace_size(lib):
    s1 = lib.mp_workspace_size(mp.MP_DIST_EUCLID, mp.MP_F32, 1 << 20, 256, None)
    sz = lib.mp_workspace_size(mp.MP_DIST_ZNORM, mp.MP_F32, 1 << 20, 256, None)
    assert s1 > 8 * (1 << 20) and sz > s1
    assert s1 % 256 == 0
    assert lib.mp_workspace_size(mp.MP_DIST_EUCLID, mp.MP_F32, 10, 11, None) == 0
    assert lib.mp_workspace_size(7, mp.MP_F32, 100, 10, None) == 0


def _call_aamp(lib, T=0x1000, dtype=0, n=100, m=10, excl=2, P=0x2000, I=0x3000, ws=0x10000,
               ws_bytes=1 << 30, opt=None):
    vp = ctypes.c_void_p
    return lib.mp_aamp(vp(T), dtype, n, m, excl, vp(P), vp(I), vp(ws), ws_bytes,
                       ctypes.byref(opt) if opt else None, vp(0))


def test_argument_checks_need_no_gpu(lib):
    """Every rejected call returns before any CUDA call (pointers are fake)."""
    E = mp
    assert _call_aamp(lib, m=0) == E.MP_ERR_INVALID_ARG
    assert _call_aamp(lib, m=101) == E.MP_ERR_INVALID_ARG
    assert _call_aamp(lib, n=0) == E.MP_ERR_INVALID_ARG
    assert _call_aamp(lib, excl=-1) == E.MP_ERR_INVALID_ARG
    assert _call_aamp(lib, dtype=5) == E.MP_ERR_INVALID_ARG
    assert _call_aamp(lib, T=0) == E.MP_ERR_INVALID_ARG
    assert _call_aamp(lib, T=0x1002) == E.MP_ERR_INVALID_ARG          # misaligned
    assert _call_aamp(lib, P=0x2004) == E.MP_ERR_INVALID_ARG
    assert _call_aamp(lib, ws=0) == E.MP_ERR_WORKSPACE
    assert _call_aamp(lib, ws_bytes=16) == E.MP_ERR_WORKSPACE
    assert _call_aamp(lib, ws=0x10010) == E.MP_ERR_INVALID_ARG        # ws not 256-aligned
    assert _call_aamp(lib, n=1 << 32, m=2) == E.MP_ERR_UNSUPPORTED     # N >= 2^31
    assert b"m =" in lib.mp_last_error() or lib.mp_last_error() != b""
    o = mp.Options()
    lib.mp_options_default(ctypes.byref(o))
    o.struct_size = 3
    assert _call_aamp(lib, opt=o) == E.MP_ERR_INVALID_ARG
    lib.mp_options_default(ctypes.byref(o))
    o.precision = 9
    assert _call_aamp(lib, opt=o) == E.MP_ERR_INVALID_ARG
    lib.mp_options_default(ctypes.byref(o))
    o.variant = mp.MP_VARIANT_FAST_FILTER_BOUND + 1
    assert _call_aamp(lib, opt=o) == E.MP_ERR_INVALID_ARG             # no such variant
    lib.mp_options_default(ctypes.byref(o))
    o.tile_rows = 1000
    assert _call_aamp(lib, opt=o) == E.MP_ERR_INVALID_ARG             # not a multiple of 1024
    o.tile_rows = -1024
    assert _call_aamp(lib, opt=o) == E.MP_ERR_INVALID_ARG
    o.tile_rows = 2048
    assert _call_aamp(lib, opt=o) == E.MP_ERR_UNSUPPORTED             # m = 10: the generic kernel's tiles are fixed
    o.tile_rows = 3072
    assert _call_aamp(lib, m=32, opt=o) == E.MP_ERR_UNSUPPORTED       # two-stream tiles: multiples of 2048 rows
    o.variant = mp.MP_VARIANT_FAST                                      # p = 3 on the two-stream kernel, on request
    assert lib.mp_pnorm(ctypes.c_void_p(0x1000), 0, 100, 32, 2, 3.0, ctypes.c_void_p(0x2000), ctypes.c_void_p(0x3000),
                        ctypes.c_void_p(0x10000), 1 << 30, ctypes.byref(o), ctypes.c_void_p(0)) == E.MP_ERR_UNSUPPORTED
    lib.mp_options_default(ctypes.byref(o))
    o.variant = mp.MP_VARIANT_ZRAW
    assert _call_aamp(lib, opt=o) == E.MP_ERR_UNSUPPORTED             # the raw-sum form is Algorithm 2's
    o.variant = mp.MP_VARIANT_ZF
    assert _call_aamp(lib, opt=o) == E.MP_ERR_UNSUPPORTED             # the F comparison is Sec. 4.3's
    o.variant = mp.MP_VARIANT_FAST_FILTER_BOUND
    assert _call_aamp(lib, opt=o) == E.MP_ERR_UNSUPPORTED             # the bound filter is the z kernel's
    o.variant = mp.MP_VARIANT_GENERIC                                   # the z-normalised distance has no generic kernel
    vp = ctypes.c_void_p
    assert lib.mp_acamp(vp(0x1000), 0, 100, 10, 2, vp(0x2000), vp(0x3000), vp(0x10000), 1 << 30,
                        ctypes.byref(o), vp(0)) == E.MP_ERR_UNSUPPORTED
    vp = ctypes.c_void_p
    assert lib.mp_pnorm(vp(0x1000), 0, 100, 10, 2, 0.5, vp(0x2000), vp(0x3000), vp(0x10000), 1 << 30,
                        None, vp(0)) == E.MP_ERR_INVALID_ARG
    assert lib.mp_acamp(vp(0x1000), 0, 100, 1, 2, vp(0x2000), vp(0x3000), vp(0x10000), 1 << 30,
                        None, vp(0)) == E.MP_ERR_INVALID_ARG


def test_batch_checks_need_no_gpu(lib):
    """mp_batch_plan_create validates the whole description before any CUDA call."""
    E = mp

    def create(lengths=(100, 50), m=(10, 8), dist=(0, 2), excl=(2, 2), p=2.0, dtype=None, opt=None,
               **patch):
        desc, keep = mp.batch_desc(lengths, m, dist, excl, p)
        if dtype is not None:
            desc.dtype = dtype
        for k, v in patch.items():
            setattr(desc, k, v)
        h = ctypes.c_void_p()
        nb = ctypes.c_size_t()
        st = lib.mp_batch_plan_create(ctypes.byref(desc), ctypes.byref(opt) if opt else None,
                                      ctypes.byref(h), ctypes.byref(nb))
        assert not h.value  # nothing was created
        return st

    assert create(num_series=0) == E.MP_ERR_INVALID_ARG
    assert create(struct_size=8) == E.MP_ERR_INVALID_ARG
    assert create(m=(10, 51)) == E.MP_ERR_INVALID_ARG           # m > n
    assert create(m=(0, 8)) == E.MP_ERR_INVALID_ARG
    assert create(lengths=(100, 0)) == E.MP_ERR_INVALID_ARG     # empty series
    assert create(dist=(0, 7)) == E.MP_ERR_INVALID_ARG
    assert create(m=(10, 1)) == E.MP_ERR_INVALID_ARG            # z-normalised with m = 1
    assert create(excl=(-1, 2)) == E.MP_ERR_INVALID_ARG
    assert create(dist=(1, 0), p=0.5) == E.MP_ERR_INVALID_ARG   # p < 1 for a p-norm series
    assert create(dtype=mp.MP_F64) == E.MP_ERR_UNSUPPORTED
    assert create(dtype=9) == E.MP_ERR_INVALID_ARG
    o = mp.Options()
    lib.mp_options_default(ctypes.byref(o))
    o.precision = mp.MP_PREC_FP64
    assert create(opt=o) == E.MP_ERR_UNSUPPORTED
    lib.mp_options_default(ctypes.byref(o))
    o.k_end = 5
    assert create(opt=o) == E.MP_ERR_UNSUPPORTED
    assert b"diagonal" in lib.mp_last_error()
    h = ctypes.c_void_p()
    assert lib.mp_batch_plan_create(None, None, ctypes.byref(h), None) == E.MP_ERR_INVALID_ARG
    assert lib.mp_batch_run(None, None, None, None, None, 0, None) == E.MP_ERR_INVALID_ARG
    assert lib.mp_batch_windows(None) == -1 and lib.mp_batch_tiles(None) == -1
    assert lib.mp_batch_plan_destroy(None) == E.MP_OK


def test_stream_checks_need_no_gpu(lib):
    """mp_stream_create rejects bad arguments before any CUDA call."""
    E = mp
    vp = ctypes.c_void_p

    def create(dist=0, T=0x1000, dtype=0, n=100, n_max=200, m=10, excl=2, p=2.0, opt=None):
        h = vp()
        st = lib.mp_stream_create(dist, vp(T), dtype, n, n_max, m, excl, p, ctypes.byref(opt) if opt else None,
                                  ctypes.byref(h), vp(0))
        assert not h.value
        return st

    assert create(dist=5) == E.MP_ERR_INVALID_ARG
    assert create(n_max=50) == E.MP_ERR_INVALID_ARG         # n_max < n
    assert create(m=101) == E.MP_ERR_INVALID_ARG            # m > n
    assert create(T=0) == E.MP_ERR_INVALID_ARG
    assert create(dist=2, m=1) == E.MP_ERR_INVALID_ARG      # z-normalised with m = 1
    assert create(dist=1, p=0.5) == E.MP_ERR_INVALID_ARG
    o = mp.Options()
    lib.mp_options_default(ctypes.byref(o))
    o.k_begin = 3
    assert create(opt=o) == E.MP_ERR_UNSUPPORTED
    assert lib.mp_stream_append(None, vp(0x1000), 0, 1, vp(0)) == E.MP_ERR_INVALID_ARG
    assert lib.mp_stream_read(None, vp(0x1000), vp(0x2000), vp(0)) == E.MP_ERR_INVALID_ARG
    assert lib.mp_stream_windows(None) == -1
    assert lib.mp_stream_destroy(None) == E.MP_OK


def test_autotune_cache_files_need_no_gpu(lib, tmp_path):
    E = mp
    good = tmp_path / "cache.txt"
    good.write_text("# comment\nNVIDIA_GB300|0|0|256|20|2 1 0 132.5\nNVIDIA_GB300|1|0|128|18|3 2 0 9.1\n")
    n0 = lib.mp_autotune_cache_size()
    assert lib.mp_autotune_cache_load(str(good).encode()) == E.MP_OK
    assert lib.mp_autotune_cache_size() == n0 + 2
    out = tmp_path / "out.txt"
    assert lib.mp_autotune_cache_save(str(out).encode()) == E.MP_OK
    assert "NVIDIA_GB300|0|0|256|20|2 1 0" in out.read_text()
    bad = tmp_path / "bad.txt"
    bad.write_text("key 9 0 1.0\n")
    assert lib.mp_autotune_cache_load(str(bad).encode()) == E.MP_ERR_INVALID_ARG
    assert lib.mp_autotune_cache_load(str(tmp_path / "missing.txt").encode()) == E.MP_ERR_INVALID_ARG
    o = mp.Options()
    lib.mp_options_default(ctypes.byref(o))
    o.variant = mp.MP_VARIANT_FAST_FILTER_BOUND + 1
    assert _call_aamp(lib, opt=o) == E.MP_ERR_INVALID_ARG
    # five-field entries (with tile_rows) load too; a tile_rows that is not a multiple of 1024 does not
    five = tmp_path / "five.txt"
    five.write_text("NVIDIA_GB300|2|0|512|20|2 2 0 175.0 16384\n")
    assert lib.mp_autotune_cache_load(str(five).encode()) == E.MP_OK
    assert lib.mp_autotune_cache_save(str(out).encode()) == E.MP_OK
    assert "NVIDIA_GB300|2|0|512|20|2 2 0 175.000000 16384" in out.read_text()
    five.write_text("NVIDIA_GB300|2|0|512|20|2 2 0 175.0 1000\n")
    assert lib.mp_autotune_cache_load(str(five).encode()) == E.MP_ERR_INVALID_ARG


def test_binding_refuses_cpu_tensors(lib):
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):
        mp.aamp(torch.zeros(100), 10, 2)
