"""Python binding of libmp (include/mp.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module only
turns torch tensors into pointers, owns a cached device workspace, and maps
status codes to exceptions.  There is no CPU fallback: if the library cannot
be loaded, every call raises.

    P, I = aamp(T, m, excl)            # pure Euclidean   (Algorithm 1)
    P, I = pnorm(T, m, excl, p)        # p-norm           (Algorithm 3)
    P, I = acamp(T, m, excl)           # z-normalised     (Algorithm 2)
    plan = BatchPlan(lengths, ms, dists, excls)   # many series, one graph
    P, I = plan.run(T_concat)
    st = StreamProfile(T, m, excl, n_max=...)     # append samples, profile kept exact
    st.append(x); P, I = st.read()

T is a 1-D float32/float64 CUDA tensor; P (float64) and I (int64) come back
on the same device.  Calls are asynchronous on the current torch stream.
"""
from __future__ import annotations

import ctypes
import threading

import torch

from . import build as _build

MP_OK, MP_ERR_INVALID_ARG, MP_ERR_UNSUPPORTED, MP_ERR_WORKSPACE, MP_ERR_CUDA, MP_ERR_INTERNAL = range(6)
MP_F32, MP_F64 = 0, 1
MP_PREC_FP32, MP_PREC_FP64 = 0, 1
MP_DIST_EUCLID, MP_DIST_PNORM, MP_DIST_ZNORM = 0, 1, 2
(MP_VARIANT_AUTO, MP_VARIANT_FAST_FILTER, MP_VARIANT_FAST, MP_VARIANT_GENERIC, MP_VARIANT_TALL, MP_VARIANT_ZRAW,
 MP_VARIANT_ZF, MP_VARIANT_CACHED, MP_VARIANT_FAST_FILTER_BOUND) = range(9)

EXPORTS = ("mp_options_default", "mp_workspace_size", "mp_aamp", "mp_pnorm", "mp_acamp",
           "mp_sync_status", "mp_last_error", "mp_status_string", "mp_version", "mp_launch_count",
           "mp_set_sweep_events", "mp_aamp_noalloc", "mp_batch_plan_create", "mp_batch_run",
           "mp_batch_windows", "mp_batch_tiles", "mp_batch_plan_destroy", "mp_stream_create",
           "mp_stream_append", "mp_stream_read", "mp_stream_windows", "mp_stream_destroy",
           "mp_anytime_create", "mp_anytime_run", "mp_anytime_read", "mp_anytime_tiles_done",
           "mp_anytime_tiles_total", "mp_anytime_checkpoint_size", "mp_anytime_checkpoint",
           "mp_anytime_restore", "mp_anytime_destroy", "mp_autotune", "mp_autotune_cache_save",
           "mp_autotune_cache_load", "mp_autotune_cache_size")


class MPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_STATUS = {0: "MP_OK", 1: "MP_ERR_INVALID_ARG", 2: "MP_ERR_UNSUPPORTED", 3: "MP_ERR_WORKSPACE",
           4: "MP_ERR_CUDA", 5: "MP_ERR_INTERNAL"}


class Options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("precision", ctypes.c_int32),
                ("reanchor", ctypes.c_int32), ("polish", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("tile_rows", ctypes.c_int32), ("k_begin", ctypes.c_int64),
                ("k_end", ctypes.c_int64)]


class BatchDesc(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("num_series", ctypes.c_int32),
                ("t_offsets", ctypes.POINTER(ctypes.c_int64)), ("m", ctypes.POINTER(ctypes.c_int32)),
                ("dist", ctypes.POINTER(ctypes.c_uint8)), ("excl", ctypes.POINTER(ctypes.c_int64)),
                ("p", ctypes.c_double), ("dtype", ctypes.c_int32), ("reserved0", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Open libmp.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(path or _build.build())
        vp, i32, i64, sz, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double
        opt_p = ctypes.POINTER(Options)
        lib.mp_options_default.argtypes = [opt_p]
        lib.mp_options_default.restype = None
        lib.mp_workspace_size.argtypes = [ctypes.c_int, ctypes.c_int, i64, i32, opt_p]
        lib.mp_workspace_size.restype = sz
        lib.mp_aamp.argtypes = [vp, ctypes.c_int, i64, i32, i64, vp, vp, vp, sz, opt_p, vp]
        lib.mp_aamp.restype = ctypes.c_int
        lib.mp_pnorm.argtypes = [vp, ctypes.c_int, i64, i32, i64, d, vp, vp, vp, sz, opt_p, vp]
        lib.mp_pnorm.restype = ctypes.c_int
        lib.mp_acamp.argtypes = [vp, ctypes.c_int, i64, i32, i64, vp, vp, vp, sz, opt_p, vp]
        lib.mp_acamp.restype = ctypes.c_int
        lib.mp_sync_status.argtypes = [vp]
        lib.mp_sync_status.restype = ctypes.c_int
        lib.mp_last_error.argtypes = []
        lib.mp_last_error.restype = ctypes.c_char_p
        lib.mp_status_string.argtypes = [ctypes.c_int]
        lib.mp_status_string.restype = ctypes.c_char_p
        lib.mp_version.argtypes = []
        lib.mp_version.restype = ctypes.c_char_p
        lib.mp_launch_count.argtypes = []
        lib.mp_launch_count.restype = ctypes.c_uint64
        lib.mp_set_sweep_events.argtypes = [vp, vp]
        lib.mp_set_sweep_events.restype = ctypes.c_int
        lib.mp_aamp_noalloc.argtypes = [vp, ctypes.c_int, i64, i32, i64, vp, vp, opt_p, vp]
        lib.mp_aamp_noalloc.restype = ctypes.c_int
        lib.mp_batch_plan_create.argtypes = [ctypes.POINTER(BatchDesc), opt_p, ctypes.POINTER(vp),
                                             ctypes.POINTER(sz)]
        lib.mp_batch_plan_create.restype = ctypes.c_int
        lib.mp_batch_run.argtypes = [vp, vp, vp, vp, vp, sz, vp]
        lib.mp_batch_run.restype = ctypes.c_int
        lib.mp_batch_windows.argtypes = [vp]
        lib.mp_batch_windows.restype = i64
        lib.mp_batch_tiles.argtypes = [vp]
        lib.mp_batch_tiles.restype = i64
        lib.mp_batch_plan_destroy.argtypes = [vp]
        lib.mp_batch_plan_destroy.restype = ctypes.c_int
        lib.mp_stream_create.argtypes = [ctypes.c_int, vp, ctypes.c_int, i64, i64, i32, i64, d, opt_p,
                                         ctypes.POINTER(vp), vp]
        lib.mp_stream_create.restype = ctypes.c_int
        lib.mp_stream_append.argtypes = [vp, vp, ctypes.c_int, i64, vp]
        lib.mp_stream_append.restype = ctypes.c_int
        lib.mp_stream_read.argtypes = [vp, vp, vp, vp]
        lib.mp_stream_read.restype = ctypes.c_int
        lib.mp_stream_windows.argtypes = [vp]
        lib.mp_stream_windows.restype = i64
        lib.mp_stream_destroy.argtypes = [vp]
        lib.mp_stream_destroy.restype = ctypes.c_int
        lib.mp_anytime_create.argtypes = [ctypes.c_int, vp, i64, i32, i64, d, ctypes.c_uint64, opt_p,
                                          ctypes.POINTER(vp), vp]
        lib.mp_anytime_create.restype = ctypes.c_int
        lib.mp_anytime_run.argtypes = [vp, i64, vp]
        lib.mp_anytime_run.restype = ctypes.c_int
        lib.mp_anytime_read.argtypes = [vp, vp, vp, vp]
        lib.mp_anytime_read.restype = ctypes.c_int
        lib.mp_anytime_tiles_done.argtypes = [vp]
        lib.mp_anytime_tiles_done.restype = i64
        lib.mp_anytime_tiles_total.argtypes = [vp]
        lib.mp_anytime_tiles_total.restype = i64
        lib.mp_anytime_checkpoint_size.argtypes = [vp]
        lib.mp_anytime_checkpoint_size.restype = sz
        lib.mp_anytime_checkpoint.argtypes = [vp, vp, sz, vp]
        lib.mp_anytime_checkpoint.restype = ctypes.c_int
        lib.mp_anytime_restore.argtypes = [vp, vp, sz, vp]
        lib.mp_anytime_restore.restype = ctypes.c_int
        lib.mp_anytime_destroy.argtypes = [vp]
        lib.mp_anytime_destroy.restype = ctypes.c_int
        lib.mp_autotune.argtypes = [ctypes.c_int, vp, ctypes.c_int, i64, i32, i64, d, vp, vp, vp, sz, opt_p, i64,
                                    ctypes.c_int, opt_p, ctypes.POINTER(d), i32, ctypes.POINTER(i32), vp]
        lib.mp_autotune.restype = ctypes.c_int
        lib.mp_autotune_cache_save.argtypes = [ctypes.c_char_p]
        lib.mp_autotune_cache_save.restype = ctypes.c_int
        lib.mp_autotune_cache_load.argtypes = [ctypes.c_char_p]
        lib.mp_autotune_cache_load.restype = ctypes.c_int
        lib.mp_autotune_cache_size.argtypes = []
        lib.mp_autotune_cache_size.restype = i64
        _lib = lib
        return lib


def options(precision: str = "fp32", reanchor: int = 0, polish: bool = True,
            k_range: tuple[int, int] | None = None, variant: int = MP_VARIANT_AUTO, tile_rows: int = 0) -> Options:
    """mp_options for the calls below.  variant (include/mp.h, mp_variant): MP_VARIANT_AUTO;
    MP_VARIANT_FAST_FILTER / MP_VARIANT_FAST: the two-stream kernel with / without its block
    filter (the z-normalised kernel with / without its filter for acamp); MP_VARIANT_GENERIC;
    MP_VARIANT_TALL; MP_VARIANT_ZRAW: Algorithm 2's raw-sum form, an ablation (acamp only);
    MP_VARIANT_ZF: the same raw sums compared through Sec. 4.3's F, an ablation (acamp only);
    MP_VARIANT_CACHED: the autotuner's cached choice if there is one; MP_VARIANT_FAST_FILTER_BOUND: the
    z-normalised kernel's filter on a looser, cheaper bound (acamp only).  tile_rows: rows per tile of
    the two-stream kernel (a multiple of 2048) and of the tall-tile kernels (a multiple of 1024); 0: the
    default."""
    o = Options()
    load().mp_options_default(ctypes.byref(o))
    o.precision = {"fp32": MP_PREC_FP32, "fp64": MP_PREC_FP64}[precision]
    o.reanchor = int(reanchor)
    o.polish = 1 if polish else 0
    o.variant = int(variant)
    o.tile_rows = int(tile_rows)
    if k_range is not None:
        o.k_begin, o.k_end = int(k_range[0]), int(k_range[1])
    return o


def _check(status: int):
    if status != MP_OK:
        raise MPError(status, load().mp_last_error().decode())


def workspace_size(dist: int, dtype: int, n: int, m: int, opt: Options | None = None) -> int:
    return int(load().mp_workspace_size(dist, dtype, n, m, ctypes.byref(opt) if opt else None))


_ws_cache: dict = {}


def _workspace(device: torch.device, nbytes: int) -> torch.Tensor:
    """A cached uint8 device buffer of at least nbytes, 256-byte aligned."""
    key = device.index if device.index is not None else torch.cuda.current_device()
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)
        _ws_cache[key] = buf
    return buf


def _prep(T: torch.Tensor):
    if not isinstance(T, torch.Tensor) or not T.is_cuda:
        raise TypeError("T must be a CUDA tensor (the library has no CPU path)")
    if T.dim() != 1:
        raise ValueError("T must be 1-D")
    if T.dtype not in (torch.float32, torch.float64):
        raise TypeError("T must be float32 or float64")
    T = T.contiguous()
    return T, MP_F32 if T.dtype == torch.float32 else MP_F64


def _call(fn_name: str, dist: int, T, m: int, excl: int, p: float | None, opt: Options,
          out=None, stream=None):
    lib = load()
    T, dtype = _prep(T)
    n = T.numel()
    N = n - m + 1
    if out is None:
        P = torch.empty(max(N, 0), dtype=torch.float64, device=T.device)
        I = torch.empty(max(N, 0), dtype=torch.int64, device=T.device)
    else:
        P, I = out
    nbytes = lib.mp_workspace_size(dist, dtype, n, m, ctypes.byref(opt))
    if nbytes == 0:
        # invalid sizes: let the entry point report the precise error
        nbytes = 256
    ws = _workspace(T.device, nbytes)
    s = stream if stream is not None else torch.cuda.current_stream(T.device)
    sp = ctypes.c_void_p(s.cuda_stream)
    args = [ctypes.c_void_p(T.data_ptr()), dtype, n, m, excl]
    if p is not None:
        args.append(float(p))
    args += [ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(I.data_ptr()),
             ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.byref(opt), sp]
    _check(getattr(lib, fn_name)(*args))
    return P, I


def aamp(T, m: int, excl: int, *, precision="fp32", reanchor=0, polish=True, k_range=None, variant=0,
         tile_rows=0, out=None, stream=None):
    """Matrix profile with the pure Euclidean distance (Algorithm 1)."""
    return _call("mp_aamp", MP_DIST_EUCLID, T, m, excl, None,
                 options(precision, reanchor, polish, k_range, variant, tile_rows), out, stream)


def pnorm(T, m: int, excl: int, p: float, *, precision="fp32", reanchor=0, polish=True,
          k_range=None, variant=0, tile_rows=0, out=None, stream=None):
    """Matrix profile with the p-norm distance (Algorithm 3).  For p = 3 with a
    float32 series the default FP32 kernel carries error-free window sums
    (include/mp.h, mp_variant); variant=MP_VARIANT_FAST runs the faster
    re-anchored two-stream kernel, which can miss the FP32 tolerance on series
    whose terms |x - y|^3 span many orders of magnitude."""
    return _call("mp_pnorm", MP_DIST_PNORM, T, m, excl, p,
                 options(precision, reanchor, polish, k_range, variant, tile_rows), out, stream)


def acamp(T, m: int, excl: int, *, precision="fp32", reanchor=0, polish=True, k_range=None, variant=0,
          tile_rows=0, out=None, stream=None):
    """Matrix profile with the z-normalised Euclidean distance (Algorithm 2)."""
    return _call("mp_acamp", MP_DIST_ZNORM, T, m, excl, None,
                 options(precision, reanchor, polish, k_range, variant, tile_rows), out, stream)


def sync_status(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(load().mp_sync_status(ctypes.c_void_p(s.cuda_stream)))


def profile(T, m, excl, dist="euclid", p=2.0, **kw):
    if dist in ("euclid", MP_DIST_EUCLID):
        return aamp(T, m, excl, **kw)
    if dist in ("pnorm", MP_DIST_PNORM):
        return pnorm(T, m, excl, p, **kw)
    return acamp(T, m, excl, **kw)


_DIST_CODES = {"euclid": MP_DIST_EUCLID, "pnorm": MP_DIST_PNORM, "znorm": MP_DIST_ZNORM}


def batch_desc(lengths, m, dist, excl, p: float = 2.0):
    """An mp_batch_desc over host arrays (kept alive in the returned tuple)."""
    import numpy as np
    lengths = np.asarray(lengths, dtype=np.int64)
    S = lengths.size
    offs = np.zeros(S + 1, dtype=np.int64)
    np.cumsum(lengths, out=offs[1:])
    ms = np.ascontiguousarray(np.broadcast_to(np.asarray(m, dtype=np.int32), (S,)))
    d = [_DIST_CODES.get(x, x) if isinstance(x, str) else int(x) for x in np.atleast_1d(dist)]
    ds = np.ascontiguousarray(np.broadcast_to(np.asarray(d, dtype=np.uint8), (S,)))
    ex = np.ascontiguousarray(np.broadcast_to(np.asarray(excl, dtype=np.int64), (S,)))
    desc = BatchDesc()
    desc.struct_size = ctypes.sizeof(BatchDesc)
    desc.num_series = S
    desc.t_offsets = offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    desc.m = ms.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    desc.dist = ds.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    desc.excl = ex.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    desc.p = float(p)
    desc.dtype = MP_F32
    return desc, (offs, ms, ds, ex)


class BatchPlan:
    """Matrix profiles of many float32 series in one graph launch (mp_batch_*).

    lengths[s], m[s], dist[s] ('euclid' | 'pnorm' | 'znorm' or mp_dist codes)
    and excl[s] describe series s; p is the exponent of every p-norm series.
    run(T) takes the series concatenated in one float32 CUDA tensor and
    returns (P, I) concatenated: series s at out_offsets[s] .. out_offsets[s+1],
    I within the series.  The plan keeps its workspace, so that repeated runs
    with the same output buffers replay the same graph."""

    def __init__(self, lengths, m, dist, excl, p: float = 2.0, polish: bool = True, device=None, variant: int = 0,
                 tile_rows: int = 0):
        import numpy as np
        lib = load()
        self._desc, keep = batch_desc(lengths, m, dist, excl, p)
        offs, ms, _, _ = keep
        self.t_offsets = offs
        N = (offs[1:] - offs[:-1]) - ms + 1
        self.out_offsets = np.zeros(N.size + 1, dtype=np.int64)
        np.cumsum(N, out=self.out_offsets[1:])
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index)
        opt = options(polish=polish, variant=variant, tile_rows=tile_rows)
        h = ctypes.c_void_p()
        nbytes = ctypes.c_size_t()
        with torch.cuda.device(self.device):
            _check(lib.mp_batch_plan_create(ctypes.byref(self._desc), ctypes.byref(opt), ctypes.byref(h),
                                            ctypes.byref(nbytes)))
        self._h = h
        self.windows = int(lib.mp_batch_windows(h))
        self.tiles = int(lib.mp_batch_tiles(h))
        self.ws_bytes = int(nbytes.value)
        self._ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=self.device)

    def run(self, T: torch.Tensor, out=None, stream=None):
        if self._h is None:
            raise RuntimeError("plan is closed")
        if not isinstance(T, torch.Tensor) or not T.is_cuda or T.dtype != torch.float32 or T.dim() != 1:
            raise TypeError("T must be a 1-D float32 CUDA tensor")
        if T.numel() != int(self.t_offsets[-1]):
            raise ValueError(f"T has {T.numel()} samples, the plan {int(self.t_offsets[-1])}")
        T = T.contiguous()
        if out is None:
            P = torch.empty(self.windows, dtype=torch.float64, device=T.device)
            I = torch.empty(self.windows, dtype=torch.int64, device=T.device)
        else:
            P, I = out
        s = stream if stream is not None else torch.cuda.current_stream(T.device)
        _check(load().mp_batch_run(self._h, ctypes.c_void_p(T.data_ptr()), ctypes.c_void_p(P.data_ptr()),
                                   ctypes.c_void_p(I.data_ptr()), ctypes.c_void_p(self._ws.data_ptr()),
                                   self._ws.numel(), ctypes.c_void_p(s.cuda_stream)))
        return P, I

    def close(self):
        """Free the plan (after waiting for the device: a run may still be in flight)."""
        if getattr(self, "_h", None) is not None:
            torch.cuda.synchronize(self.device)
            load().mp_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class StreamProfile:
    """A matrix profile kept current while samples are appended (mp_stream_*).

    StreamProfile(T, m, excl, dist='euclid', p=2.0, n_max=None) computes the
    profile of T (1-D CUDA tensor) with room for n_max samples in all;
    append(x) adds samples (a CUDA tensor), read() returns (P, I) of the
    series so far."""

    def __init__(self, T, m: int, excl: int, dist="euclid", p: float = 2.0, n_max: int | None = None,
                 precision: str = "fp32", reanchor: int = 0, stream=None):
        lib = load()
        T, dtype = _prep(T)
        self.device = T.device
        n = T.numel()
        n_max = n if n_max is None else int(n_max)
        code = _DIST_CODES.get(dist, dist) if isinstance(dist, str) else int(dist)
        opt = options(precision, reanchor, True)
        h = ctypes.c_void_p()
        s = stream if stream is not None else torch.cuda.current_stream(T.device)
        _check(lib.mp_stream_create(code, ctypes.c_void_p(T.data_ptr()), dtype, n, n_max, m, excl, float(p),
                                    ctypes.byref(opt), ctypes.byref(h), ctypes.c_void_p(s.cuda_stream)))
        self._h = h
        self._keep = T  # the input must outlive the asynchronous initial profile

    @property
    def windows(self) -> int:
        return int(load().mp_stream_windows(self._h))

    def append(self, x, stream=None):
        x, dtype = _prep(x)
        s = stream if stream is not None else torch.cuda.current_stream(x.device)
        _check(load().mp_stream_append(self._h, ctypes.c_void_p(x.data_ptr()), dtype, x.numel(),
                                       ctypes.c_void_p(s.cuda_stream)))
        self._keep = x

    def read(self, stream=None):
        N = self.windows
        P = torch.empty(N, dtype=torch.float64, device=self.device)
        I = torch.empty(N, dtype=torch.int64, device=self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        _check(load().mp_stream_read(self._h, ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(I.data_ptr()),
                                     ctypes.c_void_p(s.cuda_stream)))
        return P, I

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            torch.cuda.synchronize(self.device)
            load().mp_stream_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Anytime:
    """An anytime matrix profile (mp_anytime_*): tiles in a seeded random order,
    run(k) evaluates the next k tiles, read() gives the profile of the cells
    done so far, checkpoint() / restore() save and load the progress."""

    def __init__(self, T, m: int, excl: int, dist="euclid", p: float = 2.0, seed: int = 1, polish: bool = True,
                 stream=None):
        lib = load()
        if not isinstance(T, torch.Tensor) or not T.is_cuda or T.dtype != torch.float32 or T.dim() != 1:
            raise TypeError("T must be a 1-D float32 CUDA tensor")
        T = T.contiguous()
        self.device = T.device
        self.N = T.numel() - m + 1
        code = _DIST_CODES.get(dist, dist) if isinstance(dist, str) else int(dist)
        opt = options(polish=polish)
        h = ctypes.c_void_p()
        s = stream if stream is not None else torch.cuda.current_stream(T.device)
        _check(lib.mp_anytime_create(code, ctypes.c_void_p(T.data_ptr()), T.numel(), m, excl, float(p), int(seed),
                                     ctypes.byref(opt), ctypes.byref(h), ctypes.c_void_p(s.cuda_stream)))
        self._h = h
        self._keep = T

    @property
    def tiles_done(self) -> int:
        return int(load().mp_anytime_tiles_done(self._h))

    @property
    def tiles_total(self) -> int:
        return int(load().mp_anytime_tiles_total(self._h))

    def run(self, max_tiles: int, stream=None):
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        _check(load().mp_anytime_run(self._h, int(max_tiles), ctypes.c_void_p(s.cuda_stream)))

    def read(self, stream=None):
        P = torch.empty(self.N, dtype=torch.float64, device=self.device)
        I = torch.empty(self.N, dtype=torch.int64, device=self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        _check(load().mp_anytime_read(self._h, ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(I.data_ptr()),
                                      ctypes.c_void_p(s.cuda_stream)))
        return P, I

    def checkpoint(self) -> bytes:
        lib = load()
        n = int(lib.mp_anytime_checkpoint_size(self._h))
        buf = torch.empty(n, dtype=torch.uint8).pin_memory()
        s = torch.cuda.current_stream(self.device)
        _check(lib.mp_anytime_checkpoint(self._h, ctypes.c_void_p(buf.data_ptr()), n, ctypes.c_void_p(s.cuda_stream)))
        torch.cuda.synchronize(self.device)
        return bytes(buf.numpy().tobytes())

    def restore(self, blob: bytes):
        lib = load()
        buf = torch.frombuffer(bytearray(blob), dtype=torch.uint8).pin_memory()
        s = torch.cuda.current_stream(self.device)
        _check(lib.mp_anytime_restore(self._h, ctypes.c_void_p(buf.data_ptr()), buf.numel(),
                                      ctypes.c_void_p(s.cuda_stream)))
        torch.cuda.synchronize(self.device)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            torch.cuda.synchronize(self.device)
            load().mp_anytime_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(T, m: int, excl: int, dist="euclid", p: float = 2.0, precision: str = "fp32",
             slice_cells: int = 0, force: bool = False, stream=None):
    """Time the kernel variants for this problem (mp_autotune); returns
    (kwargs for aamp / pnorm / acamp / profile, candidate times in ms)."""
    lib = load()
    T, dtype = _prep(T)
    n = T.numel()
    N = n - m + 1
    code = _DIST_CODES.get(dist, dist) if isinstance(dist, str) else int(dist)
    opt = options(precision)
    nbytes = max(int(lib.mp_workspace_size(code, dtype, n, m, ctypes.byref(opt))), 256)
    ws = _workspace(T.device, nbytes)
    P = torch.empty(max(N, 1), dtype=torch.float64, device=T.device)
    I = torch.empty(max(N, 1), dtype=torch.int64, device=T.device)
    best = Options()
    times = (ctypes.c_double * 8)()
    nt = ctypes.c_int32()
    s = stream if stream is not None else torch.cuda.current_stream(T.device)
    _check(lib.mp_autotune(code, ctypes.c_void_p(T.data_ptr()), dtype, n, m, excl, float(p),
                           ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(I.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                           ws.numel(), ctypes.byref(opt), int(slice_cells), 1 if force else 0, ctypes.byref(best),
                           times, 8, ctypes.byref(nt), ctypes.c_void_p(s.cuda_stream)))
    return ({"precision": precision, "reanchor": best.reanchor, "variant": best.variant,
             "tile_rows": best.tile_rows},
            [times[i] for i in range(nt.value)])


def autotune_cache_save(path: str):
    _check(load().mp_autotune_cache_save(path.encode()))


def autotune_cache_load(path: str):
    _check(load().mp_autotune_cache_load(path.encode()))


def autotune_cache_size() -> int:
    return int(load().mp_autotune_cache_size())
