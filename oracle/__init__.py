"""FP64 CPU oracle for the matrix-profile sweep (arXiv:1901.05708).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline
leg of ``bench.py`` use it; the product path never imports it and shares no
code with it.  The arithmetic lives in ``mp_oracle.c`` (plain C, compensated
FP64 sums); this module compiles it with gcc and exposes numpy-level calls.

Functions and the passages they follow
  brute(...)          nested-loop definition: Def. 2.3/2.4 with the distances
                      of Sec. 2 (Euclidean, p-norm, z-normalised).
  brute_rows(...)     the same for selected rows, plus the runner-up value.
  aamp(...)           Algorithm 1 (Lemma 1 recurrence).
  pnorm(...)          Algorithm 3 (Lemma 2 recurrence).
  acamp(...)          Algorithm 2 (Lemma 3 with the five running sums).
  acamp_centred(...)  Algorithm 2's sweep on the centred covariance.
  pair_dist(...)      direct distance of given pairs (Sec. 2 definitions).
  polish(...)         P[i] = d(i, I[i]) recomputed from the definition.
  window_stats(...)   per-window mean, centred sum of squares, flat flag.

Parity: every function is pinned by ``tests/test_oracle.py`` against brute
force on tiny inputs, a library routine (scipy ``cdist``), hand-worked
examples under ``tests/golden/``, closed forms and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmp_oracle.so")

EUCLID, PNORM, ZNORM = 0, 1, 2
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``mp_oracle.c`` into ``_build/libmp_oracle.so`` (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)  # no OpenMP
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d, i64, i32, ip = ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        vp = ctypes.c_void_p
        lib.orc_brute.argtypes = [vp, i64, i32, i64, ip, d, ip, vp, vp]
        lib.orc_brute_rows.argtypes = [vp, i64, i32, i64, ip, d, ip, vp, i64, vp, vp, vp]
        lib.orc_pair_dist.argtypes = [vp, i64, i32, ip, d, ip, vp, vp, i64, vp]
        lib.orc_aamp.argtypes = [vp, i64, i32, i64, i64, i64, ip, vp, vp]
        lib.orc_pnorm.argtypes = [vp, i64, i32, i64, d, i64, i64, ip, vp, vp]
        lib.orc_acamp.argtypes = [vp, i64, i32, i64, i64, i64, ip, vp, vp]
        lib.orc_acamp_centred.argtypes = [vp, i64, i32, i64, i64, i64, ip, vp, vp]
        lib.orc_polish.argtypes = [vp, i64, i32, ip, d, ip, vp, vp]
        lib.orc_window_stats.argtypes = [vp, i64, i32, vp, vp, vp]
        lib.orc_num_threads.argtypes = []
        lib.orc_set_threads.argtypes = [ip]
        lib.orc_set_threads.restype = None
        _lib = lib
        return lib


def _t(T):
    return np.ascontiguousarray(np.asarray(T, dtype=np.float64))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, name):
    if rc != 0:
        raise ValueError(f"oracle {name} failed with status {rc}")


def _dist_code(dist):
    if isinstance(dist, str):
        return {"euclid": EUCLID, "pnorm": PNORM, "znorm": ZNORM}[dist]
    return int(dist)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def _outputs(N):
    N = max(int(N), 0)
    return np.empty(N, np.float64), np.empty(N, np.int64)


def brute(T, m, excl, dist="euclid", p=2.0, raw=False):
    """Nested-loop matrix profile (P, I) straight from the definitions."""
    T = _t(T)
    P, I = _outputs(T.size - m + 1)
    rc = _load().orc_brute(_ptr(T), T.size, m, excl, _dist_code(dist), float(p),
                           int(raw), _ptr(P), _ptr(I))
    _check(rc, "brute")
    return P, I


def brute_rows(T, m, excl, rows, dist="euclid", p=2.0, raw=False):
    """Brute force for selected rows: (P, I, P2) with P2 the runner-up outside
    the exclusion zone of the winner."""
    T = _t(T)
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    P = np.empty(rows.size, np.float64)
    I = np.empty(rows.size, np.int64)
    P2 = np.empty(rows.size, np.float64)
    rc = _load().orc_brute_rows(_ptr(T), T.size, m, excl, _dist_code(dist), float(p),
                                int(raw), _ptr(rows), rows.size, _ptr(P), _ptr(I), _ptr(P2))
    _check(rc, "brute_rows")
    return P, I, P2


def pair_dist(T, m, ii, jj, dist="euclid", p=2.0, raw=False):
    T = _t(T)
    ii = np.ascontiguousarray(np.asarray(ii, dtype=np.int64))
    jj = np.ascontiguousarray(np.asarray(jj, dtype=np.int64))
    out = np.empty(ii.size, np.float64)
    rc = _load().orc_pair_dist(_ptr(T), T.size, m, _dist_code(dist), float(p), int(raw),
                               _ptr(ii), _ptr(jj), ii.size, _ptr(out))
    _check(rc, "pair_dist")
    return out


_KMAX = np.iinfo(np.int64).max


def aamp(T, m, excl, raw=False, k_range=(0, _KMAX)):
    """Algorithm 1: diagonal sweep with the Lemma 1 update."""
    T = _t(T)
    P, I = _outputs(T.size - m + 1)
    rc = _load().orc_aamp(_ptr(T), T.size, m, excl, int(k_range[0]), int(k_range[1]),
                          int(raw), _ptr(P), _ptr(I))
    _check(rc, "aamp")
    return P, I


def pnorm(T, m, excl, p, raw=False, k_range=(0, _KMAX)):
    """Algorithm 3: diagonal sweep with the Lemma 2 update, in FP64 and, as
    the algorithm states it, without re-anchoring: where the terms |x - y|^p
    span many orders of magnitude, a small later sum keeps an absolute error
    of about 1e-16 times the largest sum met on its diagonal (9.4e-6 relative
    on one row of the sine-and-motif series at p = 3, next to its flat run);
    brute_rows, from the definition, is the reference where that matters."""
    T = _t(T)
    P, I = _outputs(T.size - m + 1)
    rc = _load().orc_pnorm(_ptr(T), T.size, m, excl, float(p), int(k_range[0]),
                           int(k_range[1]), int(raw), _ptr(P), _ptr(I))
    _check(rc, "pnorm")
    return P, I


def acamp(T, m, excl, raw=False, k_range=(0, _KMAX)):
    """Algorithm 2: z-normalised sweep on the five running sums of Lemma 3."""
    T = _t(T)
    P, I = _outputs(T.size - m + 1)
    rc = _load().orc_acamp(_ptr(T), T.size, m, excl, int(k_range[0]), int(k_range[1]),
                           int(raw), _ptr(P), _ptr(I))
    _check(rc, "acamp")
    return P, I


def acamp_centred(T, m, excl, raw=False, k_range=(0, _KMAX)):
    """Algorithm 2's sweep carried on the centred covariance."""
    T = _t(T)
    P, I = _outputs(T.size - m + 1)
    rc = _load().orc_acamp_centred(_ptr(T), T.size, m, excl, int(k_range[0]),
                                   int(k_range[1]), int(raw), _ptr(P), _ptr(I))
    _check(rc, "acamp_centred")
    return P, I


def polish(T, m, I, dist="euclid", p=2.0, raw=False):
    """P[i] = d(i, I[i]) from the definition; +inf where I[i] = -1."""
    T = _t(T)
    I = np.ascontiguousarray(np.asarray(I, dtype=np.int64))
    P = np.empty(I.size, np.float64)
    rc = _load().orc_polish(_ptr(T), T.size, m, _dist_code(dist), float(p), int(raw),
                            _ptr(I), _ptr(P))
    _check(rc, "polish")
    return P


def window_stats(T, m):
    """(mu, S, flat): window mean, centred sum of squares, flat flag."""
    T = _t(T)
    N = T.size - m + 1
    mu = np.empty(N, np.float64)
    S = np.empty(N, np.float64)
    flat = np.empty(N, np.uint8)
    rc = _load().orc_window_stats(_ptr(T), T.size, m, _ptr(mu), _ptr(S), _ptr(flat))
    _check(rc, "window_stats")
    return mu, S, flat.astype(bool)


def profile(T, m, excl, dist="euclid", p=2.0, method="incremental", raw=False):
    """Convenience dispatcher used by the tests and the CPU baseline."""
    dist = _dist_code(dist)
    if method == "brute":
        return brute(T, m, excl, dist, p, raw)
    if dist == EUCLID:
        return aamp(T, m, excl, raw)
    if dist == PNORM:
        return pnorm(T, m, excl, p, raw)
    return acamp_centred(T, m, excl, raw)
