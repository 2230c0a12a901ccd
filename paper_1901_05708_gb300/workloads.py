"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws numbers: it holds none of the matrix-profile
arithmetic, and both the CUDA path and the CPU oracle are fed from it.
Everything is drawn with numpy's PCG64 ``default_rng(seed)``.

The paper's own experiments use uniformly random values with default
n = 2^18 and m = 2^8 (Sec. 5.1, "Setup"); it names no public dataset.  The
five workloads below keep that scale family and add the structure that makes
a matrix profile meaningful (random walks, planted motifs, anomalies, a
constant segment, a batch of uneven series):

  aamp_small   float64 random walk, n = 10,000, m = 100, pure Euclidean
  aamp_1m      float32 random walk + 20 Gaussian bumps, n = 2^20, m = 256
  pnorm_262k   float32 sine + noise + 10 planted motifs + flat run, n = 2^18,
               m = 128, p in {1, 3}
  acamp_1m     float32 random walk + N(0, 0.01), n = 2^20, m = 512, z-norm
  batch_4096   4,096 float32 random walks, n ~ U{2000..65536},
               m in {32, 64, 128}, half pure Euclidean, half z-normalised

The exclusion zone is ceil(m / 4) for all of them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

EUCLID, PNORM, ZNORM = 0, 1, 2


def excl_zone(m: int) -> int:
    return int(math.ceil(m / 4))


def cells(n: int, m: int, excl: int) -> int:
    """Number of unordered pairs (i, j) with excl < j - i <= N - 1."""
    N = n - m + 1
    L = N - excl - 1
    return L * (L + 1) // 2 if L > 0 else 0


@dataclass
class Series:
    name: str
    T: np.ndarray          # float32 or float64, 1-D
    m: int
    excl: int
    dist: int = EUCLID
    p: float = 2.0
    info: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.T.size)

    @property
    def N(self) -> int:
        return self.n - self.m + 1

    @property
    def cells(self) -> int:
        return cells(self.n, self.m, self.excl)


@dataclass
class Batch:
    name: str
    series: list           # list[Series]

    @property
    def cells(self) -> int:
        return sum(s.cells for s in self.series)


def random_walk(n: int, seed: int, dtype=np.float32) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.standard_normal(n)).astype(dtype)


def aamp_small(seed: int = 0) -> Series:
    T = np.cumsum(np.random.default_rng(seed).standard_normal(10_000))  # float64
    return Series("aamp_small_n10000_m100", T, 100, excl_zone(100), EUCLID)


def aamp_1m(seed: int = 1, n: int = 1 << 20, m: int = 256, bumps: int = 20) -> Series:
    """Random walk with Gaussian bumps of amplitude 5 and width (sigma) 50."""
    rng = np.random.default_rng(seed)
    walk = np.cumsum(rng.standard_normal(n))
    centres = rng.uniform(m, n - m, size=bumps)
    t = np.arange(n, dtype=np.float64)
    for c in centres:
        lo, hi = int(max(0, c - 400)), int(min(n, c + 400))
        walk[lo:hi] += 5.0 * np.exp(-((t[lo:hi] - c) ** 2) / (2.0 * 50.0 ** 2))
    return Series(f"aamp_n{n}_m{m}", walk.astype(np.float32), m, excl_zone(m), EUCLID,
                  info={"bump_centres": np.sort(centres)})


def pnorm_262k(p: float, seed: int = 2, n: int = 1 << 18, m: int = 128,
               copies: int = 10, flat_len: int = 5000) -> Series:
    """Sine (period 1000) + N(0, 0.1), 10 planted copies of one random-walk
    motif of length m (each with fresh N(0, 0.1)), one constant run."""
    rng = np.random.default_rng(seed)
    t = np.arange(n, dtype=np.float64)
    x = np.sin(2 * np.pi * t / 1000.0) + rng.normal(0.0, 0.1, n)
    motif = np.cumsum(rng.standard_normal(m))
    flat_at = int(rng.integers(m, n - m - flat_len))
    taken = [(flat_at, flat_at + flat_len)]
    starts = []
    while len(starts) < copies:
        s = int(rng.integers(0, n - m))
        if all(s + m <= a or s >= b for a, b in taken):
            taken.append((s, s + m))
            starts.append(s)
    for s in starts:
        x[s:s + m] = motif + rng.normal(0.0, 0.1, m)
    x[flat_at:flat_at + flat_len] = x[flat_at]
    return Series(f"pnorm_p{p:g}_n{n}_m{m}", x.astype(np.float32), m, excl_zone(m), PNORM,
                  p=float(p), info={"motif_starts": sorted(starts), "flat": (flat_at, flat_len)})


def acamp_1m(seed: int = 3, n: int = 1 << 20, m: int = 512) -> Series:
    rng = np.random.default_rng(seed)
    x = np.cumsum(rng.standard_normal(n)) + rng.normal(0.0, 0.01, n)
    return Series(f"acamp_n{n}_m{m}", x.astype(np.float32), m, excl_zone(m), ZNORM)


def batch_4096(seed: int = 4, count: int = 4096, n_lo: int = 2000, n_hi: int = 65536) -> Batch:
    rng = np.random.default_rng(seed)
    lengths = rng.integers(n_lo, n_hi + 1, size=count)
    ms = rng.choice(np.array([32, 64, 128]), size=count)
    dists = np.where(rng.random(count) < 0.5, EUCLID, ZNORM)
    out = []
    for s in range(count):
        T = np.cumsum(rng.standard_normal(int(lengths[s]))).astype(np.float32)
        m = int(ms[s])
        out.append(Series(f"b{s}", T, m, excl_zone(m), int(dists[s])))
    return Batch(f"batch{count}_n{n_lo}-{n_hi}", out)


def uniform(n: int, seed: int, dtype=np.float32) -> np.ndarray:
    """The paper's timing data: i.i.d. uniform values (Sec. 5.1)."""
    return np.random.default_rng(seed).random(n).astype(dtype)


def small(kind: str, n: int, m: int, seed: int, excl: int | None = None,
          dist: int = EUCLID, p: float = 2.0, dtype=np.float64) -> Series:
    """Small seeded series for parity tests.

    kind: 'walk' (random walk), 'uniform', 'int' (integers in [-8, 8], for
    which every FP32/FP64 intermediate of the Euclidean sweep is exact),
    'motif' (walk with two planted copies of a window), 'flat' (walk with a
    constant run of 2m samples).
    """
    rng = np.random.default_rng(seed)
    if kind == "walk":
        x = np.cumsum(rng.standard_normal(n))
    elif kind == "uniform":
        x = rng.random(n)
    elif kind == "int":
        x = rng.integers(-8, 9, size=n).astype(np.float64)
    elif kind == "motif":
        x = np.cumsum(rng.standard_normal(n))
        if n >= 4 * m:
            a = int(rng.integers(0, n // 2 - m))
            b = int(rng.integers(n // 2, n - m))
            x[b:b + m] = x[a:a + m] + 0.01 * rng.standard_normal(m)
    elif kind == "flat":
        x = np.cumsum(rng.standard_normal(n))
        if n >= 4 * m:
            a = int(rng.integers(0, n - 2 * m))
            x[a:a + 2 * m] = x[a]
    else:
        raise ValueError(kind)
    if excl is None:
        excl = excl_zone(m)
    return Series(f"{kind}_n{n}_m{m}_s{seed}", x.astype(dtype), m, excl, dist, p)
