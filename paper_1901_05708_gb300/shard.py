"""Splitting one matrix profile over several ranks, and merging the parts.

The diagonal sweep is a union of independent diagonals: the pairs
(i, i + k) for k in [k_first, N).  Disjoint ranges of k can be swept
separately (mp_aamp / mp_pnorm / mp_acamp with ``k_range``) and the partial
profiles merged element-wise with the tie rule of the paper's loops
(smallest distance, then smallest |i - j|, then the left neighbour).

``diagonal_ranges`` cuts [k_first, N) into ranges of nearly equal cell count
(diagonal k holds N - k cells).  ``merge`` combines partial profiles held in
one process; ``allreduce_merge`` does the same across a torch.distributed
group with two MIN all-reduces (distance, then the tie key among the ranks
holding the minimum).
"""
from __future__ import annotations

import math

import numpy as np

_NONE = np.iinfo(np.int64).max


def diagonal_ranges(k_first: int, N: int, parts: int) -> list[tuple[int, int]]:
    """Contiguous ranges [k_lo, k_hi) covering [k_first, N) with about equal
    numbers of cells sum_k (N - k) each."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    k_first = max(int(k_first), 0)
    L = max(N - k_first, 0)          # diagonals k_first .. N-1 hold L, L-1, ..., 1 cells
    total = L * (L + 1) // 2
    bounds = [k_first]
    for r in range(1, parts):
        target = total * r / parts   # cells before the cut
        # cells in [k_first, k_first + x) = x L - x (x - 1) / 2; solve for x
        x = (2 * L + 1 - math.sqrt(max((2 * L + 1) ** 2 - 8 * target, 0.0))) / 2
        bounds.append(min(N, max(bounds[-1], k_first + int(round(x)))))
    bounds.append(max(N, k_first))
    return [(bounds[r], bounds[r + 1]) for r in range(parts)]


def tie_key(I: np.ndarray) -> np.ndarray:
    """2 |i - j| + [j > i] for I[i] = j, or int64 max where there is none."""
    I = np.asarray(I, np.int64)
    x = np.arange(I.size, dtype=np.int64)
    return np.where(I >= 0, 2 * np.abs(I - x) + (I > x), _NONE)


def index_from_key(key: np.ndarray) -> np.ndarray:
    key = np.asarray(key, np.int64)
    x = np.arange(key.size, dtype=np.int64)
    k = key >> 1
    return np.where(key == _NONE, -1, np.where(key & 1, x + k, x - k))


def merge(parts) -> tuple[np.ndarray, np.ndarray]:
    """Merge partial (P, I) profiles (numpy) with the tie rule."""
    best = bkey = None
    for P, I in parts:
        P = np.asarray(P, np.float64)
        key = tie_key(I)
        if best is None:
            best, bkey = P.copy(), key
            continue
        take = (P < best) | ((P == best) & (key < bkey))
        best = np.where(take, P, best)
        bkey = np.where(take, key, bkey)
    return best, index_from_key(bkey)


def allreduce_merge(P, I, group=None):
    """Merge this rank's partial profile with every other rank's (torch
    tensors on a device the process group supports).  Returns (P, I)."""
    import torch
    import torch.distributed as dist

    Pm = P.clone()
    dist.all_reduce(Pm, op=dist.ReduceOp.MIN, group=group)
    x = torch.arange(I.numel(), device=I.device, dtype=torch.int64)
    key = torch.where(I >= 0, 2 * (I - x).abs() + (I > x).to(torch.int64),
                      torch.full_like(I, _NONE))
    key = torch.where(P == Pm, key, torch.full_like(key, _NONE))
    dist.all_reduce(key, op=dist.ReduceOp.MIN, group=group)
    k = key >> 1
    Im = torch.where(key == _NONE, torch.full_like(key, -1), torch.where((key & 1) == 1, x + k, x - k))
    return Pm, Im
