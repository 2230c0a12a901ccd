"""Host logic of bench.py's error field (cpu_baseline.fp32_error_on_sample),
on the CPU: a stand-in for the library returns the oracle's own partial
profile with planted errors, and the field must report exactly those."""
import numpy as np

import bench
import oracle
from paper_1901_05708_gb300 import workloads as W


class _Cuda:
    @staticmethod
    def synchronize():
        pass


class _Torch:
    cuda = _Cuda


class _FakeLib:
    """Returns the oracle's partial profile of the requested diagonal range;
    the raw value of row `row` is scaled by (1 + raw_rel) and, polished, the
    index of row `row` moves to another valid candidate."""

    def __init__(self, row, raw_rel):
        self.row, self.raw_rel = row, raw_rel
        self.calls = []

    def profile(self, T, m, excl, dist, p, k_range=None, polish=True):
        self.calls.append((k_range, polish))
        P, I = oracle.aamp(np.asarray(T, np.float64), m, excl, k_range=k_range)
        if polish:
            I[self.row] = I[self.row] + 1 if I[self.row] + 1 - self.row > excl else I[self.row] - 1
        else:
            P[self.row] *= 1 + self.raw_rel
        import torch
        return torch.from_numpy(P), torch.from_numpy(I)

    def sync_status(self):
        pass


def test_slice_error_reports_planted_errors():
    s = W.aamp_small()
    cb = bench.oracle_sample(s, target_s=0.2)
    k0, k1 = cb["k_range"]
    assert k0 == s.excl + 1 and k1 > k0 and cb["ref"][0].shape == (s.N,)
    lib = _FakeLib(row=1234, raw_rel=3e-5)
    out = bench.slice_error(_Torch, lib, s, s.T, "euclid", cb)
    assert lib.calls == [((k0, k1), False), ((k0, k1), True)]
    Pr = cb["ref"][0]
    assert out["diagonals"] == [k0, k1] and out["rows"] == int(np.sum(np.isfinite(Pr) & (Pr > 0)))
    assert abs(out["raw_max_rel_err"] - 3e-5) < 1e-12
    assert out["raw_max_rel_err_at_P"] == Pr[1234]
    atol = 1e-5 * s.m ** 0.5 * np.std(np.diff(s.T.astype(np.float64)))
    expect = 3e-5 * Pr[1234] / (1e-5 * Pr[1234] + atol)
    assert abs(out["raw_max_over_bound"] - expect) < 1e-9 * expect
    assert out["polished_max_rel_err"] == 0.0 and out["polished_max_over_bound"] == 0.0
    assert out["index_mismatch"] == 1
