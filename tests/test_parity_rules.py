"""The acceptance rules of tests/parity.py, exercised on the CPU with oracle
profiles standing in for a GPU result: a planted wrong neighbour or a P off
by more than the tolerance must fail; a neighbour that ties with the
oracle's winner within the tolerance (here a shift of the same match, which
the runner-up outside the winner's zone does not see) must pass."""
import numpy as np
import pytest

import oracle
from paper_1901_05708_gb300 import workloads as W

import parity


@pytest.fixture(scope="module")
def case():
    s = W.small("walk", 1500, 24, 5)
    T = s.T
    P, I = oracle.brute(T, s.m, s.excl, "euclid")
    return s, T, P, I


def test_exact_profile_passes(case):
    s, T, P, I = case
    st = parity.check(T, s.m, s.excl, "euclid", 2.0, P, I, 1e-5, label="exact")
    assert st["i_mismatch"] == 0 and st["rows"] == s.N


def test_wrong_neighbour_fails(case):
    s, T, P, I = case
    Ig, Pg = I.copy(), P.copy()
    i = 700
    j = (I[i] + 300) % s.N  # a far, worse candidate
    if abs(j - i) <= s.excl:
        j = (j + 2 * s.excl + 1) % s.N
    Ig[i] = j
    Pg[i] = oracle.pair_dist(T, s.m, np.array([i]), np.array([j]), "euclid")[0]
    with pytest.raises(AssertionError):
        parity.check(T, s.m, s.excl, "euclid", 2.0, Pg, Ig, 1e-5, label="planted")


def test_p_off_fails(case):
    s, T, P, I = case
    Pg = P.copy()
    Pg[100] *= 1 + 1e-4
    with pytest.raises(AssertionError):
        parity.check(T, s.m, s.excl, "euclid", 2.0, Pg, I, 1e-5, label="planted")


def test_tie_inside_winner_zone_passes():
    """A p = 1 case met on the GPU: row 3695's best match is 3127, and 3129 (a
    shift of the same match, inside the winner's zone) is 7e-7 relative away;
    an FP32 sweep may return either, so either must pass."""
    s = W.small("motif", 4000, 96, 247714344, dist=W.PNORM, p=1.0)
    T = s.T
    rows = np.arange(3600, 3800)
    P, I, P2 = oracle.brute_rows(T, s.m, s.excl, rows, "pnorm", 1.0)
    k = int(np.nonzero(rows == 3695)[0][0])
    assert I[k] == 3127
    Ig, Pg = I.copy(), P.copy()
    Ig[k] = 3129
    Pg[k] = oracle.pair_dist(T, s.m, np.array([3695]), np.array([3129]), "pnorm", 1.0)[0]
    assert 0 < Pg[k] - P[k] < 1e-5 * P[k]
    Pfull = np.zeros(s.N)
    Ifull = np.zeros(s.N, dtype=np.int64)
    Pfull[rows], Ifull[rows] = Pg, Ig
    parity.check(T, s.m, s.excl, "pnorm", 1.0, Pfull, Ifull, 1e-5, rows=rows, P_ref=P, I_ref=I, P2=P2,
                 label="tie")


def test_znorm_strict_unless_raw_fp32():
    """The z-normalised rules are the contract's (1e-5 relative, rtol sqrt(m)
    floor): a P off by more than that fails, unless the check is explicitly of
    the FP32 kernel's raw sweep value (raw_fp32), whose stated q resolution
    widens rule (i) only."""
    s = W.small("walk", 900, 16, 8)
    T = s.T.copy()
    T[600:616] = T[100:116] + 1e-4 * np.random.default_rng(3).standard_normal(16)  # a near-identical pair
    P, I = oracle.brute(T, s.m, s.excl, "znorm")
    Pg = P.copy()
    x = int(np.argmin(P))
    tol = 1e-5 * P[x] + 1e-5 * np.sqrt(s.m)
    loose = np.sqrt(P[x] ** 2 + 2 * s.m * parity.Q_ATOL_Z32) - P[x]
    assert loose > 2 * tol
    Pg[x] = P[x] + tol + 0.5 * loose
    with pytest.raises(AssertionError):
        parity.check(T, s.m, s.excl, "znorm", 2.0, Pg, I, 1e-5, label="polished")
    parity.check(T, s.m, s.excl, "znorm", 2.0, Pg, I, 1e-5, label="raw", raw_fp32=True)


def test_pnorm_raw_score_resolution():
    """Near P = 0 (a flat run: exact zero distances) a raw FP32 p-norm value
    carries the score's absolute rounding, amplified by the p-th root: a
    residue of 1e-9 in the score is P = 1e-3 for p = 3.  That fails the
    contract's rules and passes only as an explicit raw FP32 check."""
    s = W.small("flat", 2000, 32, 51)
    T = s.T
    P, I = oracle.brute(T, s.m, s.excl, "pnorm", 3.0)
    x = int(np.argmin(P))
    assert P[x] == 0.0
    Pg = P.copy()
    Pg[x] = 1e-9 ** (1 / 3)
    with pytest.raises(AssertionError):
        parity.check(T, s.m, s.excl, "pnorm", 3.0, Pg, I, 1e-5, label="polished")
    parity.check(T, s.m, s.excl, "pnorm", 3.0, Pg, I, 1e-5, label="raw", raw_fp32=True)
    Pg[x] = 0.1  # far beyond the score's resolution: fails either way
    with pytest.raises(AssertionError):
        parity.check(T, s.m, s.excl, "pnorm", 3.0, Pg, I, 1e-5, label="raw", raw_fp32=True)
