"""Pins for the FP64 CPU oracle (no GPU).

Each test ties the oracle to something other than itself: a library routine
(scipy's cdist), hand-worked examples (tests/golden), exact integer
arithmetic, closed forms, invariants stated or implied by the paper, and
brute force on tiny inputs.  A plausible mistake (dropped term, wrong sign,
wrong index, swapped operand, wrong tie-break) fails at least one of them.
"""
import ast
import glob
import json
import math
import operator
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

from paper_1901_05708_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def windows(T, m):
    T = np.asarray(T, np.float64)
    N = T.size - m + 1
    return np.lib.stride_tricks.sliding_window_view(T, m)[:N]


def library_matrix(T, m, dist, p=2.0):
    """All-pairs score matrix from scipy (independent of the oracle)."""
    X = windows(T, m)
    if dist == "euclid":
        return cdist(X, X, "sqeuclidean")
    if dist == "pnorm":
        return cdist(X, X, "minkowski", p=p) ** p
    mu = X.mean(axis=1, keepdims=True)
    sd = X.std(axis=1, keepdims=True)  # population sigma (ddof = 0)
    Z = (X - mu) / sd
    return cdist(Z, Z, "sqeuclidean")


def profile_from_matrix(D, excl):
    """Min over |i - j| > excl with the paper's arrival-order tie-break,
    written as a sort on (score, |i - j|, right-side flag)."""
    N = D.shape[0]
    P = np.full(N, np.inf)
    I = np.full(N, -1, np.int64)
    for x in range(N):
        best = None
        for j in range(N):
            k = abs(j - x)
            if k <= excl or not np.isfinite(D[x, j]):
                continue
            key = (D[x, j], k, 1 if j > x else 0)
            if best is None or key < best[0]:
                best = (key, j)
        if best is not None:
            P[x] = best[0][0]
            I[x] = best[1]
    return P, I


_OPS = {ast.Add: operator.add, ast.Sub: operator.sub, ast.Mult: operator.mul,
        ast.Div: operator.truediv, ast.Pow: operator.pow, ast.USub: operator.neg}


def closed_form(expr):
    """Evaluate a golden closed form ('6-3*sqrt(3)', 'inf', '9')."""
    if expr == "inf":
        return math.inf

    def ev(node):
        if isinstance(node, ast.Expression):
            return ev(node.body)
        if isinstance(node, ast.Constant):
            return float(node.value)
        if isinstance(node, ast.BinOp):
            return _OPS[type(node.op)](ev(node.left), ev(node.right))
        if isinstance(node, ast.UnaryOp):
            return _OPS[type(node.op)](ev(node.operand))
        if isinstance(node, ast.Call) and node.func.id == "sqrt":
            return math.sqrt(ev(node.args[0]))
        raise ValueError(expr)
    return ev(ast.parse(expr, mode="eval"))


def finish(score, dist, p):
    score = np.asarray(score, np.float64)
    with np.errstate(invalid="ignore"):
        if dist == "pnorm":
            return score ** (1.0 / p)
        return np.sqrt(score)


ALL_METHODS = {
    "euclid": lambda o, T, m, e, p, raw: o.aamp(T, m, e, raw=raw),
    "pnorm": lambda o, T, m, e, p, raw: o.pnorm(T, m, e, p, raw=raw),
    "znorm": lambda o, T, m, e, p, raw: o.acamp(T, m, e, raw=raw),
    "znorm_c": lambda o, T, m, e, p, raw: o.acamp_centred(T, m, e, raw=raw),
}


# ---------------------------------------------------------------- golden
@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.json"))))
def test_golden_examples(oracle_mod, path):
    g = json.load(open(path))
    T, m, dist = g["T"], g["m"], g["dist"]
    for case in g["cases"]:
        p = case.get("p", g.get("p", 2.0))
        excl = case["excl"]
        want = np.array([closed_form(s) for s in case["score"]])
        wantI = np.array(case["I"])
        for method in ("brute", "incremental"):
            P, I = oracle_mod.profile(T, m, excl, dist, p, method=method, raw=True)
            np.testing.assert_allclose(P, want, rtol=1e-12, atol=1e-12, err_msg=f"{path} {method}")
            np.testing.assert_array_equal(I, wantI, err_msg=f"{path} {method}")
            Pf, If = oracle_mod.profile(T, m, excl, dist, p, method=method, raw=False)
            # the final root maps a raw error e near 0 to about e^(1/p)
            np.testing.assert_allclose(Pf, finish(want, dist, p), rtol=1e-12, atol=1e-6)
            np.testing.assert_array_equal(If, wantI)
        if dist == "znorm":
            P, I = oracle_mod.acamp_centred(T, m, excl, raw=True)
            np.testing.assert_allclose(P, want, rtol=1e-12, atol=1e-12)
            np.testing.assert_array_equal(I, wantI)
    for i, j in g.get("euclid_zero_pairs", []):
        d = oracle_mod.pair_dist(T, m, [i], [j], "euclid")
        assert d[0] == 0.0


# ------------------------------------------------------- library routine
@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("m", [1, 2, 3, 5, 8])
def test_brute_matches_scipy(oracle_mod, seed, m):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(m + 2, 48))
    T = np.cumsum(rng.standard_normal(n))
    for excl in sorted({0, 1, max(1, m // 4)}):
        for dist, p in (("euclid", 2.0), ("pnorm", 1.0), ("pnorm", 3.0), ("pnorm", 2.5), ("znorm", 2.0)):
            if dist == "znorm" and m < 2:
                continue
            D = library_matrix(T, m, dist, p)
            Pl, Il = profile_from_matrix(D, excl)
            P, I = oracle_mod.brute(T, m, excl, dist, p, raw=True)
            np.testing.assert_allclose(P, Pl, rtol=1e-10, atol=1e-10, err_msg=f"{dist} p={p} excl={excl}")
            np.testing.assert_array_equal(I, Il, err_msg=f"{dist} p={p} excl={excl}")


def test_pair_dist_matches_scipy(oracle_mod):
    rng = np.random.default_rng(7)
    T = np.cumsum(rng.standard_normal(300)) * 3.0 + 10.0
    m = 17
    X = windows(T, m)
    ii = rng.integers(0, X.shape[0], 200)
    jj = rng.integers(0, X.shape[0], 200)
    for dist, p in (("euclid", 2.0), ("pnorm", 1.0), ("pnorm", 3.0), ("znorm", 2.0)):
        D = library_matrix(T, m, dist, p)
        got = oracle_mod.pair_dist(T, m, ii, jj, dist, p, raw=True)
        np.testing.assert_allclose(got, D[ii, jj], rtol=1e-9, atol=1e-9)


# ------------------------------------------------ incremental vs brute
@pytest.mark.parametrize("seed", range(8))
def test_incremental_matches_brute(oracle_mod, seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(20, 90))
    m = int(rng.integers(2, 12))
    T = np.cumsum(rng.standard_normal(n))
    for excl in (0, 1, m // 4 + 1):
        for name, dist, p in (("euclid", "euclid", 2.0), ("pnorm", "pnorm", 1.0),
                              ("pnorm", "pnorm", 3.0), ("znorm", "znorm", 2.0),
                              ("znorm_c", "znorm", 2.0)):
            Pb, Ib = oracle_mod.brute(T, m, excl, dist, p, raw=True)
            Pi, Ii = ALL_METHODS[name](oracle_mod, T, m, excl, p, True)
            np.testing.assert_allclose(Pi, Pb, rtol=1e-8, atol=1e-9, err_msg=name)
            np.testing.assert_array_equal(Ii, Ib, err_msg=name)


@pytest.mark.parametrize("seed", range(20))
def test_integer_series_exact(oracle_mod, seed):
    """Integer data: every FP64 intermediate of the Euclidean and p = 1, 3
    sweeps is an exact integer, so the recurrence equals the definition bit
    for bit, and the frequent ties pin the tie-break."""
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(8, 120))
    m = int(rng.integers(1, min(64, n) + 1))
    T = rng.integers(-8, 9, n).astype(np.float64)
    for excl in (0, 1, max(0, m // 4)):
        Pb, Ib = oracle_mod.brute(T, m, excl, "euclid", raw=True)
        Pa, Ia = oracle_mod.aamp(T, m, excl, raw=True)
        np.testing.assert_array_equal(Pa, Pb)
        np.testing.assert_array_equal(Ia, Ib)
        D = library_matrix(T, m, "euclid") if n <= 80 else None
        if D is not None:
            Pl, Il = profile_from_matrix(np.rint(D), excl)
            np.testing.assert_array_equal(Pb, Pl)
            np.testing.assert_array_equal(Ib, Il)
        for p in (1.0, 3.0):
            Pb, Ib = oracle_mod.brute(T, m, excl, "pnorm", p, raw=True)
            Pp, Ip = oracle_mod.pnorm(T, m, excl, p, raw=True)
            np.testing.assert_array_equal(Pp, Pb)
            np.testing.assert_array_equal(Ip, Ib)


# ------------------------------------------------------------ invariants
def test_p2_is_euclid(oracle_mod):
    T = W.small("walk", 200, 16, 1).T
    a = oracle_mod.aamp(T, 16, 4, raw=True)
    b = oracle_mod.pnorm(T, 16, 4, 2.0, raw=True)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_symmetry(oracle_mod):
    rng = np.random.default_rng(11)
    T = np.cumsum(rng.standard_normal(150))
    ii = rng.integers(0, 140, 100)
    jj = rng.integers(0, 140, 100)
    for dist, p in (("euclid", 2.0), ("pnorm", 1.5), ("znorm", 2.0)):
        a = oracle_mod.pair_dist(T, 11, ii, jj, dist, p)
        b = oracle_mod.pair_dist(T, 11, jj, ii, dist, p)
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=0)


def test_shift_scale_affine(oracle_mod):
    T = W.small("walk", 300, 20, 5).T
    P, I = oracle_mod.aamp(T, 20, 5)
    P2, I2 = oracle_mod.aamp(T + 1000.0, 20, 5)       # shift invariance
    np.testing.assert_allclose(P2, P, rtol=1e-7)
    np.testing.assert_array_equal(I2, I)
    P3, I3 = oracle_mod.aamp(-2.5 * T, 20, 5)         # D(aT) = |a| D(T)
    np.testing.assert_allclose(P3, 2.5 * P, rtol=1e-10)
    np.testing.assert_array_equal(I3, I)
    Pp, Ip = oracle_mod.pnorm(T, 20, 5, 3.0)
    Pp3, Ip3 = oracle_mod.pnorm(4.0 * T, 20, 5, 3.0)
    np.testing.assert_allclose(Pp3, 4.0 * Pp, rtol=1e-10)
    np.testing.assert_array_equal(Ip3, Ip)
    Z, IZ = oracle_mod.acamp_centred(T, 20, 5)
    Z2, IZ2 = oracle_mod.acamp_centred(3.0 * T - 7.0, 20, 5)  # affine invariance
    np.testing.assert_allclose(Z2, Z, rtol=1e-8, atol=1e-9)
    np.testing.assert_array_equal(IZ2, IZ)


def test_znorm_range_and_extremes(oracle_mod):
    rng = np.random.default_rng(3)
    T = rng.standard_normal(200)
    m = 9
    P, I = oracle_mod.brute(T, m, 2, "znorm")
    assert np.all(P >= 0) and np.all(P <= 2 * math.sqrt(m) + 1e-12)
    # identical shape (rho = 1) -> 0; mirrored shape (rho = -1) -> 2 sqrt(m)
    base = rng.standard_normal(m)
    T2 = np.concatenate([base, rng.standard_normal(5), 3 * base + 1, rng.standard_normal(5), -base])
    j1, j2 = m + 5, 2 * m + 10
    d = oracle_mod.pair_dist(T2, m, [0, 0], [j1, j2], "znorm")
    np.testing.assert_allclose(d, [0.0, 2 * math.sqrt(m)], atol=1e-7)


def test_flat_segments(oracle_mod):
    s = W.small("flat", 400, 16, 9)
    mu, S, flat = oracle_mod.window_stats(s.T, 16)
    assert flat.sum() > 0
    P, I = oracle_mod.acamp_centred(s.T, 16, 4)
    assert np.all(np.isinf(P[flat])) and np.all(I[flat] == -1)
    assert not np.any(flat[I[I >= 0]])               # a flat window is no one's neighbour
    Pr, Ir = oracle_mod.acamp(s.T, 16, 4)
    Pb, Ib = oracle_mod.brute(s.T, 16, 4, "znorm")
    np.testing.assert_allclose(P, Pb, rtol=1e-7, atol=1e-9)
    np.testing.assert_array_equal(I, Ib)
    np.testing.assert_array_equal(Ir, Ib)
    # pure Euclidean: windows inside the constant run are at distance 0
    Pe, Ie = oracle_mod.aamp(s.T, 16, 4)
    inside = np.where(flat)[0]
    pairs = [(a, b) for a in inside for b in inside if b - a > 4]
    assert pairs and np.all(Pe[[a for a, _ in pairs]] == 0.0)


def test_lemma_identities(oracle_mod):
    """Lemma 1 (Euclidean), Lemma 2 (p-norm) and Lemma 3 (z-norm from the
    five sums) checked against the direct definitions."""
    rng = np.random.default_rng(21)
    T = np.cumsum(rng.standard_normal(120))
    m = 13
    for i, j in ((5, 40), (1, 90), (30, 31)):
        for dist, p in (("euclid", 2.0), ("pnorm", 3.0), ("pnorm", 1.0)):
            cur = oracle_mod.pair_dist(T, m, [i], [j], dist, p, raw=True)[0]
            prev = oracle_mod.pair_dist(T, m, [i - 1], [j - 1], dist, p, raw=True)[0]
            upd = prev - abs(T[i - 1] - T[j - 1]) ** p + abs(T[i + m - 1] - T[j + m - 1]) ** p
            assert cur == pytest.approx(upd, rel=1e-10)
        x, y = T[i:i + m], T[j:j + m]
        A, B, AA, BB, C = x.sum(), y.sum(), (x * x).sum(), (y * y).sum(), (x * y).sum()
        rho = (C - A * B / m) / math.sqrt((AA - A * A / m) * (BB - B * B / m))
        dz = oracle_mod.pair_dist(T, m, [i], [j], "znorm", raw=True)[0]
        assert dz == pytest.approx(2 * m * (1 - rho), rel=1e-9)
        # Sec. 4.3: F orders pairs like DZ, and 2m + 2 sign(F) sqrt|F| is DZ^2
        F = (A * B - m * C) * abs(A * B - m * C) / ((AA - A * A / m) * (BB - B * B / m))
        assert 2 * m + 2 * math.copysign(math.sqrt(abs(F)), F) == pytest.approx(dz, rel=1e-9)


def test_f_ordering(oracle_mod):
    rng = np.random.default_rng(22)
    T = np.cumsum(rng.standard_normal(200))
    m = 10
    X = windows(T, m)
    ii = rng.integers(0, X.shape[0], 300)
    jj = rng.integers(0, X.shape[0], 300)
    A, B = X[ii].sum(1), X[jj].sum(1)
    AA, BB, C = (X[ii] ** 2).sum(1), (X[jj] ** 2).sum(1), (X[ii] * X[jj]).sum(1)
    F = (A * B - m * C) * np.abs(A * B - m * C) / ((AA - A * A / m) * (BB - B * B / m))
    dz = oracle_mod.pair_dist(T, m, ii, jj, "znorm", raw=True)
    keep = np.abs(dz - 2 * m) > 1e-6
    assert np.array_equal(np.argsort(F[keep], kind="stable"), np.argsort(dz[keep], kind="stable"))


def test_centred_covariance_update(oracle_mod):
    """The centred-covariance form used by Algorithm 2's sweep tracks the raw
    five-sum form and the definition on a random walk with a large offset."""
    T = W.small("walk", 2000, 64, 13).T + 5000.0
    Pb, Ib = oracle_mod.brute_rows(T, 64, 16, np.arange(0, 1937, 37), "znorm")[:2]
    Pc, Ic = oracle_mod.acamp_centred(T, 64, 16)
    np.testing.assert_allclose(Pc[::37], Pb, rtol=1e-9)
    np.testing.assert_array_equal(Ic[::37], Ib)


# --------------------------------------------------------- edge cases
def test_no_valid_pair(oracle_mod):
    T = np.arange(10.0)
    for fn in ("brute", "incremental"):
        P, I = oracle_mod.profile(T, 4, 6, "euclid", method=fn)   # N - 1 = 6 <= excl
        assert np.all(np.isinf(P)) and np.all(I == -1)
        P, I = oracle_mod.profile(T, 10, 0, "euclid", method=fn)  # m = n: one window
        assert P.shape == (1,) and np.isinf(P[0]) and I[0] == -1


def test_m_equals_one(oracle_mod):
    T = np.array([3.0, 1.0, 4.0, 1.0, 5.0, 9.0, 2.0, 6.0])
    P, I = oracle_mod.aamp(T, 1, 0)
    np.testing.assert_array_equal(I[[1, 3]], [3, 1])
    np.testing.assert_array_equal(P[[1, 3]], [0.0, 0.0])
    Pb, Ib = oracle_mod.brute(T, 1, 0, "euclid")
    np.testing.assert_array_equal(P, Pb)
    np.testing.assert_array_equal(I, Ib)


def test_invalid_args(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.brute(np.zeros(5), 6, 0)
    with pytest.raises(ValueError):
        oracle_mod.pnorm(np.zeros(10), 3, 0, 0.5)


# ---------------------------------------- rows, polish, ranges, threads
def test_rows_polish_and_runner_up(oracle_mod):
    s = W.small("motif", 600, 24, 4)
    P, I = oracle_mod.brute(s.T, 24, 6, "euclid")
    rows = np.array([0, 7, 100, 333, 576])
    Pr, Ir, P2 = oracle_mod.brute_rows(s.T, 24, 6, rows, "euclid")
    np.testing.assert_array_equal(Pr, P[rows])
    np.testing.assert_array_equal(Ir, I[rows])
    assert np.all(P2 >= Pr)
    np.testing.assert_allclose(oracle_mod.polish(s.T, 24, I, "euclid"), P, rtol=1e-13)
    Pz, Iz = oracle_mod.acamp_centred(s.T, 24, 6)
    np.testing.assert_allclose(oracle_mod.polish(s.T, 24, Iz, "znorm"), Pz, rtol=1e-8)


def runner_up_from_matrix(D, excl, I):
    """Second-best score of each row from an all-pairs matrix: the minimum over
    candidates j of row x (|j - x| > excl) that also lie outside the winner's
    exclusion zone (|j - I[x]| > excl); +inf if there is none."""
    N = D.shape[0]
    P2 = np.full(N, np.inf)
    j = np.arange(N)
    for x in range(N):
        if I[x] < 0:
            continue
        ok = (np.abs(j - x) > excl) & (np.abs(j - I[x]) > excl) & np.isfinite(D[x])
        if ok.any():
            P2[x] = D[x, ok].min()
    return P2


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("dist,p", [("euclid", 2.0), ("pnorm", 1.0), ("pnorm", 3.0), ("znorm", 2.0)])
def test_runner_up_matches_scipy(oracle_mod, seed, dist, p):
    """orc_brute_rows' runner-up P2 (which decides where the GPU's index must
    equal the oracle's) against the same quantity taken from scipy's all-pairs
    matrix: every row of tiny series, excl in {0, 1, m/4}.  Cases where the
    winner's zone straddles the row's own zone occur on every series (the
    winner sits just outside the row's zone); a planted copy next to the row's
    zone forces one for excl = m/4."""
    rng = np.random.default_rng(900 + seed)
    m = int(rng.integers(4, 10))
    n = int(rng.integers(3 * m, 60))
    T = np.cumsum(rng.standard_normal(n))
    # a near-copy of window 5 placed so that its start is just outside the zone
    # of row 5 for excl = m // 4, whose own zone then overlaps row 5's
    c = 5 + m // 4 + 1
    if c + m <= n and 5 + m <= n:
        T[c:c + m] = T[5:5 + m] + 0.02 * rng.standard_normal(m)
    D = library_matrix(T, m, dist, p)
    N = n - m + 1
    rows = np.arange(N)
    for excl in sorted({0, 1, max(1, m // 4)}):
        Pl, Il = profile_from_matrix(D, excl)
        P2l = runner_up_from_matrix(D, excl, Il)
        Pr, Ir, P2r = oracle_mod.brute_rows(T, m, excl, rows, dist, p, raw=True)
        np.testing.assert_array_equal(Ir, Il)
        np.testing.assert_allclose(Pr, Pl, rtol=1e-12, atol=1e-12)
        fin = np.isfinite(P2l)
        assert np.array_equal(np.isfinite(P2r), fin), f"excl={excl}: runner-up exists in a different set of rows"
        np.testing.assert_allclose(P2r[fin], P2l[fin], rtol=1e-12, atol=1e-12,
                                   err_msg=f"{dist} p={p} excl={excl}")
        # the distance form (the final root) of the same runner-up
        _, _, P2d = oracle_mod.brute_rows(T, m, excl, rows, dist, p, raw=False)
        np.testing.assert_allclose(P2d[fin], finish(P2l[fin], dist, p), rtol=1e-11, atol=1e-7)
        # straddling zones: some winner lies within 2 excl of its row, so the
        # zones around the row and around the winner overlap
        if excl == max(1, m // 4):
            assert np.any((Il >= 0) & (np.abs(Il - rows) <= 2 * excl)), "no straddling case exercised"


def test_diagonal_ranges_merge(oracle_mod):
    """Disjoint diagonal ranges merged by (score, 2k + side) give the full
    profile: the rule the multi-rank merge relies on."""
    T = W.small("int", 300, 7, 8).T
    full = oracle_mod.aamp(T, 7, 2, raw=True)
    N = 300 - 7 + 1
    parts = [oracle_mod.aamp(T, 7, 2, raw=True, k_range=r) for r in ((0, 40), (40, 41), (41, N))]
    best = np.full(N, np.inf)
    bkey = np.full(N, np.iinfo(np.int64).max)
    x = np.arange(N)
    for P, I in parts:
        key = np.where(I >= 0, 2 * np.abs(I - x) + (I > x), np.iinfo(np.int64).max)
        take = (P < best) | ((P == best) & (key < bkey))
        best = np.where(take, P, best)
        bkey = np.where(take, key, bkey)
    Irec = np.where(bkey == np.iinfo(np.int64).max, -1,
                    np.where(bkey & 1, x + (bkey >> 1), x - (bkey >> 1)))
    np.testing.assert_array_equal(best, full[0])
    np.testing.assert_array_equal(Irec, full[1])


def test_thread_count_does_not_change_result(oracle_mod):
    T = W.small("int", 400, 9, 12).T
    nt = oracle_mod.num_threads()
    try:
        oracle_mod.set_threads(1)
        a = oracle_mod.aamp(T, 9, 2, raw=True)
        oracle_mod.set_threads(max(2, nt))
        b = oracle_mod.aamp(T, 9, 2, raw=True)
    finally:
        oracle_mod.set_threads(nt)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_small_workload_brute_vs_incremental(oracle_mod):
    """The 10,000-point random walk (m = 100, excl = 25): Algorithm 1 against
    the nested loop on every row."""
    s = W.aamp_small()
    Pb, Ib = oracle_mod.brute(s.T, s.m, s.excl, "euclid")
    Pa, Ia = oracle_mod.aamp(s.T, s.m, s.excl)
    np.testing.assert_allclose(Pa, Pb, rtol=1e-9)
    np.testing.assert_array_equal(Ia, Ib)
    assert s.cells == 48_762_750


def test_cell_counts():
    assert W.cells(1 << 20, 256, 64) == 549_420_844_896
    assert W.cells(1 << 18, 128, 32) == 34_317_939_120
    assert W.cells(1 << 20, 512, 128) == 549_085_454_016
    assert W.cells(8, 3, 0) == 15            # Fig. 2: 5 + 4 + 3 + 2 + 1
    assert W.cells(10, 4, 6) == 0
