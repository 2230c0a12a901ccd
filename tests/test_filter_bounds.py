"""CPU pins of the arithmetic the block filters rely on (float32 emulated in numpy).

The filters may skip a block only if no candidate of it could pass, so the
bounds they test must hold in the kernels' own FP32 arithmetic, not just in
exact arithmetic:

* two-stream sweep (Lemma 1 carried as E += e^2, F' += f^2, s = E - F'): both
  sums only grow and FP32 rounding is monotone, so fl(E(g) - F'(g + G)) is at
  most every score fl(E(u) - F'(u)) of rows g < u <= g + G, and the tagged
  score (low 3 mantissa bits replaced by the slot) keeps it above the bound
  with its tag bits cleared;
* z-normalised sweep: the row form 1 + inv_i * min_d((ch + cl) * inv_j) differs
  from the tracked pass's q = fma(cl, w, fma(ch, w, 1)), w = inv_i * inv_j, by
  far less than the margin max(2e-5, |q| 2^-18) the filter subtracts, plus the
  7 units in the last place a tag can move q; so does the folded form
  1 + inv_i * min_d(fl(ch + cl) * inv_j) of every 4th row.
"""
import numpy as np

f32 = np.float32


def fma32(a, b, c):
    """float32 fma: the float64 product of two float32 values is exact, so one
    rounding of (a b + c) to float32 (through float64) matches the hardware up to
    a rare double rounding, which is still monotone."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def sub32(a, b):
    return (a.astype(np.float64) - b.astype(np.float64)).astype(f32)


def tag(s, d):
    bits = s.view(np.int32)
    return ((bits & ~7) | d).view(f32)


def clear_tag(s):
    return (s.view(np.int32) & ~7).view(f32)


def test_group_bound_is_below_every_score_of_the_group():
    rng = np.random.default_rng(0)
    for trial in range(20):
        n, m = 4000, int(rng.choice([32, 64, 256]))
        t = np.cumsum(rng.standard_normal(n)).astype(f32) * f32(rng.uniform(0.1, 10))
        k = int(rng.integers(m // 4 + 1, n // 2))
        rows = n - m - k
        i0 = int(rng.integers(1, rows // 2))
        # the anchor: the exact window sum at row i0 rounded to float32 (the kernel's ring sum)
        w = (t[i0:i0 + m].astype(np.float64) - t[i0 + k:i0 + k + m]) ** 2
        E = np.zeros(1, f32)
        F = np.array([-w.sum()], f32)
        Es, Fs, S = [E.copy()], [F.copy()], [sub32(E, F)]
        for u in range(1, 257):
            i = i0 + u
            e = sub32(t[i + m - 1:i + m], t[i + k + m - 1:i + k + m])
            f = sub32(t[i - 1:i], t[i + k - 1:i + k])
            E = fma32(e, e, E)
            F = fma32(f, f, F)
            Es.append(E.copy())
            Fs.append(F.copy())
            S.append(sub32(E, F))
        Es, Fs, S = np.concatenate(Es), np.concatenate(Fs), np.concatenate(S)
        assert np.all(np.diff(Es) >= 0) and np.all(np.diff(Fs) >= 0)  # both sums only grow
        for G in (2, 4, 8):
            for g in range(0, 256 - G + 1, G):
                lb = sub32(Es[g:g + 1], Fs[g + G:g + G + 1])[0]
                grp = S[g + 1:g + G + 1]
                assert np.all(lb <= grp), (trial, G, g)
                for d in range(8):  # what the tracked pass compares: the tagged score
                    tagged = tag(grp.copy(), d)
                    assert np.all(clear_tag(np.array([lb], f32))[0] <= tagged)


def test_znorm_row_form_is_within_the_filter_margin():
    rng = np.random.default_rng(1)
    worst = 0.0
    for trial in range(200):
        nd = 8
        # a covariance near the windows' spread, split into a float-float pair as the kernel carries it
        S_i = rng.uniform(0.5, 50.0) * 512
        S_j = rng.uniform(0.5, 50.0, nd) * 512
        rho = rng.uniform(-1.0, 1.0, nd) ** rng.choice([1, 3])
        cov = -rho * np.sqrt(S_i * S_j)  # the words hold -cov
        ch = cov.astype(f32)
        cl = (cov - ch.astype(np.float64)).astype(f32) + f32(rng.normal(0, 1e-3)) * np.abs(ch) * f32(1e-4)
        inv_i = np.array([1.0 / np.sqrt(S_i)], f32)
        inv_j = (1.0 / np.sqrt(S_j)).astype(f32)
        wv = (inv_i.astype(np.float64) * inv_j).astype(f32)
        q_t = fma32(cl, wv, fma32(ch, wv, np.ones(nd, f32)))           # tracked pass
        v = fma32(cl, inv_j, (ch.astype(np.float64) * inv_j).astype(f32))  # filter: (ch + cl) inv_j
        q_f = fma32(np.array([v.min()], f32), inv_i, np.ones(1, f32))[0]  # 1 + inv_i min_d
        qmin = q_t.min()
        margin = max(2e-5, abs(float(q_f)) * 2.0 ** -18)
        ulp = np.spacing(np.abs(qmin).astype(f32))
        diff = abs(float(q_f) - float(qmin)) + 7 * float(ulp)
        worst = max(worst, diff / margin)
        assert float(q_f) - margin <= float(clear_tag(np.array([qmin], f32))[0]), trial
    assert worst < 0.5, worst  # the margin is at least twice what rounding and tags need


def test_znorm_folded_row_form_is_within_the_filter_margin():
    """On every 4th row the z-normalised filter pass folds the float-float
    state first (Fast2Sum: h = fl(ch + cl), l = cl - (h - ch)) and bounds the
    row from the high word alone, 1 + inv_i min_d h inv_j, while the tracked
    pass scores the unfolded words.  The difference stays well inside the
    margin the filter subtracts, tags included."""
    rng = np.random.default_rng(3)
    worst = 0.0
    for trial in range(400):
        nd = 8
        S_i = rng.uniform(0.5, 50.0) * 512
        S_j = rng.uniform(0.5, 50.0, nd) * 512
        rho = rng.uniform(-1.0, 1.0, nd) ** rng.choice([1, 3, 9])
        cov = -rho * np.sqrt(S_i * S_j)
        ch = cov.astype(f32)
        # the low word before a fold: the rounding of ch plus a few rows of increments
        cl = (cov - ch.astype(np.float64)).astype(f32) + f32(rng.normal(0, 1.0)) * np.abs(ch) * f32(rng.choice([1e-4, 1e-2]))
        inv_i = np.array([1.0 / np.sqrt(S_i)], f32)
        inv_j = (1.0 / np.sqrt(S_j)).astype(f32)
        wv = (inv_i.astype(np.float64) * inv_j).astype(f32)
        q_t = fma32(cl, wv, fma32(ch, wv, np.ones(nd, f32)))      # tracked pass, unfolded words
        h = (ch.astype(np.float64) + cl).astype(f32)                # Fast2Sum's high word
        v = (h.astype(np.float64) * inv_j).astype(f32)
        q_f = fma32(np.array([v.min()], f32), inv_i, np.ones(1, f32))[0]
        qmin = q_t.min()
        margin = max(2e-5, abs(float(q_f)) * 2.0 ** -18)
        ulp = np.spacing(np.abs(qmin).astype(f32))
        worst = max(worst, (abs(float(q_f) - float(qmin)) + 7 * float(ulp)) / margin)
        assert float(q_f) - margin <= float(clear_tag(np.array([qmin], f32))[0]), trial
    assert worst < 0.5, worst


def test_znorm_partner_scale_bound_is_conservative():
    """The z-normalised filter's cheaper bound (MP_VARIANT_FAST_FILTER_BOUND):
    with c = fl(ch + cl) and the block's largest partner scale inv_max,
    fl(fma(min(0, min_d c) inv_max, inv_i, 1)) minus the filter's margin is at
    most every tagged q of the row (q = fma(cl, w, fma(ch, w, 1)), w = inv_i
    inv_j, inv_j <= inv_max), whatever the partners' spread."""
    rng = np.random.default_rng(2)
    for trial in range(400):
        nd = 8
        S_i = rng.uniform(0.5, 50.0) * 512
        S_j = rng.uniform(0.5, 50.0) * 512 * rng.uniform(0.9, 1.1, nd) ** rng.choice([1, 5])
        rho = rng.uniform(-1.0, 1.0, nd) ** rng.choice([1, 3, 9])
        cov = -rho * np.sqrt(S_i * S_j)
        ch = cov.astype(f32)
        cl = (cov - ch.astype(np.float64)).astype(f32) + f32(rng.normal(0, 1e-3)) * np.abs(ch) * f32(1e-4)
        inv_i = np.array([1.0 / np.sqrt(S_i)], f32)
        inv_j = (1.0 / np.sqrt(S_j)).astype(f32)
        wv = (inv_i.astype(np.float64) * inv_j).astype(f32)
        q_t = fma32(cl, wv, fma32(ch, wv, np.ones(nd, f32)))
        c = (ch.astype(np.float64) + cl).astype(f32)
        rmin = np.array([min(0.0, float(c.min()))], f32)
        imax = np.array([inv_j.max()], f32)
        prod = (rmin.astype(np.float64) * imax).astype(f32)
        b = fma32(prod, inv_i, np.ones(1, f32))[0]
        margin = max(2e-5, abs(float(b)) * 2.0 ** -18)
        assert float(b) - margin <= float(clear_tag(np.array([q_t.min()], f32))[0]), trial
