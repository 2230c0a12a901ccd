"""CPU pin of the p = 3 window-sum arithmetic, in emulated float32 (numpy
float32 scalars round every operation as the kernels' lanes do).

Along one diagonal of a sine with noise 0.1 and a planted random-walk motif,
the window sum of |x - y|^3 climbs to about 10^5 while the motif passes and
falls back to about 0.3 a few rows after it has left.  The re-anchored FP32
form (E += |e| e^2, F' += |f| f^2, s = E - F', F' restarted at minus the
window sum every m/4 rows, as the two-stream kernel carries Lemma 2's update
for p = 3) keeps an error of the size of the large terms until its next
anchor; the error-free form (the leaving term off the high word by Fast2Sum,
the entering one on by Fast2Sum after ordering the two nonnegative operands,
their rounding errors into the low word, a Fast2Sum fold every second row, as
the tall-tile kernel does for p = 3) stays at float-float precision of the
exact sum of the window's FP32 terms."""
import math

import numpy as np

f32 = np.float32


def fma32(a, b, c):
    """float32 fma: the float64 product of two float32 values is exact."""
    return f32(float(a) * float(b) + float(c))


def term(x):
    """|x|^3 as the tall kernel computes it: fl(|x| fl(x x))."""
    return f32(abs(x) * f32(x * x))


def series(seed=5, n=6000, m=128):
    rng = np.random.default_rng(seed)
    t = np.arange(n)
    x = np.sin(2 * np.pi * t / 1000.0) + rng.normal(0.0, 0.1, n)
    x[2000:2000 + m] = np.cumsum(rng.standard_normal(m)) * 3.0 + rng.normal(0.0, 0.1, m)
    return x.astype(f32)


def exact_window_sums(x, m, k, rows, term_fn):
    """fsum of the window's float32 terms (float32 differences) for each row."""
    out = []
    for i in rows:
        out.append(math.fsum(float(term_fn(f32(x[i + l] - x[i + k + l]))) for l in range(m)))
    return np.array(out)


def test_error_free_p3_sums_track_the_exact_sum():
    m, k = 128, 1000
    x = series(m=m)
    rows = range(1700, 2500)  # the motif enters row windows at 1873 and leaves them after 2127
    ref = exact_window_sums(x, m, k, rows, term)
    assert ref.max() > 1e4 and ref[-1] < 5.0  # the dynamic range this pins

    # error-free float-float carry (tall-tile kernel, p = 3)
    i0 = rows.start
    ch, cl = f32(0), f32(0)
    for l in range(m):  # the anchor: TwoSum of every term from the definition
        p = term(f32(x[i0 + l] - x[i0 + k + l]))
        t = f32(ch + p)
        bb = f32(t - ch)
        cl = f32(cl + f32(f32(ch - f32(t - bb)) + f32(p - bb)))
        ch = t
    worst = 0.0
    for u, i in enumerate(rows):
        if u > 0:
            xe = term(f32(x[i + m - 1] - x[i + k + m - 1]))
            xf = term(f32(x[i - 1] - x[i + k - 1]))
            s1 = f32(ch - xf)
            e1 = f32(f32(ch - s1) - xf)
            hi, lo = max(s1, xe), min(s1, xe)
            s2 = f32(hi + lo)
            e2 = f32(lo - f32(s2 - hi))
            ch = s2
            cl = f32(cl + f32(e1 + e2))
            if u % 2 == 0:  # fold (Fast2Sum)
                t = f32(ch + cl)
                cl = f32(cl - f32(t - ch))
                ch = t
        got = float(ch) + float(cl)
        worst = max(worst, abs(got - ref[u]) / ref[u])
    # float-float precision: the low word's own rounding, of order eps^2 times the largest sums met
    assert worst < 1e-7, worst


def test_reanchored_fp32_sums_lose_small_distances():
    m, k = 128, 1000
    B = m // 4
    x = series(m=m)
    rows = range(1700, 2500)
    ref = exact_window_sums(x, m, k, rows, lambda v: abs(float(v)) ** 3)
    worst = 0.0
    for u, i in enumerate(rows):
        if u % B == 0:  # re-anchor: F' = -(window sum), E = 0 (the window sum itself rounded to float32)
            E, F = f32(0), f32(-ref[u])
        else:
            e = f32(x[i + m - 1] - x[i + k + m - 1])
            f = f32(x[i - 1] - x[i + k - 1])
            E = fma32(abs(e), f32(e * e), E)
            F = fma32(abs(f), f32(f * f), F)
        s = float(f32(E - F))
        worst = max(worst, abs(s - ref[u]) / ref[u])
    assert worst > 1e-3, worst  # far outside the FP32 tolerance on P^3 (3e-5)


def _error_free_walk(x, m, k, rows):
    i0 = rows.start
    ch, cl = f32(0), f32(0)
    for l in range(m):
        p = term(f32(x[i0 + l] - x[i0 + k + l]))
        t = f32(ch + p)
        bb = f32(t - ch)
        cl = f32(cl + f32(f32(ch - f32(t - bb)) + f32(p - bb)))
        ch = t
    sums = []
    for u, i in enumerate(rows):
        if u > 0:
            xe = term(f32(x[i + m - 1] - x[i + k + m - 1]))
            xf = term(f32(x[i - 1] - x[i + k - 1]))
            s1 = f32(ch - xf)
            e1 = f32(f32(ch - s1) - xf)
            hi, lo = max(s1, xe), min(s1, xe)
            s2 = f32(hi + lo)
            e2 = f32(lo - f32(s2 - hi))
            ch = s2
            cl = f32(cl + f32(e1 + e2))
            if u % 2 == 0:
                t = f32(ch + cl)
                cl = f32(cl - f32(t - ch))
                ch = t
        sums.append(float(ch) + float(cl))
    return np.array(sums)


def test_error_free_p3_sums_single_spike():
    """A window sum made of one large term: while the spike is in the window
    the high word is that term (ch = term(f) when it leaves, the edge of
    Fast2Sum's condition), and after it leaves the sum returns to the small
    terms' exact sum."""
    m, k = 64, 300
    rng = np.random.default_rng(9)
    x = (rng.normal(0.0, 1e-3, 2000)).astype(f32)
    x[1000] = f32(40.0)  # |x|^3 = 64,000 against terms of about 1e-9
    rows = range(900, 1200)
    ref = exact_window_sums(x, m, k, rows, term)
    got = _error_free_walk(x, m, k, rows)
    assert ref.max() > 6e4 and ref[-1] < 1e-6
    rel = np.abs(got - ref) / ref
    assert rel.max() < 1e-6, rel.max()
