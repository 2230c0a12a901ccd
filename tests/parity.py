"""Parity checks of a GPU matrix profile against the FP64 oracle.

Acceptance (for FP32 sweeps rtol = 1e-5, for FP64 sweeps rtol = 1e-12):
  (i)   |P - P_ref| <= rtol * P_ref + atol, with the absolute floor
        atol = rtol * m^(1/p) * sd(diff(T)) (pure / p-norm) or rtol * sqrt(m)
        (z-norm) that only matters near zero (flat runs, planted copies);
  (ii)  P[i] equals d(i, I[i]) recomputed by the oracle;
  (iii) I[i] == I_ref[i] wherever the oracle's runner-up (outside the
        winner's exclusion zone, and inside it but not the winner itself) is
        more than the tolerance above the best; elsewhere I[i] must still be a
        valid neighbour within tolerance.

These are the contract's rules, for the polished profile (the default) and
for raw sweep values alike.  One property of the FP32 sweeps is stated
separately and applies only to their raw sweep values (``raw_fp32=True``):
they carry the score (P^p for the pure / p-norm distances, q = 1 - rho =
DZ^2 / 2m for the z-normalised one), whose FP32 rounding is absolute in that
space, so near P = 0 (flat runs, identical windows) the raw value's error is
set by the score's resolution, not by P:
  - pure / p-norm: the score is resolved to S_ATOL = rtol m sd(diff T)^p (the
    floor of rule (i), taken in score space), so the raw P may be off by up to
    (P^p + S_ATOL)^(1/p) - P;
  - z-normalised: q is resolved to an absolute Q_ATOL_Z32 (the FP32 rounding
    of the window scale factors and of their product), so the raw DZ may be
    off by up to sqrt(P^2 + 2m Q_ATOL_Z32) - P.
These terms widen rule (i) (and (ii)) of a raw FP32 check only.
"""
from __future__ import annotations

import numpy as np

import oracle

Q_ATOL_Z32 = 2e-7


def atol_for(T, m, dist, p, rtol):
    T = np.asarray(T, np.float64)
    if dist == "znorm":
        return rtol * np.sqrt(m)
    sd = np.std(np.diff(T)) if T.size > 1 else 0.0
    return rtol * m ** (1.0 / p) * max(sd, 1e-300)


def check(T, m, excl, dist, p, P, I, rtol, rows=None, P_ref=None, I_ref=None, P2=None,
          label="", raw_fp32=False):
    """Compare (P, I) (numpy, full length N) with the oracle on `rows`
    (all rows if None).  Reference values may be passed in; otherwise brute
    force rows are computed here.  Returns a dict of error statistics."""
    T = np.asarray(T, np.float64)
    N = T.size - m + 1
    P = np.asarray(P, np.float64)
    I = np.asarray(I, np.int64)
    assert P.shape == (N,) and I.shape == (N,), (P.shape, I.shape, N)
    rows = np.arange(N) if rows is None else np.asarray(rows, np.int64)
    if P_ref is None:
        P_ref, I_ref, P2 = oracle.brute_rows(T, m, excl, rows, dist, p)
    atol = atol_for(T, m, dist, p, rtol)
    Pg, Ig = P[rows], I[rows]
    Pfin = np.where(np.isfinite(P_ref), P_ref, 0.0)
    tol = rtol * Pfin + atol
    tol_p = tol
    if raw_fp32 and dist == "znorm":
        # the raw FP32 z-normalised value (rules (i), (ii) only; see the module docstring)
        tol_p = tol + np.sqrt(Pfin ** 2 + 2 * m * Q_ATOL_Z32) - Pfin
    elif raw_fp32:
        # the raw FP32 pure / p-norm value: the score's absolute resolution
        pp = 2.0 if dist == "euclid" else p
        sd = np.std(np.diff(T)) if T.size > 1 else 0.0
        s_atol = rtol * m * max(sd, 1e-300) ** pp
        tol_p = tol + (Pfin ** pp + s_atol) ** (1.0 / pp) - Pfin

    none = I_ref < 0
    assert np.all(Ig[none] == -1), f"{label}: rows without candidates got an index"
    assert np.all(np.isinf(Pg[none])), f"{label}: rows without candidates got a finite P"
    has = ~none
    assert np.all(Ig[has] >= 0), f"{label}: {np.sum(Ig[has] < 0)} rows lost their neighbour"
    # (i)
    err = np.abs(Pg[has] - P_ref[has])
    bad = err > tol_p[has]
    assert not np.any(bad), (f"{label}: P off in {bad.sum()} rows; worst rel "
                             f"{np.max(err / np.maximum(P_ref[has], 1e-300)):.3e} at row "
                             f"{rows[has][np.argmax(err - tol_p[has])]}")
    # neighbours must respect the exclusion zone
    assert np.all(np.abs(Ig[has] - rows[has]) > excl), f"{label}: neighbour inside the exclusion zone"
    # (ii)
    d = oracle.pair_dist(T, m, rows[has], Ig[has], dist, p)
    assert np.all(np.abs(d - Pg[has]) <= tol_p[has]), f"{label}: P[i] != d(i, I[i])"
    # (iii)
    unique = (P2[has] - P_ref[has]) > tol[has]
    mism = unique & (Ig[has] != I_ref[has])
    if np.any(mism):
        # P2 skips the winner's own zone; a candidate inside it (a shift of the
        # same match) can still tie with the winner within tolerance, and then
        # the index is not unique either
        hr, hI, hP, ht = rows[has], I_ref[has], P_ref[has], tol[has]
        for x in np.nonzero(mism)[0]:
            i, w = int(hr[x]), int(hI[x])
            js = np.arange(max(0, w - excl), min(N, w + excl + 1))
            js = js[(js != w) & (np.abs(js - i) > excl)]
            if js.size and np.min(oracle.pair_dist(T, m, np.full(js.size, i), js, dist, p)) - hP[x] <= ht[x]:
                unique[x] = False
        mism = unique & (Ig[has] != I_ref[has])
    assert not np.any(mism), (f"{label}: I differs in {mism.sum()} rows with a unique winner, e.g. row "
                              f"{rows[has][np.argmax(mism)]}: got {Ig[has][np.argmax(mism)]}, "
                              f"want {I_ref[has][np.argmax(mism)]}")
    assert np.all(d <= P_ref[has] + tol[has]), f"{label}: a non-unique winner is not within tolerance"
    rel = err / np.maximum(P_ref[has], atol)
    return {"rows": int(rows.size), "max_rel_err": float(rel.max()) if rel.size else 0.0,
            "i_mismatch": int(np.sum(Ig[has] != I_ref[has])), "unique": int(unique.sum())}
