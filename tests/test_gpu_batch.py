"""Batches (mp_batch_*): many independent profiles in one graph launch.

Every series of a batch must get exactly what the single-series entry point
gives for it (same tiles, same kernels, same polish), and both must pass the
parity checks against the FP64 oracle.  The mixed batch touches all four
tile queues: the two-stream Euclidean sweep (m a multiple of 32), the
generic sweep for other m, the generic p-norm sweep, and the z-normalised
sweep, plus series without any candidate pair and a flat run."""
import numpy as np
import pytest

import oracle
from paper_1901_05708_gb300 import workloads as W

import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL32 = 1e-5
NAMES = {W.EUCLID: "euclid", W.PNORM: "pnorm", W.ZNORM: "znorm"}


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_05708_gb300 import mp as lib
    lib.load()
    return lib


def mixed_batch(seed, p):
    rng = np.random.default_rng(seed)
    out = []
    specs = [("walk", 3000, 32, W.EUCLID), ("walk", 2500, 40, W.EUCLID), ("int", 1800, 64, W.EUCLID),
             ("walk", 2200, 7, W.PNORM), ("motif", 4000, 96, W.PNORM), ("walk", 3500, 64, W.ZNORM),
             ("flat", 3000, 32, W.ZNORM), ("walk", 900, 5, W.ZNORM), ("walk", 40, 16, W.EUCLID),
             ("walk", 60, 30, W.ZNORM), ("uniform", 5000, 128, W.EUCLID), ("walk", 1, 1, W.EUCLID),
             ("motif", 2600, 50, W.EUCLID)]
    for k, (kind, n, m, dist) in enumerate(specs):
        s = W.small(kind, n, m, int(rng.integers(1 << 30)), dist=dist, p=p, dtype=np.float32)
        out.append(s)
    # no candidate pair at all: N - 1 <= excl
    out.append(W.small("walk", 70, 40, 7, excl=40, dtype=np.float32))
    return out


def run_batch(mp, series, p, **kw):
    lengths = [s.n for s in series]
    plan = mp.BatchPlan(lengths, [s.m for s in series], [s.dist for s in series], [s.excl for s in series], p=p,
                        **kw)
    T = torch.from_numpy(np.concatenate([s.T for s in series]).astype(np.float32)).cuda()
    P, I = plan.run(T)
    torch.cuda.synchronize()
    mp.sync_status()
    return plan, T, P.cpu().numpy(), I.cpu().numpy()


def single(mp, s, p, **kw):
    T = torch.from_numpy(np.ascontiguousarray(s.T, dtype=np.float32)).cuda()
    P, I = mp.profile(T, s.m, s.excl, NAMES[s.dist], p, **kw)
    torch.cuda.synchronize()
    return P.cpu().numpy(), I.cpu().numpy()


def single_as_batched(mp, s, p):
    """The single call with the kernel the batch runs: the default one, except
    for p = 3, where single calls default to the tall-tile kernel (error-free
    sums) and batches run the re-anchored two-stream or generic kernel."""
    if s.dist != W.PNORM or p != 3.0:
        return single(mp, s, p)
    try:
        return single(mp, s, p, variant=mp.MP_VARIANT_FAST)
    except mp.MPError:
        return single(mp, s, p, variant=mp.MP_VARIANT_GENERIC)


@pytest.mark.parametrize("p", [1.0, 3.0, 2.5])
def test_mixed_batch_matches_single_calls_and_oracle(mp, p):
    series = mixed_batch(100 + int(p * 10), p)
    plan, T, P, I = run_batch(mp, series, p)
    o = plan.out_offsets
    assert plan.windows == o[-1] == P.size
    for k, s in enumerate(series):
        Pk, Ik = P[o[k]:o[k + 1]], I[o[k]:o[k + 1]]
        Ps, Is = single_as_batched(mp, s, p)
        np.testing.assert_array_equal(Ik, Is, err_msg=f"series {k} ({s.name}) I differs from the single call")
        np.testing.assert_array_equal(Pk, Ps, err_msg=f"series {k} ({s.name}) P differs from the single call")
        dist = NAMES[s.dist]
        parity.check(s.T.astype(np.float64), s.m, s.excl, dist, p, Pk, Ik, RTOL32, label=f"batch {k} {s.name}")
    plan.close()


def test_replay_and_rebuild(mp):
    series = mixed_batch(7, 1.0)
    plan, T, P0, I0 = run_batch(mp, series, 1.0)
    P1, I1 = plan.run(T)  # new output buffers: the graph is recorded again
    P2, I2 = plan.run(T, out=(P1, I1))  # the previous run's pointers: the graph is replayed
    torch.cuda.synchronize()
    for P, I in ((P1, I1), (P2, I2)):
        np.testing.assert_array_equal(P.cpu().numpy(), P0)
        np.testing.assert_array_equal(I.cpu().numpy(), I0)
    plan.close()


def test_filter_variant_gives_the_same_profile(mp):
    """MP_VARIANT_FAST_FILTER only skips candidates that cannot pass: bit-identical results."""
    series = mixed_batch(13, 1.0)
    lengths, ms = [s.n for s in series], [s.m for s in series]
    dists, excls = [s.dist for s in series], [s.excl for s in series]
    T = torch.from_numpy(np.concatenate([s.T for s in series]).astype(np.float32)).cuda()
    a = mp.BatchPlan(lengths, ms, dists, excls, p=1.0)
    b = mp.BatchPlan(lengths, ms, dists, excls, p=1.0, variant=mp.MP_VARIANT_FAST_FILTER)
    Pa, Ia = a.run(T)
    Pb, Ib = b.run(T)
    torch.cuda.synchronize()
    assert torch.equal(Pa, Pb) and torch.equal(Ia, Ib)
    with pytest.raises(mp.MPError):
        mp.BatchPlan(lengths, ms, dists, excls, p=1.0, variant=mp.MP_VARIANT_GENERIC)
    a.close()
    b.close()


def test_polish_off_keeps_sweep_values(mp):
    """polish = 0: same neighbours, P is the sweep's own FP32 value (for the
    z-normalised series q = 1 - rho carries an absolute FP32 error)."""
    series = mixed_batch(9, 3.0)[:6]
    _, _, P, I = run_batch(mp, series, 3.0, polish=False)
    plan, _, Pp, Ip = run_batch(mp, series, 3.0)
    np.testing.assert_array_equal(I, Ip)
    o = plan.out_offsets
    for k, s in enumerate(series):
        a, b = P[o[k]:o[k + 1]], Pp[o[k]:o[k + 1]]
        fin = np.isfinite(b)
        np.testing.assert_array_equal(np.isfinite(a), fin)
        if s.dist == W.ZNORM:
            tol = 2e-5 * b[fin] + np.sqrt(b[fin] ** 2 + 2 * s.m * parity.Q_ATOL_Z32) - b[fin]
            assert np.all(np.abs(a[fin] - b[fin]) <= tol), k
        else:
            # compare the sums the sweep carries (P^p): FP32 rounding of the running
            # sum is absolute, on the scale of the series' largest sums
            p_ = 3.0 if s.dist == W.PNORM else 2.0
            sa, sb = a[fin] ** p_, b[fin] ** p_
            assert np.all(np.abs(sa - sb) <= 2e-5 * sb + 1e-5 * sb.max()), k
    plan.close()


def test_batch_4096_sampled(mp):
    """The 4,096-series workload (lengths 2,000..65,536, m in {32, 64, 128},
    half Euclidean, half z-normalised): 256 series chosen by seed with 16
    sampled rows each, plus 3 sampled rows (and the first and last) of every
    series, by brute force; and the whole-profile properties on every
    series."""
    b = W.batch_4096()
    series = b.series
    plan, T, P, I = run_batch(mp, series, 2.0)
    o = plan.out_offsets
    rng = np.random.default_rng(21)
    pick = set(rng.choice(len(series), 256, replace=False).tolist())
    for k, s in enumerate(series):
        Pk, Ik = P[o[k]:o[k + 1]], I[o[k]:o[k + 1]]
        count = 16 if k in pick else 3
        rows = np.unique(np.concatenate([rng.choice(s.N, count, replace=False), [0, s.N - 1]]))
        ref = oracle.brute_rows(s.T.astype(np.float64), s.m, s.excl, rows, NAMES[s.dist])
        parity.check(s.T.astype(np.float64), s.m, s.excl, NAMES[s.dist], 2.0, Pk, Ik, RTOL32, rows=rows,
                     P_ref=ref[0], I_ref=ref[1], P2=ref[2], label=f"batch4096 series {k}")
    # every row of every series has a valid neighbour outside its zone
    for k, s in enumerate(series):
        Ik = I[o[k]:o[k + 1]]
        x = np.arange(s.N)
        assert np.all(Ik >= 0) and np.all(Ik < s.N) and np.all(np.abs(Ik - x) > s.excl), k
    plan.close()
