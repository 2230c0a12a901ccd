"""Multi-rank split of one matrix profile over diagonal ranges (CPU, gloo).

Each rank sweeps its own range of diagonals with the oracle and the ranks
merge with two MIN all-reduces; the result must equal the single-rank
profile exactly, ties included (integer data makes ties frequent)."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1901_05708_gb300 import shard
from paper_1901_05708_gb300 import workloads as W


def test_diagonal_ranges_balance():
    for k_first, N, parts in ((65, 1_048_321, 8), (1, 100, 3), (26, 9901, 2), (5, 7, 4)):
        r = shard.diagonal_ranges(k_first, N, parts)
        assert r[0][0] == k_first and r[-1][1] == N
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        cells = [sum(N - k for k in range(lo, hi)) for lo, hi in r]
        total = sum(cells)
        if N - k_first > 10 * parts:
            assert max(cells) - min(cells) <= 2 * N, cells
        assert total == (N - k_first) * (N - k_first + 1) // 2


def test_merge_in_process():
    T = W.small("int", 600, 7, 3).T
    N = 600 - 7 + 1
    full = oracle.aamp(T, 7, 1)
    parts = [oracle.aamp(T, 7, 1, k_range=r) for r in shard.diagonal_ranges(2, N, 3)]
    P, I = shard.merge(parts)
    np.testing.assert_array_equal(P, full[0])
    np.testing.assert_array_equal(I, full[1])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, T, m, excl, out_path, dist_name, p):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        N = T.size - m + 1
        lo, hi = shard.diagonal_ranges(excl + 1, N, world)[rank]
        if dist_name == "euclid":
            P, I = oracle.aamp(T, m, excl, k_range=(lo, hi))
        elif dist_name == "pnorm":
            P, I = oracle.pnorm(T, m, excl, p, k_range=(lo, hi))
        else:
            P, I = oracle.acamp_centred(T, m, excl, k_range=(lo, hi))
        Pm, Im = shard.allreduce_merge(torch.from_numpy(P), torch.from_numpy(I))
        if rank == 0:
            np.savez(out_path, P=Pm.numpy(), I=Im.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("dist_name,p", [("euclid", 2.0), ("pnorm", 1.0), ("znorm", 2.0)])
def test_two_ranks_gloo(tmp_path, dist_name, p):
    import torch.multiprocessing as mp
    T = W.small("int", 900, 8, 11).T if dist_name != "znorm" else W.small("walk", 900, 8, 11).T
    m, excl = 8, 2
    out = str(tmp_path / "merged.npz")
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, T, m, excl, out, dist_name, p))
             for r in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    got = np.load(out)
    if dist_name == "euclid":
        P, I = oracle.aamp(T, m, excl)
    elif dist_name == "pnorm":
        P, I = oracle.pnorm(T, m, excl, p)
    else:
        P, I = oracle.acamp_centred(T, m, excl)
    np.testing.assert_array_equal(got["P"], P)
    np.testing.assert_array_equal(got["I"], I)


def _rank_main_libmp(rank, world, port, T, m, excl, out_path, dist_name, p):
    """One rank: the CUDA library sweeps this rank's diagonal range on the
    GPU; the parts are merged over gloo on host tensors."""
    import torch
    import torch.distributed as dist
    from paper_1901_05708_gb300 import mp
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        N = T.size - m + 1
        lo, hi = shard.diagonal_ranges(excl + 1, N, world)[rank]
        Tt = torch.from_numpy(T).cuda()
        P, I = mp.profile(Tt, m, excl, dist_name, p, k_range=(lo, hi))
        torch.cuda.synchronize()
        mp.sync_status()
        Pm, Im = shard.allreduce_merge(P.cpu(), I.cpu())
        if rank == 0:
            np.savez(out_path, P=Pm.numpy(), I=Im.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
@pytest.mark.parametrize("dist_name,p,kind", [("euclid", 2.0, "int"), ("pnorm", 1.0, "int"),
                                               ("euclid", 2.0, "walk"), ("znorm", 2.0, "walk")])
def test_two_ranks_libmp(tmp_path, dist_name, p, kind):
    """Two processes run the CUDA library on their diagonal ranges (here on
    the one GPU, one after the other or side by side: the sweeps never wait on
    each other) and merge with two MIN all-reduces over gloo.  Integer series:
    the merged profile equals the single call bit for bit; random walks: it
    passes the parity rules against the oracle."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as tmp
    import parity
    from paper_1901_05708_gb300 import mp
    n, m, excl = 20_000, 64, 16
    T = W.small(kind, n, m, 23, dtype=np.float32).T
    out = str(tmp_path / "merged.npz")
    port = _free_port()
    ctx = tmp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main_libmp, args=(r, 2, port, T, m, excl, out, dist_name, p))
             for r in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=300)
        assert pr.exitcode == 0
    got = np.load(out)
    Tt = torch.from_numpy(T).cuda()
    P1, I1 = mp.profile(Tt, m, excl, dist_name, p)
    torch.cuda.synchronize()
    P1, I1 = P1.cpu().numpy(), I1.cpu().numpy()
    if kind == "int":
        np.testing.assert_array_equal(got["P"], P1)
        np.testing.assert_array_equal(got["I"], I1)
    else:
        parity.check(T, m, excl, dist_name, p, got["P"], got["I"], 1e-5, label=f"two ranks {dist_name}")
