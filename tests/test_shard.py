"""Sharding of the uneven batch over ranks: LPT partition properties, and world-size-2
gloo runs in which each rank takes its share and only the step time is reduced (no
data-path collective); in the second, each rank factorises and solves its share of
small Gaussian-kernel systems (the oracle stands in for the GPU on the CPU runner)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2509_11152_b300.shard import lpt_partition


def test_lpt_is_a_partition_within_the_greedy_bound():
    from h2gen import uneven_sizes
    n = uneven_sizes()
    for r in (1, 2, 3, 4, 8):
        parts = lpt_partition(n, r)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(n)))
        loads = [sum(n[i] for i in p) for p in parts]
        # LPT: the heaviest rank exceeds the lightest by at most the largest job
        assert max(loads) - min(loads) <= max(n)
        assert max(loads) <= sum(n) / r + max(n)


def test_lpt_small_cases():
    assert lpt_partition([5, 4, 3, 3, 3], 2) == [[0, 3], [1, 2, 4]]
    assert lpt_partition([1.0], 3) == [[0], [], []]
    with pytest.raises(ValueError):
        lpt_partition([1], 0)


def test_memory_bins_fit_and_cover():
    from h2gen import uneven_sizes
    from paper_2509_11152_b300.shard import memory_bins
    n = uneven_sizes(64, 2048, 131072)
    for cap in (max(n), 2.5 * max(n), sum(n) / 3, sum(n)):
        bins = memory_bins(n, cap)
        flat = sorted(i for b in bins for i in b)
        assert flat == list(range(len(n)))
        assert all(sum(n[i] for i in b) <= cap for b in bins)
        # first fit decreasing never needs more than 11/9 OPT + 1 bins; OPT >= sum / cap
        assert len(bins) <= 11 / 9 * (sum(n) / cap) + 2
    assert memory_bins(n, sum(n)) == [list(range(len(n)))]
    assert memory_bins([5, 4, 3, 3, 3], 9) == [[0, 1], [2, 3, 4]]
    assert memory_bins([], 1.0) == []
    with pytest.raises(ValueError):
        memory_bins([1, 10], 5)
    with pytest.raises(ValueError):
        memory_bins([1], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, sizes, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    mine = lpt_partition(sizes, ws)[rank]
    work = float(sum(sizes[i] for i in mine))         # stands in for this rank's step time
    t = torch.tensor([work], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, mine, float(t.item())))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_disjoint_shares():
    sizes = [2083, 109154, 5460, 44788, 17210, 7404, 64899, 3410]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = [o[1] for o in out]
    assert sorted(shares[0] + shares[1]) == list(range(len(sizes)))
    loads = [sum(sizes[i] for i in s) for s in shares]
    assert out[0][2] == out[1][2] == max(loads)


def _solve_worker(rank, ws, port, sizes, q):
    import time

    import numpy as np

    from conftest import problem
    from h2gen import rhs
    from oracle import dense, rs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    mine = lpt_partition(sizes, ws)[rank]
    t0 = time.perf_counter()
    errs = []
    for s in mine:
        pb = problem("gauss3d", n=sizes[s], leaf=32, seed=s)
        A = pb.A.numpy()
        b = rhs(A.n, 2, seed=s)
        x = rs.solve(rs.factorize(A, 1e-10, pb.norm_a), b)
        xd = np.linalg.solve(dense.expand(A), b)
        errs.append(float(np.linalg.norm(x - xd) / np.linalg.norm(xd)))
    mine_t = time.perf_counter() - t0
    t = torch.tensor([mine_t], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, mine, mine_t, float(t.item()), errs))
    dist.destroy_process_group()


def test_two_gloo_ranks_solve_their_shares():
    sizes = [700, 300, 900, 500, 400, 600]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_solve_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = [o[1] for o in out]
    assert sorted(shares[0] + shares[1]) == list(range(len(sizes)))
    assert all(len(o[4]) == len(o[1]) and max(o[4], default=0.0) <= 1e-6 for o in out), out
    assert out[0][3] == out[1][3] == max(out[0][2], out[1][2])
