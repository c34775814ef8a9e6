"""The N > 1 path of bench.py on CPU: replicas on two gloo ranks, whose per-format times
are combined by an element-wise max over ranks (the slowest replica decides)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = {"f64": 10.0 + rank, "f32": 6.0 - rank, "f16": 5.0 + 0.5 * rank}
    out = bench.max_over_ranks(mine, "cpu")
    q.put((rank, out))
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert res[r] == {"f16": 5.5, "f32": 6.0, "f64": 11.0}


def _batch_rank_main(rank, world, port, q):
    """One rank of the batch split: its contiguous share of the systems (shard_units),
    solved here by the oracle standing in for the GPU solver, its solve time maxed over
    the ranks, its solutions gathered on every rank."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import time

    import numpy as np

    import bench
    import oracle as O
    import workloads as W
    O.set_threads(1)
    mats = W.stencil_batch(nsys=7, nmin=100, nmax=600, config_id=4)
    mine = bench.shard_units(len(mats), world, rank)
    t0 = time.perf_counter()
    sols = {}
    for i in mine:
        A = mats[i]
        b = W.rhs_from_solution(A, W.exact_solution(A.n, 4, salt=i))
        r = O.gmres(A, b, m=30, fmt=O.F32, precond=O.PC_JACOBI, tol=1e-8, maxit=100000)
        sols[i] = (r["iters"], r["x"].tolist())
    dt = time.perf_counter() - t0
    tmax = bench.max_over_ranks({"batch": dt}, "cpu")["batch"]
    gathered = [None] * world
    dist.all_gather_object(gathered, {"rank": rank, "units": list(mine), "sols": sols, "t": dt})
    q.put((rank, tmax, gathered))
    dist.destroy_process_group()


def test_batch_split_over_two_gloo_ranks():
    """The batch workload under torchrun: every rank solves its share of the systems with
    no data-path collective; the shares cover every system exactly once, each system's
    solution equals the one-process solve, and the batch time is the slowest rank's."""
    import numpy as np

    import bench
    import oracle as O
    import workloads as W
    for n, world in ((7, 2), (512, 3), (5, 8)):
        shares = [bench.shard_units(n, world, r) for r in range(world)]
        assert sorted(i for s in shares for i in s) == list(range(n))
        assert max(len(s) for s in shares) - min(len(s) for s in shares) <= 1
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    gathered = res[0][2]
    assert all(abs(r[1] - max(g["t"] for g in gathered)) < 1e-12 for r in res)
    units = sorted(i for g in gathered for i in g["units"])
    assert units == list(range(7))
    mats = W.stencil_batch(nsys=7, nmin=100, nmax=600, config_id=4)
    for g in gathered:
        for i, (iters, x) in g["sols"].items():
            A = mats[i]
            b = W.rhs_from_solution(A, W.exact_solution(A.n, 4, salt=i))
            r = O.gmres(A, b, m=30, fmt=O.F32, precond=O.PC_JACOBI, tol=1e-8, maxit=100000)
            assert iters == r["iters"] and np.array_equal(np.array(x), r["x"])
