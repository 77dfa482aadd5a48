"""The multi-GPU path of bench.py on CPU: two gloo ranks.  Weak scaling gives
each rank its own problem instance of the same shape (no data-path
collective); the only exchange is the MAX of the timed region over ranks, and
the job rate is every rank's units over the slowest rank's time."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2506_11547_gb300 import synth
    p, g, lev = bench.rank_problem(synth, "small_n1e3_32", rank)
    mine = 1.5 + rank  # this rank's timed seconds
    slowest = bench.reduce_max(mine, dist, "cpu")
    rate = bench.whole_job_rate(p.n * 19544, 4, world, slowest)
    out.put((rank, float(p.a[0, 0]), g, lev, slowest, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    (_, a0, g0, l0, s0, r0), (_, a1, g1, l1, s1, r1) = res
    assert (g0, l0) == (g1, l1) == (32, 0)  # same shape on every rank
    assert a0 != a1  # its own instance per rank
    assert s0 == s1 == 2.5  # the slowest rank's time, everywhere
    assert r0 == r1 == pytest.approx(1000 * 19544 * 4 * 2 / 2.5)
