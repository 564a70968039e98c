"""The replicas-only multi-GPU logic of bench.py on CPU ranks (gloo).

Each rank runs its own independent replica of the workload; the only
collective is the max of the ranks' times after the timed region, and the
whole-job rate counts the units of every rank over the slowest rank's time.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = [12.5, 20.0][rank]                       # the ranks' own times
    slowest = bench.max_over_ranks(ms, dist, "cpu")
    rate = bench.whole_job_rate(10, world, slowest / 1000.0)
    out.put((rank, slowest, rate))
    dist.destroy_process_group()


def test_max_over_ranks_and_rate_with_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate in got:
        assert slowest == 20.0                   # every rank sees the slowest time
        assert rate == pytest.approx(10 * 2 / 0.020)


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(20, 1, 0.5) == 40.0
