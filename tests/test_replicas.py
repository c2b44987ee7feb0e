"""Two-rank (gloo, CPU) tests of the replica bookkeeping used by bench.py for
N > 1: the job time is the slowest rank's, the rate counts every rank's
units, and a single process needs no process group."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1406_6573_gb300 import replicas


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = 1.0 + 0.5 * rank              # rank 1 is the slow one
        units = 100.0 * (rank + 1)
        res = (replicas.world_size(), replicas.max_over_ranks(seconds),
               replicas.sum_over_ranks(units), replicas.job_rate(units, seconds))
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_two_rank_job_rate_uses_max_time_and_summed_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        world, tmax, usum, rate = got[r]
        assert world == 2
        assert tmax == 1.5
        assert usum == 300.0
        assert rate == pytest.approx(300.0 / 1.5)


def test_single_process_needs_no_group():
    assert not (dist.is_available() and dist.is_initialized())
    assert replicas.world_size() == 1
    assert replicas.max_over_ranks(2.5) == 2.5
    assert replicas.job_rate(10.0, 4.0) == 2.5
