"""Replicated multi-rank runs on CPU (gloo, world size 2): the job time is the
slowest rank's and the throughput counts every rank's work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1210_2536_gb300.dist import max_over_ranks, weak_scaling_throughput


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 20.25][rank]          # the second rank is slower
    m = max_over_ranks(ms)
    out[rank] = (m, weak_scaling_throughput(1e9, m / 1e3, world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1]
    m, v = out[0]
    assert m == 20.25
    assert abs(v - 2 * 1e9 / 0.02025) < 1e-3


def test_single_process_is_identity():
    assert max_over_ranks(3.5) == 3.5
    assert weak_scaling_throughput(10.0, 2.0, 1) == 5.0
