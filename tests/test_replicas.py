"""Multi-GPU runs are independent replicas (no collective on the data path); the bench's
only cross-rank step, the job time (slowest rank) and the job's work (sum over ranks), is
checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, work = bench.reduce_over_ranks(5.0 + 10.0 * rank, 100.0 + rank, torch.device("cpu"))
    out[rank] = (ms, work)
    dist.destroy_process_group()


def test_two_rank_reduction():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (15.0, 201.0)
