"""The N-GPU path of the benchmark runs independent replicas and reports the units of all
ranks over the slowest rank's time.  Checked here with two gloo ranks on the CPU."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, t = bench.aggregate(1.0 + rank, 5, world, "cpu")
    out[rank] = (value, t)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_takes_the_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(world):
            value, t = out[r]
            assert t == pytest.approx(2.0)
            assert value == pytest.approx(world * 5 / 2.0)


def test_aggregate_single_rank():
    import bench
    assert bench.aggregate(2.0, 4, 1, "cpu") == (2.0, 2.0)
