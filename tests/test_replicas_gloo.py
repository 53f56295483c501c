"""The replica path of bench.py (`--gpus N` under torchrun: N independent solves, no
data-path collective) on two CPU processes with the gloo backend: the barrier, the maximum over
ranks that ends the timed region, and the whole-job value."""
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
    bench.barrier(world)
    ms_local = 2.0 + rank  # rank 1 is the slower replica
    ms, value = bench.replica_value(ms_local, world)
    out[rank] = (ms, value)
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, value = res[rank]
        assert ms == 3.0  # the maximum over ranks, seen by every rank
        assert value == pytest.approx(world * 1000.0 / 3.0)


def test_single_process_needs_no_group():
    import bench
    assert bench.replica_value(4.0, 1) == (4.0, 250.0)
