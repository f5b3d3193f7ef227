"""The N-GPU path of bench.py runs independent replicas (the plain LB-IB
step does not shard); its only collective is the max over ranks of the
timed region.  Checked here with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank r took (10 + r) ms for the step and (4 + r) ms in the fluid kernel
    value, ms = bench.replica_throughput([10.0 + rank, 4.0 + rank], cells=1000, steps=50, world=world)
    out[rank] = (value, ms)
    dist.destroy_process_group()


def test_replica_throughput_takes_slowest_rank_and_all_work():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        value, ms = out[r]
        assert ms == [11.0, 5.0]  # max over ranks, on every rank
        assert value == pytest.approx(world * 1000 * 50 / 11e-3 / 1e6)


def test_single_process_needs_no_collective():
    import bench

    value, ms = bench.replica_throughput([8.0, 2.0], cells=400 * 1200, steps=100, world=1)
    assert ms == [8.0, 2.0] and value == pytest.approx(400 * 1200 * 100 / 8e-3 / 1e6)
