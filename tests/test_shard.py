"""The screening batch split over ranks: every lattice goes to exactly one
rank, the cell counts stay balanced, every rank computes the same split,
and the whole-job rate sums the ranks' cells over the slowest rank's time.
The ranks are two gloo processes on CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1606_01805_gb300 import workloads as W
from paper_1606_01805_gb300.shard import rank_instances, shard_instances


def _cells():
    return [w.cells for w in W.batched_screening(steps=0)]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_split_covers_every_lattice_once_and_balances_cells(world):
    cells = _cells()
    parts = shard_instances(cells, world)
    assert len(parts) == world
    flat = sorted(k for p in parts for k in p)
    assert flat == list(range(len(cells)))
    loads = [sum(cells[k] for k in p) for p in parts]
    # greedy largest-first: no rank exceeds the lightest by more than the
    # largest single lattice
    assert max(loads) - min(loads) <= max(cells)
    assert all(p == sorted(p) for p in parts)


def test_split_special_cases():
    assert shard_instances([5, 5, 5], 1) == [[0, 1, 2]]
    # equal sizes: round robin in index order
    assert shard_instances([7, 7, 7, 7], 2) == [[0, 2], [1, 3]]
    # one large and three small: the large one alone
    assert shard_instances([1, 9, 2, 3], 2) == [[1], [0, 2, 3]]
    # more ranks than lattices: some ranks idle
    assert shard_instances([4, 4], 3) == [[0], [1], []]
    with pytest.raises(ValueError):
        shard_instances([1], 0)
    with pytest.raises(ValueError):
        rank_instances([1], 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    cells = _cells()
    mine = rank_instances(cells, rank, world)
    local = sum(cells[k] for k in mine)
    # rank r took (2 + r) ms per step, (1.5 + r) ms in the fluid kernel
    value, total, ms = bench.sharded_throughput(local, [2.0 + rank, 1.5 + rank], world)
    out[rank] = (mine, local, value, total, ms)
    dist.destroy_process_group()


def test_sharded_rate_sums_cells_and_takes_slowest_rank():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    cells = _cells()
    assert sorted(out[0][0] + out[1][0]) == list(range(len(cells)))
    assert out[0][1] + out[1][1] == sum(cells)
    for r in range(world):
        mine, local, value, total, ms = out[r]
        assert total == sum(cells)
        assert ms == [3.0, 2.5]
        assert value == pytest.approx(sum(cells) / 3e-3 / 1e6)


def test_single_rank_rate_needs_no_collective():
    import bench

    value, total, ms = bench.sharded_throughput(1000, [4.0, 3.0], 1)
    assert total == 1000 and ms == [4.0, 3.0] and value == pytest.approx(1000 / 4e-3 / 1e6)
