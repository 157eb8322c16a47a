"""Multi-process host logic on CPU (gloo, world size 2): element shards of the
order-free element loop partition the mesh, each rank's shard of a seeded mesh
is reproducible, and the benchmark's max-over-ranks timing reduction works."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1604_05872_gb300 import inputs


def _worker(rank, world, port, E, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    start, count = inputs.shard(E, rank, world)
    ranges = [None] * world
    dist.all_gather_object(ranges, (start, count))
    coords, _ = inputs.workload(inputs.HELMHOLTZ, 2, E, seed=11)
    mine = coords[start:start + count]
    sums = torch.tensor([float(mine.sum())], dtype=torch.float64)
    dist.all_reduce(sums)
    t = torch.tensor([0.5 + rank], dtype=torch.float64)   # a per-rank "time"
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((ranges, float(sums.item()), float(coords.sum()), float(t.item())))
    dist.destroy_process_group()


@pytest.mark.parametrize("E", [10, 1001])
def test_two_rank_shards_partition_and_reduce(E):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, E, q)) for r in range(2)]
    for p in procs:
        p.start()
    ranges, s, total, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ranges[0][0] == 0 and ranges[0][0] + ranges[0][1] == ranges[1][0]
    assert ranges[1][0] + ranges[1][1] == E
    assert abs(s - total) < 1e-9 * abs(total)
    assert tmax == 1.5


def test_shard_arithmetic():
    for E in (0, 1, 7, 100, 12345):
        for world in (1, 2, 3, 8):
            got = [inputs.shard(E, r, world) for r in range(world)]
            assert sum(c for _, c in got) == E
            assert all(got[r][0] + got[r][1] == got[r + 1][0] for r in range(world - 1))
