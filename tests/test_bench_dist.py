"""Host-side multi-rank logic of bench.py on CPU (gloo, world size 2): every rank
gets its own samples (weak scaling, disjoint shards), and the timed region's
duration is the max over ranks."""
import os

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    idx = bench.shard(8, rank, world)
    t = bench.reduce_max(10.0 + rank * 5.0, dist)
    gathered = [None] * world
    dist.all_gather_object(gathered, idx.tolist())
    if rank == 0:
        out.put((t, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_weak_scaling_shards_and_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    t, shards = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == 15.0
    assert sorted(shards[0] + shards[1]) == list(range(16))
    assert not set(shards[0]) & set(shards[1])
