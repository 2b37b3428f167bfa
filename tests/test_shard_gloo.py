"""Replica sharding over two ranks on CPU (gloo): the shards partition the
workload, each rank solves its own graphs (the oracle stands in for the GPU
solve here), and the results gathered on rank 0 equal a single-process run;
the timing reductions give the slowest rank's time and the total count."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1602_04386_gb300 import inputs, shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, count, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        ws, r, _ = shard.dist_env()
        assert (ws, r) == (world, rank)
        mine = shard.shard_indices(count, rank, world)
        lams = {}
        for i in mine:
            g = inputs.batch_mix_item(i, scale_range=(6, 7), side_range=(6, 12))
            lams[i] = oracle.solve(g).lam
        t_max = shard.reduce_max(float(rank + 1), dist)
        n_sum = shard.reduce_sum(float(len(mine)), dist)
        gathered = [None] * world
        dist.all_gather_object(gathered, lams)
        if rank == 0:
            merged = {}
            for part in gathered:
                merged.update(part)
            out.put((merged, t_max, n_sum))
    finally:
        dist.destroy_process_group()


def test_shards_partition_the_workload():
    for count in (0, 1, 7, 4096):
        for world in (1, 2, 3, 8):
            parts = [shard.shard_indices(count, r, world) for r in range(world)]
            flat = sorted(i for p in parts for i in p)
            assert flat == list(range(count))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        shard.shard_indices(4, 2, 2)


def test_two_rank_replicas_match_one_process():
    import oracle
    count, world = 10, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, count, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged, t_max, n_sum = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t_max == 2.0 and n_sum == count
    assert sorted(merged) == list(range(count))
    for i in range(count):
        g = inputs.batch_mix_item(i, scale_range=(6, 7), side_range=(6, 12))
        assert merged[i] == oracle.solve(g).lam
