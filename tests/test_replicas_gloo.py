"""The N > 1 path on CPU: two gloo ranks shard the workload into disjoint runs
and reduce the timing (max) and the attempted updates (sum), as bench.py does
under torchrun."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2207_05535_gb300 import replicas
from paper_2207_05535_gb300 import workloads as W


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        descs = replicas.shard(W.glass_L16_R5000(n_samples=3), rank)
        ids = sorted((d.run_id, d.disorder_id) for d in descs)
        pairs = [d.paired for d in descs]
        ms, upd = replicas.reduce_timing(10.0 * (rank + 1), 1000.0 * (rank + 1), dist)
        dist.barrier()
        q.put((rank, ids, pairs, ms, upd))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 2000
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        rank, ids, pairs, ms, upd = q.get(timeout=120)
        got[rank] = (ids, pairs, ms, upd)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ids0, ids1 = set(got[0][0]), set(got[1][0])
    assert len(ids0) == len(got[0][0]) == 6 and not (ids0 & ids1)          # disjoint runs and disorder samples
    assert {r for r, _ in ids0} == {0, 1, 2, 3, 4, 5}
    assert got[0][1] == got[1][1] == [1, 0, 3, 2, 5, 4]                    # pairing is batch-local
    for r in range(world):
        assert got[r][2] == 20.0 and got[r][3] == 3000.0                    # max time, summed updates


def test_single_process_reduce_is_identity():
    assert replicas.reduce_timing(3.5, 7.0, None) == (3.5, 7.0)
