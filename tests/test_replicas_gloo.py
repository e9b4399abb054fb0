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


def _split_worker(rank, world, port, q):
    import numpy as np

    import oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        batch = _batch()
    except Exception as exc:  # report instead of leaving the parent waiting
        q.put(([], repr(exc)))
        raise
    try:
        local, idx = replicas.split(batch, rank, world)
        recs = [O.OracleRun.from_desc(d) for d in local]
        for r in recs:
            r.run_to_end()
        out = replicas.gather_records([r.records() for r in recs], idx, len(batch), dist)
        if rank == 0:
            q.put((idx, [np.asarray(x).tobytes() for x in out]))
        else:
            q.put((idx, None))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _batch():
    import dataclasses
    fm = W.ferro_runs(L=6, R=60, theta=1, beta_f=0.6, n=5, M=5, seed=2)
    return fm + [dataclasses.replace(d, paired=d.paired + len(fm))
                 for d in W.glass_pairs(L=6, R=50, theta=1, beta_f=1.5, n=5, n_samples=2, seed=3)]


def test_fixed_batch_split_over_two_ranks_gives_one_rank_weighted_averages():
    """A fixed batch (5 ferromagnet runs and 2 glass samples of two paired
    populations) split over two gloo ranks: the records gathered to rank 0 are
    those of one process annealing the whole batch, so the free-energy
    weighted averages (Eqs. W_conf, W_F) over groups of runs are identical."""
    import numpy as np

    import oracle as O
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 31500 + os.getpid() % 2000
    procs = [ctx.Process(target=_split_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    assert not any(isinstance(g, str) for _, g in res), res
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    idx = sorted(j for i, _ in res for j in i)
    batch = _batch()
    assert idx == list(range(len(batch)))                                  # every run exactly once
    gathered = next(g for _, g in res if g is not None)
    one = []
    for d in batch:
        r = O.OracleRun.from_desc(d)
        r.run_to_end()
        one.append(r.records())
    assert gathered == [x.tobytes() for x in one]
    recs = np.stack([np.frombuffer(x, dtype=O.RECORD_DTYPE) for x in gathered])
    for grp, (lo, hi) in enumerate([(0, 5), (5, 7), (7, 9)]):
        a = O.weighted_average(recs[lo:hi], 36, 0)[0]
        b = O.weighted_average(np.stack(one[lo:hi]), 36, 0)[0]
        assert a.tobytes() == b.tobytes(), grp


def test_split_keeps_pairs_together_and_covers_the_batch():
    batch = _batch()
    for world in (1, 2, 3, 4):
        seen = []
        for rank in range(world):
            local, idx = replicas.split(batch, rank, world)
            seen += idx
            for d, j in zip(local, idx):
                if d.paired >= 0:
                    assert idx[d.paired] == batch[j].paired
        assert seen == list(range(len(batch)))
