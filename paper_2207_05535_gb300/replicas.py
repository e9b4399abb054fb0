"""Multi-GPU form of the engine: independent replicas, no collective on the data path.

Population-annealing runs are independent (their randomness is keyed by run
and disorder ids), so N GPUs anneal disjoint runs with no exchange step:
  - weak scaling (`shard`): every rank anneals the whole workload shape with
    its run and disorder ids offset, so no two ranks draw the same runs;
  - a fixed batch over N GPUs (`split`): the batch's runs are divided into
    contiguous blocks (pairs of populations stay together) and, after the
    anneal, every run's records are gathered to rank 0 (`gather_records`) in
    batch order, where the free-energy-weighted averages over groups of M runs
    (Sec. IV, Eqs. W_conf, W_F) come out exactly as on one GPU: a run's records
    do not depend on which runs share its GPU.
The only other cross-rank traffic is the measurement: a barrier, the max of
the ranks' device times and the sum of their attempted updates.
"""
from __future__ import annotations

import dataclasses

RUN_STRIDE = 200000
DISORDER_STRIDE = 100000


def shard(descs, rank: int):
    """Rank `rank`'s batch: the same workload with run and disorder ids offset
    (pair indices inside the batch are unchanged)."""
    out = []
    for d in descs:
        out.append(dataclasses.replace(d, run_id=d.run_id + RUN_STRIDE * rank,
                                       disorder_id=d.disorder_id + DISORDER_STRIDE * rank))
    return out


def reduce_timing(ms: float, updates: float, dist=None, device="cpu"):
    """Whole-job figures: (max over ranks of the timed ms, sum of updates)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, updates
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def split(descs, rank: int, world: int):
    """Rank `rank`'s block of a fixed batch divided over `world` ranks: (its
    descriptors, their indices in the batch).  Blocks are contiguous and a
    paired population stays with its partner (pair indices are re-based)."""
    units, k = [], 0
    while k < len(descs):  # a unit is one run, or a run and its partner when they are adjacent
        p = descs[k].paired
        n = 2 if p == k + 1 and descs[k + 1].paired == k else 1
        units.append(list(range(k, k + n)))
        k += n
    for u in units:
        for j in u:
            p = descs[j].paired
            if p >= 0 and p not in u:
                raise ValueError("paired populations must be adjacent in the batch")
    per = (len(units) + world - 1) // world
    mine = [j for u in units[rank * per:(rank + 1) * per] for j in u]
    first = mine[0] if mine else 0
    local = [dataclasses.replace(descs[j], paired=descs[j].paired - first if descs[j].paired >= 0 else -1)
             for j in mine]
    return local, mine


def gather_records(local_records, batch_idx, n_total: int, dist=None):
    """Every run's records on rank 0, in batch order: local_records[k] (a
    record array) belongs to batch run batch_idx[k].  Returns the list of
    n_total record arrays on rank 0 and None elsewhere (the local list when
    there is no process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(local_records)
    import numpy as np
    payload = [(int(j), r.dtype.descr, r.tobytes()) for j, r in zip(batch_idx, local_records)]
    parts = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
    dist.gather_object(payload, parts, dst=0)
    if dist.get_rank() != 0:
        return None
    out = [None] * n_total
    for part in parts:
        for j, descr, raw in part:
            out[j] = np.frombuffer(raw, dtype=np.dtype(descr)).copy()
    if any(r is None for r in out):
        raise RuntimeError("records missing for some runs of the batch")
    return out
