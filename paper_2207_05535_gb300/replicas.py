"""Multi-GPU form of the engine: independent replicas, no collective on the data path.

Population-annealing runs are independent (their randomness is keyed by run
and disorder ids), so N GPUs each anneal their own batch: rank r offsets the
ids so no two ranks draw the same runs.  The only cross-rank traffic is the
measurement: a barrier, the max of the ranks' device times and the sum of
their attempted updates.
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
