"""Continuous-batching server for population-annealing jobs.

One server engine (pa_server_create) holds the resident jobs in fixed device
pools.  The request loop admits queued jobs first-in first-out whenever the
pools have room (pa_admit answers PA_ERR_BUSY otherwise), advances every
resident job by one temperature per step in shared launches, and streams each
finished job's records back before retiring it, which frees its memory for the
next admissions.  A job's result is the same alone and in the mix: its
randomness is keyed by its own seed and ids.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time

import numpy as np

from . import _lib
from . import workloads as W

BUSY = 8


def config_for_budget(budget_bytes: int, max_runs: int = 4096, min_L: int = 8, max_L: int = 64,
                      max_n_beta: int = 300, overlap_frac: float = 0.0, table_bytes: int = 512 << 20):
    """Pool sizes for a device-memory budget, for jobs with even L uniform in
    min_L..max_L and at most max_n_beta temperatures.  Per-replica and per-run
    words come from the engine's own layout (pa_pool_sizes of one small run per
    lattice size); the replicas share what the per-run parts leave."""
    Ls = range(min_L + (min_L & 1), max_L + 1, 2)
    if not Ls:
        raise ValueError("no even lattice size in min_L..max_L")
    one = [_lib.pa_pool_sizes([W.RunDesc(L, W.FERRO, 1, 1, W.schedule(1.0, 2))]) for L in Ls]
    words_per_replica = math.ceil(sum(c.spin_words // c.replica_capacity for c in one) / len(one))
    # per replica: both spin buffers, E, M and family in both buffers, parent and copy
    # number, and half a 64-bit scratch word (the multinomial member list)
    bytes_per_replica = 2 * 4 * words_per_replica + 2 * 3 * 4 + 2 * 4 + 4
    N_max = max_L * max_L
    coupling = max(c.coupling_words for c in one)          # 32-bit words per run
    scratch_run = max(c.scratch_words for c in one) + 1    # 64-bit words per run (histograms, level tables)
    per_step = _lib.RECORD_DTYPE.itemsize + 8 + 16 + 8     # record, beta, two thresholds, table offset
    n_q = int(overlap_frac * max_runs)
    qhist_bytes = 3 * 4 * n_q * max_n_beta * (N_max + 1)  # index-shift, two-population and Wang histograms
    per_run_fixed = per_step * max_n_beta + 8 * scratch_run + 4 * coupling
    rest = budget_bytes - table_bytes - max_runs * per_run_fixed - qhist_bytes
    if rest <= 0:
        raise ValueError("budget too small for the slot count")
    reps = int(rest // bytes_per_replica)
    cfg = _lib.pa_server_config()
    cfg.max_runs = max_runs
    cfg.replica_capacity = reps
    cfg.spin_words = reps * words_per_replica
    cfg.record_capacity = max_runs * max_n_beta
    cfg.qhist_words = n_q * max_n_beta * (N_max + 1)
    cfg.scratch_words = reps // 2 + max_runs * scratch_run
    cfg.coupling_words = max_runs * coupling
    cfg.table_doubles = table_bytes // 8
    return cfg


@dataclasses.dataclass
class Job:
    desc: object
    arrival: float
    slot: int = -1
    admitted: float = 0.0
    finished: float = 0.0
    records: object = None


class Server:
    """A server engine and its resident jobs."""

    def __init__(self, cfg, stream=None, flags=0, engine=None):
        self.api = engine or _lib
        self.h = self.api.pa_server_create(cfg, stream, flags)
        self.resident = {}  # slot -> Job

    def close(self):
        if self.h:
            self.api.pa_destroy(self.h)
            self.h = None

    def try_admit(self, job) -> bool:
        try:
            (slot,) = self.api.pa_admit(self.h, [job.desc])
        except _lib.PAError as e:
            if e.code == BUSY:
                return False
            raise
        job.slot = slot
        self.resident[slot] = job
        return True

    def step(self):
        self.api.pa_anneal_step(self.h, 1, False)

    def collect(self):
        """Records of the jobs that reached their last temperature; retires them."""
        done = []
        fin = self.api.pa_finished(self.h)
        if fin:
            self.api.pa_sync(self.h)
        for slot in fin:
            job = self.resident.pop(slot)
            d = job.desc
            job.records = self.api.pa_records(self.h, slot, d.n_beta, d.N, False)
            self.api.pa_retire(self.h, slot)
            done.append(job)
        return done


def serve(arrivals, server, clock=time.perf_counter, sleep=time.sleep):
    """Run a stream of (arrival_seconds, RunDesc) through `server` in real time.

    Returns the finished jobs (with admission/finish times) and loop statistics."""
    arrivals = sorted(arrivals, key=lambda a: a[0])
    queue = collections.deque()
    nxt, done, steps = 0, [], 0
    t0 = clock()
    while nxt < len(arrivals) or queue or server.resident:
        now = clock() - t0
        while nxt < len(arrivals) and arrivals[nxt][0] <= now:
            queue.append(Job(arrivals[nxt][1], arrivals[nxt][0]))
            nxt += 1
        while queue:  # first in, first out: a job that does not fit blocks the ones behind it
            if not server.try_admit(queue[0]):
                break
            job = queue.popleft()
            job.admitted = clock() - t0
        if not server.resident:
            if nxt < len(arrivals):
                sleep(max(0.0, arrivals[nxt][0] - (clock() - t0)))
            continue
        server.step()
        steps += 1
        for job in server.collect():
            job.finished = clock() - t0
            done.append(job)
    wall = clock() - t0
    return done, {"steps": steps, "wall_s": wall}


def summarize(done, wall_s):
    lat = np.array([j.finished - j.arrival for j in done]) if done else np.zeros(1)
    updates = sum(int(sum(j.desc.theta * j.desc.N * int(r) for r in j.records["R"][1:])) for j in done)
    return {"jobs": len(done), "wall_s": wall_s, "jobs_per_s": len(done) / wall_s if wall_s else 0.0,
            "updates_per_ns": updates / (wall_s * 1e9) if wall_s else 0.0,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "max_latency_s": float(lat.max())}
