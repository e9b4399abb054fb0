"""Continuous batching: admission, retirement and results independent of the mix.

The GPU tests run jobs through a server engine (admitted at different steps,
retired as they finish, admitted again when memory frees up) and check each
job bit for bit against the same job run alone in its own engine, and against
the oracle.  The CPU test drives the request loop with a fake engine.
"""
import numpy as np
import pytest

from paper_2207_05535_gb300 import _lib, build, serve
from paper_2207_05535_gb300 import workloads as W


def _jobs():
    out = []
    for k, (L, model, R, n) in enumerate([(8, 0, 300, 7), (16, 1, 200, 5), (10, 1, 120, 9), (8, 1, 77, 4),
                                          (32, 0, 40, 6), (16, 0, 500, 8), (12, 0, 90, 3), (6, 1, 60, 10)]):
        out.append(W.RunDesc(L, model, R, 2, W.schedule(1.0 if model == 0 else 2.5, n), seed=5, run_id=100 + k,
                             disorder_id=k, overlap=W.Q_SHIFT if k % 3 == 0 else 0))
    return out


def _small_cfg():
    cfg = _lib.pa_server_config()
    cfg.max_runs = 3
    cfg.replica_capacity = 1500
    cfg.spin_words = 1500 * 40
    cfg.record_capacity = 40
    cfg.qhist_words = 2 * 10 * 1100
    cfg.scratch_words = 20000
    cfg.coupling_words = 3 * 200
    cfg.table_doubles = 200000
    return cfg


@pytest.mark.gpu
def test_server_results_equal_alone_and_oracle():
    import oracle as O
    jobs = _jobs()
    srv = serve.Server(_small_cfg())
    pending = list(range(len(jobs)))
    got, busy_seen, steps = {}, 0, 0
    while pending or srv.resident:
        while pending:  # admit in order while there is room
            j = serve.Job(jobs[pending[0]], 0.0)
            j.index = pending[0]
            if not srv.try_admit(j):
                busy_seen += 1
                break
            pending.pop(0)
        srv.step()
        steps += 1
        for job in srv.collect():
            got[job.index] = job.records
    srv.close()
    assert busy_seen > 0, "the small pools must force admissions to wait"
    assert len(got) == len(jobs)
    for k, d in enumerate(jobs):
        with _lib.Engine([d]) as eng:
            eng.run_to_end()
            alone = eng.records(0)
        assert np.array_equal(got[k], alone), k
        o = O.OracleRun.from_desc(d)
        o.run_to_end()
        orec = o.records()
        for f in ("sumE", "sumE2", "sumAbsM", "sumM2", "sumE3", "sumE4", "sumAbsM3", "sumM4", "sum_c2", "sum_absq", "R",
                  "n_fam", "max_fam", "n_q"):
            assert np.array_equal(got[k][f], orec[f]), (k, f)
        assert np.allclose(got[k]["minus_betaF"], orec["minus_betaF"], rtol=1e-12, atol=0)


@pytest.mark.gpu
def test_admission_is_all_or_nothing_and_memory_is_reused():
    cfg = _small_cfg()
    h = _lib.pa_server_create(cfg)
    try:
        big = W.RunDesc(16, 0, 1100, 1, W.schedule(1.0, 3), run_id=1)
        (s0,) = _lib.pa_admit(h, [big])
        with pytest.raises(_lib.PAError) as ei:
            _lib.pa_admit(h, [W.RunDesc(16, 0, 1100, 1, W.schedule(1.0, 3), run_id=2)])
        assert ei.value.code == serve.BUSY
        _lib.pa_anneal_step(h, 2, False)
        assert _lib.pa_finished(h) == [s0]
        _lib.pa_retire(h, s0)
        (s1,) = _lib.pa_admit(h, [W.RunDesc(16, 0, 1100, 1, W.schedule(1.0, 3), run_id=2)])
        _lib.pa_anneal_step(h, 2, False)
        step, R, status = _lib.pa_run_state(h, s1)
        assert step == 2 and status == 0 and R > 1000
    finally:
        _lib.pa_destroy(h)


class _FakeEngine:
    """Engine double: runs finish after n_beta - 1 steps; capacity in runs."""

    def __init__(self, cap):
        self.cap, self.res, self.next = cap, {}, 0

    def pa_server_create(self, cfg, stream, flags):
        return 1

    def pa_admit(self, h, runs):
        if len(self.res) + len(runs) > self.cap:
            raise _lib.PAError(serve.BUSY, "pa_admit")
        slots = []
        for d in runs:
            self.res[self.next] = [d, 0]
            slots.append(self.next)
            self.next += 1
        return slots

    def pa_anneal_step(self, h, n, g):
        for v in self.res.values():
            v[1] = min(v[0].n_beta - 1, v[1] + n)

    def pa_finished(self, h):
        return [s for s, v in self.res.items() if v[1] == v[0].n_beta - 1]

    def pa_sync(self, h):
        pass

    def pa_records(self, h, slot, n, N, q):
        r = np.zeros(n, dtype=_lib.RECORD_DTYPE)
        r["R"] = self.res[slot][0].R
        return r

    def pa_retire(self, h, slot):
        del self.res[slot]

    def pa_destroy(self, h):
        pass


def test_request_loop_admits_fifo_and_accounts_latency():
    clock = {"t": 0.0}
    descs = [W.RunDesc(8, 0, 10, 1, W.schedule(1.0, n)) for n in (3, 5, 2, 4, 3)]
    arrivals = [(0.1 * k, d) for k, d in enumerate(descs)]
    srv = serve.Server(None, engine=_FakeEngine(cap=2))

    def tick_clock():
        clock["t"] += 0.05
        return clock["t"]

    done, stats = serve.serve(arrivals, srv, clock=tick_clock, sleep=lambda s: clock.__setitem__("t", clock["t"] + s))
    assert len(done) == 5 and stats["steps"] > 0
    assert [j.desc for j in sorted(done, key=lambda j: j.admitted)] == descs     # FIFO admission
    assert all(j.finished >= j.admitted >= j.arrival for j in done)
    s = serve.summarize(done, stats["wall_s"])
    assert s["jobs"] == 5 and s["p99_latency_s"] >= s["p50_latency_s"] > 0


def _pool_bytes(c):
    """Device bytes of a server's pools (both spin and E/M/family buffers; records with
    their beta, two thresholds and table offset; three overlap histograms)."""
    return (2 * 4 * c.spin_words + (2 * 3 + 2) * 4 * c.replica_capacity
            + (_lib.RECORD_DTYPE.itemsize + 32) * c.record_capacity + 3 * 4 * c.qhist_words
            + 4 * c.coupling_words + 8 * c.scratch_words + 8 * c.table_doubles)


def test_config_for_budget_scales_with_memory():
    build.build()
    a = serve.config_for_budget(8 << 30)
    b = serve.config_for_budget(32 << 30)
    q = serve.config_for_budget(8 << 30, max_runs=256, overlap_frac=0.5)
    assert b.replica_capacity > 3 * a.replica_capacity
    assert a.record_capacity == 4096 * 300 and q.qhist_words == 128 * 300 * 4097
    for c, budget in ((a, 8 << 30), (b, 32 << 30), (q, 8 << 30)):
        assert 0.95 * budget < _pool_bytes(c) <= budget
    # the spin pool holds the replica pool at the mean stride of the even L in 8..64
    one = [_lib.pa_pool_sizes([W.RunDesc(L, W.FERRO, 1, 1, W.schedule(1.0, 2))]) for L in range(8, 65, 2)]
    mean = sum(c.spin_words / c.replica_capacity for c in one) / len(one)
    assert a.spin_words >= a.replica_capacity * mean
    with pytest.raises(ValueError):
        serve.config_for_budget(1 << 20)
