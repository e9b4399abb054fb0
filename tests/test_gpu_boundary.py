"""Boundary calls beyond the anneal itself, through the C ABI on the GPU.

- pa_step_records: every run's record at the temperature it has reached, in
  one gather, equals the per-run copies.
- pa_set_allocator: an engine whose pools come from PyTorch's caching
  allocator gives records identical to the default (cudaMalloc) engine, and
  returns every block; an allocator that refuses the k-th request makes
  pa_create fail with PA_ERR_OOM after handing back every block it had
  granted (no leak), for every k.
- Cancelling a served job before its last temperature leaves the other
  resident jobs bit-identical to running alone.
"""
import numpy as np
import pytest

from paper_2207_05535_gb300 import _lib
from paper_2207_05535_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2207_05535_gb300 import build
    build.build()
    _lib.load()


def _mixed():
    import dataclasses
    fm = W.ferro_runs(L=8, R=300, theta=2, beta_f=0.6, n=9, M=3, seed=2)
    pair = [dataclasses.replace(d, paired=d.paired + len(fm))
            for d in W.glass_pairs(L=16, R=200, theta=2, beta_f=2.0, n=9, n_samples=1, seed=3)]
    return fm + pair + [W.RunDesc(12, W.EA_PMJ, 150, 2, W.schedule(1.5, 6), seed=4, run_id=9, disorder_id=2)]


def test_step_records_gather_equals_per_run_records():
    descs = _mixed()
    idx = np.arange(len(descs), dtype=np.uint32)
    with _lib.Engine(descs) as eng:
        for i in range(1, 9):
            eng.step(1)
            got = eng.step_records(idx[::-1])
            for k in range(len(descs)):
                step = min(i, descs[k].n_beta - 1)
                want = eng.records(k)[step]
                assert got[len(descs) - 1 - k].tobytes() == want.tobytes(), (i, k)
        with pytest.raises(_lib.PAError):
            eng.step_records(np.array([len(descs)], dtype=np.uint32))


def test_engine_on_torch_caching_allocator_matches_default():
    import torch
    torch.cuda.set_device(0)
    descs = _mixed()
    with _lib.Engine(descs) as ref:
        ref.run_to_end()
        want = [ref.records(k) for k in range(len(descs))]
    live, wrong = {}, []

    def alloc(nbytes, device, stream, ctx):
        p = torch.cuda.caching_allocator_alloc(nbytes, device, stream)
        live[p] = nbytes
        return p

    def free(ptr, nbytes, device, stream, ctx):
        if live.pop(ptr, None) != nbytes:  # an exception would not cross the callback
            wrong.append(ptr)
        torch.cuda.caching_allocator_delete(ptr)

    base = torch.cuda.memory_allocated()
    _lib.pa_set_allocator(alloc, free)
    try:
        eng = _lib.Engine(descs)
    finally:
        _lib.pa_set_allocator()
    assert live and torch.cuda.memory_allocated() - base >= sum(live.values())
    eng.run_to_end()
    for k in range(len(descs)):
        assert eng.records(k).tobytes() == want[k].tobytes(), k
    eng.weighted_average(np.arange(3, dtype=np.uint32), 3, 0)  # grows an engine buffer through the allocator
    eng.close()
    assert not live and not wrong, "blocks not returned, or returned with another size"
    assert torch.cuda.memory_allocated() == base


def test_refused_allocation_fails_create_without_leaks():
    import torch
    torch.cuda.set_device(0)
    descs = _mixed()
    state = {"n": 0, "fail_at": 0}
    live = set()

    def alloc(nbytes, device, stream, ctx):
        state["n"] += 1
        if state["n"] == state["fail_at"]:
            return None
        p = torch.cuda.caching_allocator_alloc(nbytes, device, stream)
        live.add(p)
        return p

    def free(ptr, nbytes, device, stream, ctx):
        live.discard(ptr)
        torch.cuda.caching_allocator_delete(ptr)

    # count the requests of one creation, then refuse each of them in turn
    _lib.pa_set_allocator(alloc, free)
    try:
        _lib.Engine(descs).close()
        total = state["n"]
        assert total > 10 and not live
        for k in range(1, total + 1):
            state.update(n=0, fail_at=k)
            with pytest.raises(_lib.PAError) as ei:
                _lib.Engine(descs)
            assert ei.value.code == 2  # PA_ERR_OOM
            assert not live, k
    finally:
        _lib.pa_set_allocator()
    with _lib.Engine(descs) as eng:  # the default allocator again
        eng.run_to_end()


def test_cancelled_job_leaves_the_others_unchanged():
    jobs = [W.RunDesc(8, W.FERRO, 300, 2, W.schedule(0.8, 10), seed=6, run_id=1),
            W.RunDesc(16, W.EA_PMJ, 200, 2, W.schedule(2.0, 10), seed=6, run_id=2, disorder_id=1,
                      overlap=W.Q_SHIFT),
            W.RunDesc(12, W.EA_PMJ, 100, 2, W.schedule(2.0, 10), seed=6, run_id=3, disorder_id=2)]
    alone = []
    for d in jobs:
        with _lib.Engine([d]) as e:
            e.run_to_end()
            alone.append(e.records(0, qhist=bool(d.overlap)))
    cfg = _lib.pa_server_config()
    cfg.max_runs, cfg.replica_capacity, cfg.spin_words = 3, 3000, 3000 * 40
    cfg.record_capacity, cfg.qhist_words, cfg.scratch_words = 40, 3 * 10 * 300, 20000
    cfg.coupling_words, cfg.table_doubles = 600, 100000
    h = _lib.pa_server_create(cfg)
    try:
        slots = _lib.pa_admit(h, jobs)
        _lib.pa_anneal_step(h, 4)
        _lib.pa_retire(h, slots[1])  # cancelled at temperature 4 of 9
        _lib.pa_anneal_step(h, 5)
        _lib.pa_sync(h)
        for k in (0, 2):
            got = _lib.pa_records(h, slots[k], jobs[k].n_beta)
            assert got.tobytes() == alone[k].tobytes(), k
    finally:
        _lib.pa_destroy(h)


def test_weighted_average_beyond_65535_groups():
    """Groups run along the grid's x dimension: 65,600 groups of one run each
    (more than a grid's y dimension holds).  With M = 1 every weight is 1, so a
    group's W[e] is its run's own mean energy per site at each temperature."""
    n = 65600
    descs = [W.RunDesc(4, W.FERRO, 4, 1, W.schedule(0.5, 3), seed=5, run_id=r) for r in range(n)]
    with _lib.Engine(descs) as eng:
        eng.run_to_end()
        est = eng.weighted_average(np.arange(n, dtype=np.uint32), 1)
        assert est.shape == (n, 3)
        for k in (0, 1, 65534, 65535, 65536, n - 1):
            rec = eng.records(k)
            e = rec["sumE"].astype(np.float64) / (16.0 * rec["R"].astype(np.float64))
            assert np.allclose(est["W_e"][k], e, rtol=1e-12, atol=0.0), k
