"""Checkpoint and resume of runs between anneal steps, and the launch count
the engine reports for graph replays."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2207_05535_gb300 import _lib
from paper_2207_05535_gb300 import workloads as W
from tests.helpers import compare_records

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2207_05535_gb300 import build
    build.build()
    _lib.load()


def _descs():
    b = W.schedule(2.0, 9)
    Jr, Jd = O.couplings(4, W.FERRO, 3, 0)
    log_g = np.array([math.log(c) if c else -math.inf for c in O.dos_transfer(4, Jr, Jd)])
    return W.glass_pairs(L=16, R=300, theta=2, beta_f=2.0, n=9, n_samples=1, seed=4) + [
        W.RunDesc(8, W.FERRO, 500, 3, W.schedule(0.5, 9), seed=4, run_id=5),
        W.RunDesc(8, W.EA_PMJ, 400, 2, b, seed=4, run_id=6, disorder_id=2, resample=W.MULTINOMIAL),
        W.RunDesc(4, W.FERRO, 700, W.THETA_INF, W.schedule(0.6, 9), seed=4, run_id=7, log_g=log_g),
    ]


def _state(eng, descs, k):
    rec = eng.records(k, qhist=bool(descs[k].overlap))
    return rec, eng.population(k)


def test_resumed_runs_finish_as_if_never_stopped():
    descs = _descs()
    with _lib.Engine(descs) as ref:
        ref.run_to_end()
        want = [_state(ref, descs, k) for k in range(len(descs))]
    with _lib.Engine(descs) as a:
        a.step(4)
        a.sync()
        blobs = [a.checkpoint(k) for k in range(len(descs))]
    with _lib.Engine(descs) as b:
        for k, blob in enumerate(blobs):
            b.restore(k, blob)
        b.run_to_end()
        for k, d in enumerate(descs):
            rec, pop = _state(b, descs, k)
            wrec, wpop = want[k]
            if d.overlap:
                for x, y in zip(rec[1:], wrec[1:]):
                    assert np.array_equal(x, y), k
                rec, wrec = rec[0], wrec[0]
            compare_records(rec, wrec, rtol=0.0)
            for x, y in zip(pop, wpop):
                assert np.array_equal(x, y), k


def test_restore_rejects_another_descriptor_and_leaves_the_run_alone():
    descs = _descs()
    with _lib.Engine(descs) as a:
        a.step(2)
        a.sync()
        blob = a.checkpoint(2)
        before = _state(a, descs, 3)
        with pytest.raises(_lib.PAError) as ei:
            a.restore(3, blob)  # run 3 is another descriptor
        assert ei.value.code == 1
        with pytest.raises(_lib.PAError):
            a.restore(2, blob[:-8])  # truncated
        after = _state(a, descs, 3)
        compare_records(after[0], before[0], rtol=0.0)
        a.restore(2, blob)  # the run's own checkpoint restores cleanly


def test_graph_replays_report_the_kernels_they_launch():
    descs = _descs()
    counts = {}
    for use_graph in (False, True):
        with _lib.Engine(descs) as e:
            e.step(1, use_graph)  # the first step also tunes the sweep shapes
            e.sync()
            l0 = e.launches
            e.step(3, use_graph)
            e.sync()
            counts[use_graph] = e.launches - l0
    assert counts[True] == counts[False] > 0
