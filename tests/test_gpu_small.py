"""The one-launch-per-step path of small runs (anneal_small_kernel).

Runs with L = 8, 16 or 32, nearest-integer resampling, no overlaps and
R_cap <= 8192 are resampled, swept and measured by one thread-block cluster
per run and temperature (all temperatures in one launch when every resident
run is small).  They must equal the oracle bit for bit, equal the per-stage
kernels (PA_CREATE_SEPARATE_KERNELS) byte for byte, and not depend on the
cluster size or on which runs share the launch.
"""
import numpy as np
import pytest

from paper_2207_05535_gb300 import _lib
from paper_2207_05535_gb300 import workloads as W
from tests.helpers import compare_records, oracle_runs

pytestmark = pytest.mark.gpu
SEPARATE = 4  # PA_CREATE_SEPARATE_KERNELS


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2207_05535_gb300 import build
    build.build()
    _lib.load()


def _small_mix():
    return [W.RunDesc(8, W.FERRO, 500, 3, W.schedule(0.5, 9), seed=1, run_id=0),
            W.RunDesc(8, W.EA_PMJ, 33, 2, W.schedule(2.0, 7), seed=1, run_id=1, disorder_id=4),
            W.RunDesc(16, W.EA_PMJ, 700, 2, W.schedule(3.0, 8), seed=1, run_id=2, disorder_id=5),
            W.RunDesc(16, W.FERRO, 1, 3, W.schedule(0.6, 6), seed=1, run_id=3),
            W.RunDesc(32, W.FERRO, 150, 2, W.schedule(0.44, 5), seed=1, run_id=4),
            W.RunDesc(32, W.EA_PMJ, 90, 1, W.schedule(1.5, 6), seed=1, run_id=5, disorder_id=6)]


def _state(eng, descs):
    out = []
    for k in range(len(descs)):
        out.append((eng.records(k).tobytes(),) + tuple(np.asarray(x).tobytes() for x in eng.population(k)))
    return out


def test_small_runs_equal_oracle():
    descs = _small_mix()
    ora = oracle_runs(descs)
    with _lib.Engine(descs) as eng:
        l0 = eng.launches
        eng.run_to_end()
        assert eng.launches - l0 == 3  # one launch per lattice size for the whole anneal
        for k, d in enumerate(descs):
            compare_records(eng.records(k), ora[k].records())
            s, E, M, fam, step = eng.population(k)
            os_, oE, oM, ofam = ora[k].population()
            assert step == d.n_beta - 1
            assert np.array_equal(s, os_) and np.array_equal(E, oE) and np.array_equal(M, oM)
            assert np.array_equal(fam, ofam)


@pytest.mark.parametrize("use_graph", [True, False])
def test_small_path_equals_separate_kernels(use_graph):
    descs = _small_mix()
    with _lib.Engine(descs) as a, _lib.Engine(descs, flags=SEPARATE) as b:
        for n in (1, 3, 10):  # step by step, then several steps per call
            a.step(n, use_graph)
            b.step(n, use_graph)
            assert _state(a, descs) == _state(b, descs), n


def test_small_runs_beside_other_runs_and_cluster_sizes():
    """Small runs share every tick with runs on the per-stage kernels (graph
    replays); a run's result does not depend on the path or the cluster size
    (one run alone gets a cluster of 8 CTAs; 200 runs, too many for a cluster
    each, go to the per-stage kernels)."""
    small = _small_mix()
    big = [W.RunDesc(10, W.EA_PMJ, 200, 2, W.schedule(2.0, 8), seed=2, run_id=10, disorder_id=1,
                     overlap=W.Q_SHIFT),
           W.RunDesc(64, W.FERRO, 30, 1, W.schedule(0.44, 4), seed=2, run_id=11),
           W.RunDesc(8, W.FERRO, 300, 2, W.schedule(0.5, 6), seed=2, run_id=12, resample=W.MULTINOMIAL)]
    descs = small + big
    ora = oracle_runs(descs)
    with _lib.Engine(descs) as eng:
        eng.run_to_end(True)
        for k in range(len(descs)):
            compare_records(eng.records(k), ora[k].records())
    crowd = [W.RunDesc(8, W.FERRO, 500, 3, W.schedule(0.5, 9), seed=9, run_id=100 + r) for r in range(199)]
    with _lib.Engine(small[:1]) as alone, _lib.Engine(small[:1] + crowd) as many:
        alone.run_to_end()
        many.run_to_end()
        assert alone.records(0).tobytes() == many.records(0).tobytes()
        assert [np.asarray(x).tobytes() for x in alone.population(0)] == \
               [np.asarray(x).tobytes() for x in many.population(0)]


def test_small_run_near_capacity_and_overflow():
    """R_cap = 8192, the largest population the small path accepts (this one
    gets no launch shape that keeps its cluster's CTAs to one tile each, so the
    engine anneals it per stage); then a capacity overflow on the small path
    stops the run with its status, like the per-stage path."""
    d = [W.RunDesc(16, W.EA_PMJ, 7600, 1, W.schedule(2.0, 5), seed=3, run_id=0, disorder_id=2, R_cap=8192)]
    ora = oracle_runs(d)
    with _lib.Engine(d) as eng:
        eng.run_to_end()
        compare_records(eng.records(0), ora[0].records())
    tight = [W.RunDesc(8, W.EA_PMJ, 200, 1, W.schedule(3.0, 30), run_id=0, disorder_id=1, R_cap=201)]
    recs = []
    for flags in (0, SEPARATE):
        with _lib.Engine(tight, flags=flags) as eng:
            eng.step(29)
            with pytest.raises(_lib.PAError) as ei:
                eng.sync()
            assert ei.value.code == 3
            recs.append(eng.records(0).tobytes())
    assert recs[0] == recs[1]


@pytest.mark.slow
def test_ising_L8_R500_workload_small_path():
    """The 20-run Ising L=8 workload (R=500, 51 temperatures, theta=10) on the
    small path: four runs against the oracle, all twenty against the
    per-stage kernels."""
    descs = W.ising_L8_R500(M=20)
    ora = oracle_runs(descs, [0, 7, 13, 19])
    with _lib.Engine(descs) as a, _lib.Engine(descs, flags=SEPARATE) as b:
        a.run_to_end()
        b.run_to_end()
        for k in range(20):
            assert a.records(k).tobytes() == b.records(k).tobytes(), k
        for k in (0, 7, 13, 19):
            compare_records(a.records(k), ora[k].records())
