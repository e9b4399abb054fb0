"""Parity of theta = infinity runs (Sec. V.B: energies drawn from the exact
density of states instead of sweeps) with the oracle, alone, mixed with
sweeping runs in one engine, and served."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2207_05535_gb300 import _lib, serve
from paper_2207_05535_gb300 import workloads as W
from tests.helpers import compare_records, oracle_runs

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2207_05535_gb300 import build
    build.build()
    _lib.load()


def _log_g(g):
    return np.array([math.log(c) if c else -math.inf for c in g])


def log_dos(L, model, seed, dis):
    if L == 8 and model == W.FERRO:  # stored exact L = 8 ferromagnet density of states
        with open(os.path.join(GOLD, "dos_fm_L8.json")) as f:
            gE = {int(k): int(v) for k, v in json.load(f)["g_by_E"].items()}
        return _log_g([gE.get(2 * u - 128, 0) for u in range(129)])
    Jr, Jd = O.couplings(L, model, seed, dis)
    return _log_g(O.dos_transfer(L, Jr, Jd))


def check(eng, descs, ora, k):
    d = descs[k]
    compare_records(eng.records(k), ora[k].records())
    s, E, M, fam, step = eng.population(k)
    os_, oE, oM, ofam = ora[k].population()
    assert step == d.n_beta - 1
    assert np.array_equal(E, oE) and np.array_equal(fam, ofam) and np.all(M == 0) and np.all(oM == 0)
    assert np.all(s == -1) and np.all(os_ == -1)


def _inf(L, model, R, betas, run_id, dis=0, resample=W.NEAREST, seed=3):
    return W.RunDesc(L, model, R, W.THETA_INF, betas, seed=seed, run_id=run_id, disorder_id=dis, resample=resample,
                     log_g=log_dos(L, model, seed, dis))


@pytest.mark.parametrize("L,model,R,resample", [(4, 0, 300, 0), (8, 0, 500, 0), (8, 0, 257, 1), (4, 1, 128, 0),
                                                (6, 1, 200, 1)])
def test_theta_inf_runs_bit_exact(L, model, R, resample):
    betas = W.schedule(0.6 if model == 0 else 2.0, 9)
    descs = [_inf(L, model, R, betas, r, dis=2, resample=resample) for r in range(3)]
    ora = oracle_runs(descs)
    with _lib.Engine(descs) as eng:
        eng.run_to_end()
        for k in range(len(descs)):
            check(eng, descs, ora, k)


@pytest.mark.parametrize("R,resample", [(20000, 0), (36000, 0), (6000, 1)])
def test_theta_inf_populations_over_several_ctas(R, resample):
    """Populations spanning several CTAs of the draw, resampling and
    measurement kernels (16384 replicas per CTA), L = 8 ferromagnet."""
    betas = W.schedule(0.6, 13)
    descs = [_inf(8, 0, R, betas, r, resample=resample) for r in range(2)]
    ora = oracle_runs(descs)
    with _lib.Engine(descs) as eng:
        eng.run_to_end()
        for k in range(len(descs)):
            check(eng, descs, ora, k)


def test_theta_inf_mixed_with_sweeping_runs():
    b8 = W.schedule(0.5, 7)
    descs = [_inf(8, 0, 400, b8, 0), W.RunDesc(8, W.FERRO, 300, 2, b8, seed=3, run_id=1),
             W.RunDesc(16, W.EA_PMJ, 200, 2, W.schedule(2.0, 5), seed=3, run_id=2, disorder_id=1,
                       overlap=W.Q_SHIFT),
             _inf(4, 1, 90, W.schedule(1.5, 11), 3, dis=5)]
    ora = oracle_runs(descs)
    with _lib.Engine(descs) as eng:
        eng.run_to_end()
        for k in (0, 3):
            check(eng, descs, ora, k)
        for k in (1, 2):
            compare_records(eng.records(k, qhist=False), ora[k].records())
        # no sweep group for L = 4 (theta = infinity) nor for L = 8 (a small run: one launch per step)
        assert [s[0] for s in _lib.pa_sweep_shapes(eng.h)] == [16]


def test_theta_inf_jobs_served_in_reused_memory():
    cfg = _lib.pa_server_config()
    cfg.max_runs = 2
    cfg.replica_capacity = 800
    cfg.spin_words = 800 * 8
    cfg.record_capacity = 40
    cfg.qhist_words = 0
    cfg.scratch_words = 4000
    cfg.coupling_words = 400
    cfg.table_doubles = 20000
    b = W.schedule(0.6, 6)
    job_inf = _inf(8, 0, 500, b, 7)
    job_sweep = W.RunDesc(8, W.FERRO, 500, 3, b, seed=3, run_id=8)
    ora = oracle_runs([job_inf, job_sweep])
    srv = serve.Server(cfg)
    try:
        got = {}
        for k, d in enumerate([job_inf, job_sweep]):  # the second job reuses the first one's memory
            j = serve.Job(d, 0.0)
            assert srv.try_admit(j)
            while k not in got:
                srv.step()
                for done in srv.collect():
                    got[k] = done.records
        for k in range(2):
            compare_records(got[k], ora[k].records())
    finally:
        srv.close()
