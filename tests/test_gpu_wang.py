"""Parity of the Wang pairing (Sec. III.D: pairs (k, pi*_k) from random
permutations with a random search pattern, no pair within one family) between
the CUDA engine and the oracle: records (sums, pair counts, number of swaps)
and histograms bit for bit, weighted |q| and P(q) within 1e-12."""
import numpy as np
import pytest

import oracle as O
from paper_2207_05535_gb300 import _lib
from paper_2207_05535_gb300 import workloads as W
from tests.helpers import compare_records, oracle_runs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2207_05535_gb300 import build
    build.build()
    _lib.load()


def check(eng, descs, ora, k):
    d = descs[k]
    rec, qw = eng.records(k, wang=True)
    compare_records(rec, ora[k].records())
    for i in range(d.n_beta):
        assert np.array_equal(qw[i], ora[k].qhist_wang(i)), ("wang histogram", k, i)
    return rec


def test_wang_pairs_glass_and_ferromagnet():
    b = W.schedule(2.0, 8)
    descs = [W.RunDesc(8, W.EA_PMJ, 300, 2, b, seed=4, run_id=r, disorder_id=1, overlap=W.Q_SHIFT | W.Q_WANG)
             for r in range(2)]
    descs += [W.RunDesc(16, W.FERRO, 777, 2, W.schedule(0.6, 6), seed=4, run_id=5, overlap=W.Q_WANG),
              W.RunDesc(6, W.EA_PMJ, 65, 1, W.schedule(3.0, 9), seed=4, run_id=6, disorder_id=2, overlap=W.Q_WANG)]
    ora = oracle_runs(descs)
    with _lib.Engine(descs) as eng:
        eng.run_to_end()
        recs = [check(eng, descs, ora, k) for k in range(len(descs))]
    assert sum(int(r["wang_swaps"].sum()) for r in recs) > 0


def test_wang_pairing_skipped_where_a_family_dominates():
    # a small population quenched hard: one family takes over and no valid pairing exists
    descs = [W.RunDesc(4, W.FERRO, 12, 1, np.array([0.0, 0.05, 3.0, 3.0]), seed=s, run_id=s, overlap=W.Q_WANG)
             for s in range(8)]
    ora = oracle_runs(descs)
    with _lib.Engine(descs) as eng:
        eng.run_to_end()
        recs = [check(eng, descs, ora, k) for k in range(len(descs))]
    n = np.concatenate([r["n_q_wang"] for r in recs])
    assert np.any(n == 0) and np.any(n > 0)


def test_wang_pairs_near_the_capacity_limit():
    descs = [W.RunDesc(8, W.FERRO, 7000, 1, W.schedule(0.5, 4), seed=2, run_id=9, R_cap=8192, overlap=W.Q_WANG)]
    ora = oracle_runs(descs)
    with _lib.Engine(descs) as eng:
        eng.run_to_end()
        check(eng, descs, ora, 0)


@pytest.mark.parametrize("kind", [0, 1])
def test_weighted_wang_overlaps(kind):
    b = W.schedule(2.0, 6)
    descs = [W.RunDesc(8, W.EA_PMJ, 200, 2, b, seed=6, run_id=r, disorder_id=3, overlap=W.Q_WANG) for r in range(4)]
    ora = oracle_runs(descs)
    recs = np.stack([ora[k].records() for k in range(4)])
    qw = np.stack([np.stack([ora[k].qhist_wang(i) for i in range(6)]) for k in range(4)])
    o, _, _, oPw = O.weighted_average(recs, 64, kind, qh_wang=qw)
    with _lib.Engine(descs) as eng:
        eng.run_to_end()
        g, gPw = eng.weighted_average(np.arange(4, dtype=np.uint32), 4, kind, wang=True)
    assert np.allclose(g[0]["W_absq_wang"], o["W_absq_wang"], rtol=1e-12, atol=0)
    assert np.allclose(gPw[0], oPw, rtol=1e-12, atol=1e-15)
    h, _, _, hPw = _lib.pa_weighted_average(recs, 64, kind, qh_wang=qw)
    assert np.allclose(h["W_absq_wang"], o["W_absq_wang"], rtol=1e-12, atol=0)
    assert np.allclose(hPw, oPw, rtol=1e-12, atol=1e-15)
