"""The weighted-averaging analysis suite: exact references, statistics, and
the same analysis on engine records and on oracle records."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2207_05535_gb300 import analysis as A
from paper_2207_05535_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_kaufman_matches_oracle_and_paper_ranges():
    for L in (4, 8, 16, 64, 128):
        for b in (0.05, 0.3, 0.4407, 0.6, 1.0):
            assert abs(A.kaufman_lnZ(L, b)[0] - O.kaufman_lnZ(L, b)) <= 1e-13 * O.kaufman_lnZ(L, b)
    with open(os.path.join(GOLD, "paper_values.json")) as f:
        for r in json.load(f)["minus_betaF_range_FM"]:
            assert r["lo"] <= A.kaufman_lnZ(r["L"], r["beta"])[0] <= r["hi"]


def test_exact_energy_and_heat_capacity_against_enumeration_and_dos():
    Jr, Jd = O.couplings(4, 0, 1, 0)
    ex = A.exact_ferro(4, [0.1, 0.4, 0.8])
    for k, b in enumerate([0.1, 0.4, 0.8]):
        bf = O.bruteforce(4, Jr, Jd, b)
        assert ex["e"][k] == pytest.approx(bf["e"], rel=1e-7)
        assert ex["c"][k] == pytest.approx(bf["c"], rel=1e-5)
    with open(os.path.join(GOLD, "dos_fm_L8.json")) as f:
        gE = {int(k): int(v) for k, v in json.load(f)["g_by_E"].items()}
    Es = np.array(sorted(gE), float)
    lg = np.array([math.log(gE[int(e)]) for e in Es])
    for b in (0.3, 0.4407, 0.6):
        p = np.exp(lg - b * Es - (lg - b * Es).max())
        p /= p.sum()
        e = (p * Es).sum() / 64
        c = b * b * ((p * Es * Es).sum() - (p * Es).sum() ** 2) / 64
        ex = A.exact_ferro(8, [b])
        assert ex["e"][0] == pytest.approx(e, rel=1e-7) and ex["c"][0] == pytest.approx(c, rel=1e-5)


def test_statistics_helpers():
    M = np.array([1, 2, 4, 8, 16, 32])
    a, b, s = A.fit_power_law(M, 0.37 * M ** -0.83)
    assert a == pytest.approx(0.37, rel=1e-12) and b == pytest.approx(0.83, rel=1e-12) and s < 1e-10
    rng = np.random.default_rng(0)
    x = rng.normal(size=50)
    m, se = A.jackknife(x)
    assert m == pytest.approx(x.mean()) and se == pytest.approx(x.std(ddof=1) / math.sqrt(50), rel=1e-12)
    est = rng.normal(1.0, 0.5, size=(2000, 3))
    assert np.allclose(A.rmsd(est, 0.0), np.sqrt(est.mean(0) ** 2 + est.var(0)))
    # Eq. varWpred against normalised weights of Gaussian -beta F: the log-normal
    # prediction holds for large M (Sec. IV.G); at M = 64 it is within a few percent
    Mw, s2 = 64, 0.09
    F = rng.normal(0.0, math.sqrt(s2), size=(8000, Mw))
    w = np.exp(F) / np.exp(F).sum(axis=1, keepdims=True)
    assert np.var(w) == pytest.approx(A.varw_prediction(F.reshape(-1), Mw), rel=0.05)


@pytest.mark.gpu
def test_analysis_on_engine_records_equals_analysis_on_oracle_records():
    from paper_2207_05535_gb300 import _lib
    descs = W.ferro_runs(L=6, R=120, theta=2, beta_f=0.6, n=7, M=48, seed=3)
    with _lib.Engine(descs) as eng:
        eng.run_to_end()
        ex = lambda b: A.exact_ferro(6, b)["e"]
        rows = A.bias_vs_M(eng, np.arange(48), [1, 2, 4, 8, 16], ex, obs="W_e")
    recs = []
    for d in descs:
        o = O.OracleRun.from_desc(d)
        o.run_to_end()
        recs.append(o.records())
    recs = np.stack(recs)
    for (M, S, bias, se) in rows:
        est = np.stack([O.weighted_average(recs[g * M:(g + 1) * M], 36, 0)[0] for g in range(48 // M)])
        diff = est["W_e"] - ex(est["beta"][0])[None, :]
        assert bias == pytest.approx(np.mean(np.abs(diff.mean(axis=0))), rel=1e-10, abs=1e-14)
        assert S == 48 // M


def test_bootstrap_standard_error():
    """The bootstrap standard error of a sample mean approaches the exact
    sqrt(var / n) (population variance of the sample) as resamples grow; it
    is reproducible with its seed and zero for a constant sample."""
    rng = np.random.default_rng(5)
    x = rng.normal(2.0, 3.0, size=400)
    m, se = A.bootstrap(x, n_boot=8000, seed=1)
    assert m == pytest.approx(x.mean())
    assert se == pytest.approx(x.std(ddof=0) / math.sqrt(len(x)), rel=0.05)
    assert A.bootstrap(x, n_boot=500, seed=7) == A.bootstrap(x, n_boot=500, seed=7)
    assert A.bootstrap(np.full(30, 1.5), n_boot=200)[1] == 0.0
    # a statistic over rows of a 2-D sample (as bias_vs_M resamples groups)
    y = rng.normal(size=(300, 4))
    _, se2 = A.bootstrap(y, lambda d: d.mean(axis=0)[0], n_boot=8000, seed=2)
    assert se2 == pytest.approx(y[:, 0].std(ddof=0) / math.sqrt(300), rel=0.05)


class _GroupedRecords:
    """Stands in for an engine: weighted_average returns fixed group estimates."""

    def __init__(self, est):
        self.est = est

    def weighted_average(self, runs, M, kind):
        return self.est[M]


def test_bias_vs_M_error_kinds():
    rng = np.random.default_rng(11)
    beta = np.array([0.40, 0.42, 0.44])
    est = {}
    for M, S in ((1, 64), (4, 16)):
        a = np.zeros((S, 3), dtype=[("beta", "f8"), ("W_e", "f8")])
        a["beta"] = beta
        a["W_e"] = 0.1 / M + rng.normal(0.0, 0.05, size=(S, 3))
        est[M] = a
    eng = _GroupedRecords(est)
    ex = lambda b: np.zeros_like(b)
    spread = A.bias_vs_M(eng, np.arange(64), [1, 4], ex)
    boot = A.bias_vs_M(eng, np.arange(64), [1, 4], ex, errors="bootstrap", n_boot=4000)
    jack = A.bias_vs_M(eng, np.arange(64), [1, 4], ex, errors="jackknife")
    for r_s, r_b, r_j in zip(spread, boot, jack):
        assert r_s[:3] == r_b[:3] == r_j[:3]                # same M, S and bias
        assert r_j[3] == pytest.approx(r_s[3], rel=1e-12)   # the jackknife error of a mean is the spread's
        assert r_b[3] == pytest.approx(r_s[3], rel=0.1)     # the bootstrap's approaches it
    with pytest.raises(ValueError):
        A.bias_vs_M(eng, np.arange(64), [1], ex, errors="median")
