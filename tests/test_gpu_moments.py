"""Parity of the higher-moment sums and of the central-moment and Binder
estimators (Sec. IV.E) where the sums need more than 64 bits.

A quench of the L = 256 ferromagnet to beta = 3 lowers |H| of every replica
past 2^16, so a single H^4 exceeds 2^64 and the 128-bit carry path of the
measurement is exercised; sum H^3 is negative, which exercises the sign.
"""
import numpy as np
import pytest

import oracle as O
from paper_2207_05535_gb300 import _lib
from paper_2207_05535_gb300 import workloads as W
from tests.helpers import compare_records, oracle_runs, wavg_close

pytestmark = pytest.mark.gpu

MOMENT_FIELDS = ("W_e3", "W_e4", "W_m3", "W_m4", "Wk3_e", "Wk4_e", "Wk3_m", "Wk4_m", "W_U4", "W_U4_conf")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2207_05535_gb300 import build
    build.build()
    _lib.load()


def test_moment_sums_beyond_64_bits_and_their_weighted_averages():
    betas = np.array([0.0, 3.0])
    descs = [W.RunDesc(256, W.FERRO, 24, 6, betas, seed=8, run_id=r) for r in range(2)]
    ora = oracle_runs(descs)
    orecs = np.stack([ora[k].records() for k in range(2)])
    last = orecs[:, -1]
    assert all(O.i128(w) > 1 << 64 for w in last["sumE4"]), "the case must overflow 64 bits"
    assert all(O.i128(w) < 0 for w in last["sumE3"])
    with _lib.Engine(descs) as eng:
        eng.run_to_end()
        for k in range(2):
            compare_records(eng.records(k), orecs[k])
        g = eng.weighted_average(np.arange(2, dtype=np.uint32), 2, 0)
    o, _, _ = O.weighted_average(orecs, 256 * 256, 0)
    wavg_close(g[0], o, _lib.WAVG_DTYPE.names, 256 * 256)
    h, _, _ = _lib.pa_weighted_average(orecs, 256 * 256, 1)
    o1, _, _ = O.weighted_average(orecs, 256 * 256, 1)
    wavg_close(h, o1, MOMENT_FIELDS, 256 * 256)


@pytest.mark.parametrize("kind", [0, 1])
def test_central_moments_and_binder_over_many_ferromagnet_runs(kind):
    descs = W.ferro_runs(L=8, R=300, theta=3, beta_f=0.5, n=11, M=12, seed=4)
    ora = oracle_runs(descs)
    orecs = np.stack([ora[k].records() for k in range(len(descs))])
    with _lib.Engine(descs) as eng:
        eng.run_to_end()
        g = eng.weighted_average(np.arange(len(descs), dtype=np.uint32), 4, kind)
    for grp in range(3):
        o, _, _ = O.weighted_average(orecs[4 * grp:4 * grp + 4], 64, kind)
        wavg_close(g[grp], o, MOMENT_FIELDS, 64)
