"""Full-size parity on sampled outputs, in the launch configuration the
benchmark times (autotuned shapes, all runs in one engine).

Ising L=256, R=1e5, 16 runs, theta=20: the oracle cannot anneal a whole run,
so each part of a step is checked where it can be recomputed independently:
  - beta_0 spins of sampled replicas from the Philox keying (tag INIT);
  - every copy number of a step from the previous step's energies: level
    histogram, S summed in ascending levels with libm's exp, tau = R w / S and
    the nearest-integer draw from Philox (tag RESAMPLE); the children of each
    parent then form a contiguous block, which gives every child's parent;
  - sampled children: the oracle's theta sweeps of their parent's spins.
The uneven batch (4096 runs, L and R drawn by seed) is checked by running the
oracle on the smallest sampled runs in full.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2207_05535_gb300 import _lib
from paper_2207_05535_gb300 import workloads as W
from tests.helpers import compare_records, oracle_runs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2207_05535_gb300 import build
    build.build()
    _lib.load()


def init_spins(L, seed, run_id, j):
    N = L * L
    s = np.empty(N, dtype=np.int8)
    for c0 in range(N // 4):
        w = O.philox4x32_10([c0, j, 0, 1 << 24], [seed, run_id])
        for q in range(4):
            s[4 * c0 + q] = 1 if (int(w[q]) >> 31) else -1
    return s


def copy_numbers(E, N, R_target, dbeta, seed, run_id, step):
    """Nearest-integer copy numbers of Sec. II.B step (iii) (Eqs. tauBoltz, QBoltz)."""
    Emin = int(E.min())
    lev = (E.astype(np.int64) - Emin) // 4
    h = np.bincount(lev, minlength=N + 1)
    w = [math.exp(-(4.0 * n) * dbeta) for n in range(N + 1)]
    S = 0.0
    for n in range(N + 1):
        S = S + float(h[n]) * w[n]
    r = np.empty(len(E), dtype=np.int64)
    for j in range(len(E)):
        tau = (float(R_target) * w[lev[j]]) / S
        fl = math.floor(tau)
        u = int(O.philox4x32_10([j, 0, step, 3 << 24], [seed, run_id])[0])
        r[j] = fl + (1 if u * (1.0 / 4294967296.0) < tau - fl else 0)
    return r


def test_ising_L256_R1e5_full_size_sampled():
    descs = W.ising_L256_R1e5()
    for d in descs:
        d.betas = d.betas[:3]
    runs = (0, 9)
    kids = (0, 1, 4321, 55555)
    L, N = 256, 65536
    Jr, Jd = O.couplings(L, W.FERRO, 1, 0)
    with _lib.Engine(descs) as eng:
        E0 = {k: _lib.pa_population_slice(eng.h, k, 0, 200000, N, spins=False)[1] for k in runs}
        for k in runs:  # beta_0 draw of a few replicas, spins and energies
            s, E, M, fam, R, step = _lib.pa_population_slice(eng.h, k, 777, 1, N)
            ref = init_spins(L, descs[k].seed, descs[k].run_id, 777)
            assert np.array_equal(s[0], ref) and E[0] == O.energy(L, ref, Jr, Jd) and M[0] == int(ref.sum())
        eng.step(1)
        E1, fam1 = {}, {}
        for k in runs:
            _, E1[k], _, fam1[k], R1, step = _lib.pa_population_slice(eng.h, k, 0, 200000, N, spins=False)
            d = descs[k]
            r = copy_numbers(E0[k], N, d.R, d.betas[1] - d.betas[0], d.seed, d.run_id, 1)
            assert R1 == int(r.sum()) and step == 1
            assert np.array_equal(np.repeat(np.arange(len(r)), r), fam1[k])  # children contiguous, in parent order
        eng.step(1)
        kid2 = {}
        for k in runs:
            d = descs[k]
            _, E2, _, fam2, R2, _ = _lib.pa_population_slice(eng.h, k, 0, 200000, N, spins=False)
            r = copy_numbers(E1[k], N, d.R, d.betas[2] - d.betas[1], d.seed, d.run_id, 2)
            parent = np.repeat(np.arange(len(r)), r)
            assert R2 == len(parent) and np.array_equal(fam2, fam1[k][parent])
            kid2[k] = {}
            for j in kids:
                s, E, M, _, _, _ = _lib.pa_population_slice(eng.h, k, j, 1, N)
                kid2[k][j] = (int(parent[j]), s[0], int(E[0]), int(M[0]))
        eng.reset()   # the same anneal again, to read the step-1 parents
        eng.step(1)
        for k in runs:
            d = descs[k]
            for j, (p, s_child, E_child, M_child) in kid2[k].items():
                s_par = _lib.pa_population_slice(eng.h, k, p, 1, N)[0][0]
                s, E, M = O.sweep_lattice(L, s_par, Jr, Jd, d.betas[2], d.theta, d.seed, d.run_id, j, 2)
                assert np.array_equal(s, s_child) and E == E_child and M == M_child, (k, j)


def test_uneven_4096_full_size_sampled():
    descs = W.batched_uneven()
    for d in descs:
        d.betas = d.betas[:3]
    want = [(16, 1000), (32, 1000), (16, 10000)]
    idx = [next(m for m, d in enumerate(descs) if (d.L, d.R) == lr) for lr in want]
    ora = oracle_runs(descs, idx)
    with _lib.Engine(descs) as eng:
        eng.run_to_end()
        for k in idx:
            compare_records(eng.records(k), ora[k].records())
            s, E, M, fam, step = eng.population(k)
            os_, oE, oM, ofam = ora[k].population()
            assert np.array_equal(s, os_) and np.array_equal(E, oE) and np.array_equal(fam, ofam)
        recs = [eng.records(k) for k in range(0, len(descs), 97)]
    for rec in recs:  # every sampled run: sizes near the target, records complete
        assert np.all(rec["R"] > 0) and np.all(np.abs(rec["R"].astype(np.int64) - rec["R_target"]) <
                                               8 * np.sqrt(rec["R_target"]) + 64)
