"""Pins of the oracle's theta = infinity mode (Sec. V.B): the Metropolis sweeps
are replaced by simple sampling of the exact energy distribution
P_beta(E) = g(E) exp(-beta E) / Z(beta), with g from the transfer-matrix density
of states (itself pinned against enumeration and Kaufman's Z).

  - After every step the population is R_i independent draws from P_beta_i, so
    its energy histogram passes a chi^2 test against the exact distribution
    (from the density of states and, for the ferromagnet, from enumeration).
  - Given R_{i-1}, Q_i is the mean of exp(-dbeta E) over independent draws from
    P_beta_{i-1}, so E[Q_i] = Z(beta_i) / Z(beta_{i-1}) exactly and, by the tower
    property, E[prod_k Q_k] = Z(beta_i) / 2^N for every R; both are checked
    against Kaufman's finite-lattice Z.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O


def log_dos(L, model, seed=0, dis=0):
    Jr, Jd = O.couplings(L, model, seed, dis)
    g = O.dos_transfer(L, Jr, Jd)
    return np.array([math.log(c) if c else -math.inf for c in g]), g, (Jr, Jd)


def exact_levels(g, N, beta):
    """P_beta over u = (E + 2N)/2 (exact rational weights evaluated in floats)."""
    E = np.array([2 * u - 2 * N for u in range(2 * N + 1)], dtype=np.float64)
    lw = np.array([math.log(c) if c else -math.inf for c in g]) - beta * E
    p = np.exp(lw - lw.max())
    return p / p.sum()


def chi2_p(counts, probs):
    keep = probs * counts.sum() >= 5
    obs = np.append(counts[keep], counts[~keep].sum())
    exp = np.append(probs[keep], probs[~keep].sum()) * counts.sum()
    if exp[-1] == 0:
        obs, exp = obs[:-1], exp[:-1]
    return stats.chisquare(obs, exp * obs.sum() / exp.sum()).pvalue


@pytest.mark.parametrize("model", [0, 1])
def test_energies_are_exact_draws_at_every_temperature(model):
    L, N, R = 4, 16, 20000
    lg, g, (Jr, Jd) = log_dos(L, model, 0, 7)
    betas = [0.0, 0.2, 0.44, 0.8]
    o = O.OracleRun(L, model, R, R + 2000, O.THETA_INF, betas, 11, 0, 7, log_g=lg)
    for i, b in enumerate(betas):
        if i:
            assert o.step() == 0
        _, E, M, fam = o.population()
        assert np.all(M == 0) and np.all(np.diff(fam.astype(np.int64)) >= 0)
        counts = np.bincount((E + 2 * N) // 2, minlength=2 * N + 1).astype(np.float64)
        assert chi2_p(counts, exact_levels(g, N, b)) > 1e-4, (model, b)
        if model == 0:  # enumeration gives the same law over (E + 2N)/4
            pE = O.bruteforce(L, Jr, Jd, b)["pE"]
            c4 = np.bincount((E + 2 * N) // 4, minlength=N + 1).astype(np.float64)
            assert chi2_p(c4, pE) > 1e-4, b
        rec = o.record(i)
        assert rec["sumM2"] == 0 and rec["R"] == len(E)


def test_partition_function_ratios_are_unbiased():
    L, N, R, runs = 4, 16, 40, 400
    lg, _, _ = log_dos(L, 0)
    betas = [0.0, 0.15, 0.3, 0.45, 0.6]
    lnQ = np.zeros((runs, len(betas)))
    for r in range(runs):
        o = O.OracleRun(L, 0, R, 4 * R, O.THETA_INF, betas, 5, r, 0, log_g=lg)
        o.run_to_end()
        lnQ[r] = o.records()["lnQ"]
    lnZ = np.array([O.kaufman_lnZ(L, b) if b > 0 else N * math.log(2) for b in betas])
    for i in range(1, len(betas)):
        q = np.exp(lnQ[:, i])
        z = (q.mean() - math.exp(lnZ[i] - lnZ[i - 1])) / (q.std(ddof=1) / math.sqrt(runs))
        assert abs(z) < 4.5, (i, z)
    prod = np.exp(lnQ[:, 1:].sum(axis=1))
    z = (prod.mean() - math.exp(lnZ[-1] - N * math.log(2))) / (prod.std(ddof=1) / math.sqrt(runs))
    assert abs(z) < 4.5, z


def test_multinomial_keeps_R_and_records_stay_consistent():
    L, N, R = 6, 36, 3000
    lg, g, _ = log_dos(L, 0)
    betas = np.linspace(0, 0.5, 6)
    o = O.OracleRun(L, 0, R, R, O.THETA_INF, betas, 2, 1, 0, resample=1, log_g=lg)
    o.run_to_end()
    recs = o.records()
    assert np.all(recs["R"] == R)
    _, E, _, _ = o.population()
    counts = np.bincount((E + 2 * N) // 2, minlength=2 * N + 1).astype(np.float64)
    assert chi2_p(counts, exact_levels(g, N, betas[-1])) > 1e-4


def test_theta_inf_needs_a_density_of_states_and_no_overlaps():
    with pytest.raises(ValueError):
        O.OracleRun(4, 0, 10, 20, O.THETA_INF, [0.0, 0.1], 1, 0, 0)
    lg, _, _ = log_dos(4, 0)
    with pytest.raises(ValueError):
        O.OracleRun(4, 0, 10, 20, O.THETA_INF, [0.0, 0.1], 1, 0, 0, overlap=1, log_g=lg)
