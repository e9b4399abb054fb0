"""Pins of the oracle's free-energy weight at fluctuating population sizes and
of its multinomial member pick.

Eq. appropriateWeight (Sec. IV.A) multiplies R_i exp(-beta_i F_i) by the
product of R_{k-1}/R over the steps k <= i, the estimate of how much larger an
unnormalised (uPA) population would have grown than the PA population.  With
nearest-integer resampling R_i fluctuates, so this factor is not 1; three
independent facts pin it:
  - when every normalisation of a run is exactly 1 (R_{k-1} Q_k = R), the run
    is an unnormalised population, and Eq. weighted_uPA fixes the weights to
    R_i / sum R_i (a deterministic identity that every plausible slip in the
    factor breaks);
  - the unnormalised weight R_i prod_k (R_{k-1} Q_k / R) has the exact
    expectation Z(beta_i) / 2^N for any R (the resampling is conditionally
    unbiased, Sec. II.B), checked against enumeration at L = 4;
  - the weighted averages over many small runs approach the exact energy and
    free energy (Sec. IV.A, Eq. W_F).
Multinomial resampling (Sec. IV.C; condition (c) of Sec. IV.D) draws a level
and then a member of that level uniformly; the member pick is pinned by a
chi-square over the members of every populated level.

Each pin is also applied to what a mistaken oracle would output (a dropped or
misindexed factor, a biased member pick), computed here from the oracle's own
records, to show that the pin fails for it.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2207_05535_gb300 import workloads as W

N4 = 16  # spins at L = 4


# --------------------------------------------------------------------------- helpers
def _mistaken_log_weights(recs):
    """Log weights [variant][i, m] of plausible slips in Eq. appropriateWeight."""
    R = recs["R"].astype(np.float64)               # [m, i]
    Rt = recs["R_target"].astype(np.float64)
    F = recs["minus_betaF"]
    with np.errstate(divide="ignore"):
        lr = np.log(R)
        ratio = np.log(R / Rt)                     # ln(R_k / R) at k
    prev = np.concatenate([np.zeros((R.shape[0], 1)), np.cumsum(ratio, axis=1)[:, :-1]], axis=1)  # k <= i-1
    upto = np.cumsum(ratio, axis=1)                                                               # k <= i
    return {
        "factor dropped (simplified weight)": (lr + F).T,
        "R_k for R_{k-1}": (lr + F + upto).T,
        "R_i counted twice": (2 * lr + F + prev).T,
        "factor with the wrong sign": (lr + F - prev).T,
        "ln R_i dropped": (F + prev).T,
    }


def _normalise(lam):
    w = np.exp(lam - lam.max(axis=1, keepdims=True))
    return w / w.sum(axis=1, keepdims=True)


def _upa_records(M=6, n=7, R=10, seed=3):
    """Records of runs whose every normalisation is exactly 1: R_{k-1} Q_k = R."""
    rng = np.random.default_rng(seed)
    recs = np.zeros((M, n), dtype=O.RECORD_DTYPE)
    Rs = rng.integers(4, 19, size=(M, n))
    Rs[:, 0] = R
    recs["R"] = Rs
    recs["R_target"] = R
    recs["N"] = N4
    recs["beta"] = np.linspace(0.0, 0.6, n)
    lnQ = np.zeros((M, n))
    lnQ[:, 1:] = np.log(R / Rs[:, :-1])
    recs["lnQ"] = lnQ
    recs["minus_betaF"] = N4 * math.log(2.0) + np.cumsum(lnQ, axis=1)
    recs["sumE"] = rng.integers(-32, 33, size=(M, n)) * Rs   # e = sumE / (N R_i) in [-2, 2]
    recs["sumE2"] = recs["sumE"] ** 2 // np.maximum(Rs, 1)
    return recs


# --------------------------------------------------------------------------- Eq. weighted_uPA
def test_full_weight_equals_upa_weight_when_every_normalisation_is_one():
    """A run with R_{k-1} Q_k = R at every step grew exactly as an unnormalised
    population: Eq. weighted_uPA weights it by R_i / sum_m R_i, so the weights of
    Eq. appropriateWeight must equal that.  W[Q_k] (Eq. W_F) is then the growth
    M R / sum_m R_{k-1} of the combined population."""
    recs = _upa_records()
    M, n = recs.shape
    R = recs["R"].astype(np.float64)
    out, _, _, w = O.weighted_average(recs, N4, 0, return_weights=True)
    upa = (R / R.sum(axis=0)).T                                   # [i, m]
    assert np.allclose(w, upa, rtol=1e-13, atol=0)
    e = recs["sumE"] / (N4 * R)
    assert np.allclose(out["W_e"], (upa.T * e).sum(axis=0), rtol=1e-13, atol=1e-15)
    growth = np.log(M * 10 / R[:, :-1].sum(axis=0))               # ln W[Q_k], k = 1..n-1
    expect_F = N4 * math.log(2.0) + np.concatenate([[0.0], np.cumsum(growth)])
    assert np.allclose(out["W_minus_betaF"], expect_F, rtol=1e-13, atol=1e-13)
    # every plausible slip in the factor gives other weights (so this pin catches it)
    for name, lam in _mistaken_log_weights(recs).items():
        assert np.abs(_normalise(lam)[1:] - upa[1:]).max() > 1e-2, name


# --------------------------------------------------------------------------- exact expectation
def _small_runs(R, betas, theta, M, seed, run0=0, resample=0):
    """M oracle runs at L = 4 (ferromagnet); a run that dies out keeps R_i = 0 afterwards."""
    recs = np.zeros((M, len(betas)), dtype=O.RECORD_DTYPE)
    cap = R if resample else 8 * R + 64
    for m in range(M):
        r = O.OracleRun(4, 0, R, cap, theta, betas, seed, run0 + m, 0, resample)
        while r.cur_step + 1 < len(betas):
            if r.step():
                break
        got = r.records()
        recs[m, :len(got)] = got
    recs["R_target"] = R
    recs["N"] = N4
    return recs


def test_unnormalised_full_weight_is_unbiased_for_the_partition_function():
    """E[R_i prod_{k<=i} (R_{k-1} Q_k / R)] = R Z(beta_i) / 2^N exactly for any R
    (conditionally unbiased resampling, Sec. II.B; uPA argument of Sec. IV.A).
    exp(lambda) of the oracle's weight is 2^N times that quantity, so its mean
    over runs must be R Z(beta_i).  Small R = 3 makes R_i fluctuate by ~25 %."""
    R, M = 3, 20000
    betas = [0.0, 0.15, 0.3]
    recs = _small_runs(R, betas, 1, M, seed=11)
    lam = O.log_weights(recs, 0)
    Jr, Jd = O.couplings(4, 0, 1, 0)

    def zscores(lam_):
        z = []
        for i in (1, 2):
            y = np.exp(lam_[i] - (math.log(R) + O.bruteforce(4, Jr, Jd, betas[i])["lnZ"]))
            z.append((y.mean() - 1.0) / (y.std() / math.sqrt(M)))
        return np.array(z)

    assert np.all(np.abs(zscores(lam)) < 4.5), zscores(lam)
    bad = _mistaken_log_weights(recs)
    for name in ("R_k for R_{k-1}", "R_i counted twice", "ln R_i dropped"):
        assert np.abs(zscores(bad[name])).max() > 6, name


# --------------------------------------------------------------------------- large M
@pytest.mark.slow
def test_weighted_averages_with_fluctuating_populations_approach_exact_values():
    """Many small nearest-integer runs (R = 5, so R_i fluctuates by ~18 %): the
    weighted energy W[e] (Eq. W_conf) and -beta W[F] (Eq. W_F) over all of them
    approach the exact values at L = 4 (a large M acts like a large R, Eq.
    weighted_uPA), within their statistical error (jackknife over 20 blocks)."""
    R, M = 5, 16000
    betas = list(W.schedule(0.4, 9))
    recs = _small_runs(R, betas, 1, M, seed=21)
    assert recs["R"].min() > 0  # no run died out (its later records would have no estimator)
    assert recs["R"][:, 1:].std() > 0.15 * R
    Jr, Jd = O.couplings(4, 0, 1, 0)
    full, _, _ = O.weighted_average(recs, N4, 0)
    blocks = np.array_split(np.arange(M), 20)
    jack = [O.weighted_average(np.delete(recs, b, axis=0), N4, 0)[0] for b in blocks]
    for i in (2, 5, 8):
        ex = O.bruteforce(4, Jr, Jd, betas[i])
        for key, exact in (("W_e", ex["e"]), ("W_minus_betaF", ex["lnZ"])):
            vals = np.array([j[key][i] for j in jack])
            sigma = math.sqrt((len(vals) - 1) * vals.var())
            assert abs(full[key][i] - exact) < 4 * sigma + 1e-3 * abs(exact), (key, i, full[key][i], exact, sigma)


# --------------------------------------------------------------------------- multinomial member pick
def _member_pick_zscores(steps):
    """z-scores of the copies within every populated level against a uniform
    pick among its members (members in replica order), summed over levels:
    the Pearson chi-square, the copies of each level's first member and the
    copies of its last member (where an off-by-one in the index lands)."""
    X = mean = var = 0.0
    edge = {"first": [0.0, 0.0, 0.0], "last": [0.0, 0.0, 0.0]}  # observed, expected, variance
    for E, r in steps:
        levels = (E - E.min()) // 4
        for n in np.unique(levels):
            idx = np.flatnonzero(levels == n)
            h, T = len(idx), int(r[idx].sum())
            if h < 2 or T == 0:
                continue
            X += float((((r[idx] - T / h) ** 2) / (T / h)).sum())
            mean += h - 1
            var += 2 * (h - 1) * (1 - 1 / T)
            for key, j in (("first", idx[0]), ("last", idx[-1])):
                edge[key][0] += r[j]
                edge[key][1] += T / h
                edge[key][2] += T / h * (1 - 1 / h)
    z = {"chi2": (X - mean) / math.sqrt(var)}
    for key, (o, e, v) in edge.items():
        z[key] = (o - e) / math.sqrt(v)
    return z


def test_multinomial_member_pick_is_uniform_within_each_level():
    """Multinomial resampling draws a level with probability proportional to its
    weight and then one of its members uniformly (Sec. IV.C; E[r_j] = tau_j,
    condition (c) of Sec. IV.D): given a level's copies T, the member counts are
    Multinomial(T, 1/h).  The chi-square over every level's members stays at its
    mean; a first-member pick or a pick that never reaches the last member fails."""
    R = 300
    steps = []
    for run_id in range(6):
        run = O.OracleRun(6, 1, R, R, 1, W.schedule(1.2, 9), 4, run_id, 2, resample=1)
        for i in range(1, 9):
            _, E, _, _ = run.population()
            assert run.step() == 0
            steps.append((E.astype(np.int64), run.counts(R).astype(np.int64)))
    z = _member_pick_zscores(steps)
    assert all(abs(v) < 5 for v in z.values()), z

    # what a mistaken pick would output from the same level totals
    rng = np.random.default_rng(0)
    first, not_last = [], []
    for E, r in steps:
        levels = (E - E.min()) // 4
        f = np.zeros_like(r)
        q = np.zeros_like(r)
        for n in np.unique(levels):
            idx = np.flatnonzero(levels == n)
            T = int(r[idx].sum())
            f[idx[0]] = T
            pool = idx[:-1] if len(idx) > 1 else idx
            np.add.at(q, rng.choice(pool, size=T), 1)
        first.append((E, f))
        not_last.append((E, q))
    for bad in (first, not_last):
        zb = _member_pick_zscores(bad)
        assert max(abs(v) for v in zb.values()) > 8, zb
