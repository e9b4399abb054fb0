"""Pins of the oracle's higher moments, central-moment estimators W_k and the
Binder cumulant (Sec. IV.E) against closed forms, a second exact method and
the binomial theorem.

  - Infinite temperature: e = -(1/N) sum_b J_b sigma_b over the B = 2N bonds,
    whose products sigma_b are uniform +-1 and independent except around closed
    loops.  Hence <E> = <E^3> = 0 and <E^4> = 3B^2 - 2B + 24 sum_{4-loops} prod J
    (ordered 4-tuples of paired bonds, plus 4! orderings of each 4-bond loop:
    the N plaquettes, and at L = 4 also the 2L straight loops around the torus).
    M is a sum of N independent +-1: <M^2> = N, <M^4> = 3N^2 - 2N, and <|M|^k>
    is a binomial sum.
  - Finite temperature: the energy moments of brute-force enumeration equal
    those of the transfer-matrix density of states; deep in the ordered phase
    |m| -> 1 and e -> -2.
  - One run (M = 1): the weight is 1 and W_k must equal the population's
    central moment (1/R) sum_j (o_j - mean)^k, computed here in exact rational
    arithmetic from the population itself (two passes, no binomial expansion).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2207_05535_gb300 import workloads as W


def _loops4(L, Jr, Jd):
    """Sum over the 4-bond closed loops of the product of their couplings."""
    J = lambda a, x, y: int(a[(y % L) * L + (x % L)])
    s = 0
    for y in range(L):
        for x in range(L):  # plaquette with corner (x, y)
            s += J(Jr, x, y) * J(Jd, x + 1, y) * J(Jr, x, y + 1) * J(Jd, x, y)
    if L == 4:  # straight loops around the torus
        for y in range(L):
            s += math.prod(J(Jr, x, y) for x in range(L))
        for x in range(L):
            s += math.prod(J(Jd, x, y) for y in range(L))
    return s


def _absm_moment(N, k):
    return Fraction(sum(math.comb(N, n) * abs(N - 2 * n) ** k for n in range(N + 1)), 2 ** N * N ** k)


def _beta0_moments(L, Jr, Jd):
    N, B = L * L, 2 * L * L
    e = [Fraction(0), Fraction(B, N * N), Fraction(0), Fraction(3 * B * B - 2 * B + 24 * _loops4(L, Jr, Jd), N ** 4)]
    m = [_absm_moment(N, k) for k in (1, 2, 3, 4)]
    return e, m


@pytest.mark.parametrize("model,dis", [(0, 0), (1, 3), (1, 11)])
def test_bruteforce_moments_at_infinite_temperature(model, dis):
    Jr, Jd = O.couplings(4, model, 9, dis)
    e, m = O.bruteforce_moments(4, Jr, Jd, 0.0)
    ee, mm = _beta0_moments(4, Jr, Jd)
    assert m[1] == pytest.approx(1 / 16, rel=1e-14) and m[3] == pytest.approx((3 * 256 - 32) / 16 ** 4, rel=1e-14)
    for k in range(4):
        assert e[k] == pytest.approx(float(ee[k]), rel=1e-13, abs=1e-15), ("e", k + 1)
        assert m[k] == pytest.approx(float(mm[k]), rel=1e-13), ("m", k + 1)


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("beta", [0.2, 0.4407, 1.0])
def test_bruteforce_energy_moments_equal_transfer_matrix(model, beta):
    L, N = 4, 16
    Jr, Jd = O.couplings(L, model, 9, 5)
    e, _ = O.bruteforce_moments(L, Jr, Jd, beta)
    g = O.dos_transfer(L, Jr, Jd)
    Es = [2 * t - 2 * N for t in range(2 * N + 1)]
    Emin = min(E for E, c in zip(Es, g) if c)
    wts = [c * math.exp(-beta * (E - Emin)) for E, c in zip(Es, g)]
    Z = math.fsum(wts)
    for k in range(1, 5):
        ref = math.fsum(w * (E / N) ** k for w, E in zip(wts, Es)) / Z
        assert e[k - 1] == pytest.approx(ref, rel=1e-12, abs=1e-14), k


def test_bruteforce_moments_ordered_limit():
    Jr, Jd = O.couplings(4, 0, 0, 0)
    e, m = O.bruteforce_moments(4, Jr, Jd, 8.0)
    for k in range(4):
        assert m[k] == pytest.approx(1.0, abs=1e-9)
        assert e[k] == pytest.approx((-2.0) ** (k + 1), abs=1e-9)


def _i128s(recs, f):
    return np.array([O.i128(w) for w in recs[f]], dtype=object)


@pytest.mark.parametrize("L,model", [(4, 0), (6, 0), (6, 1)])
def test_record_sums_at_infinite_temperature(L, model):
    """Step-0 records of independent runs: per-replica means of E^3, E^4,
    |M|^3 and M^4 agree with the closed forms (z-test over the runs), and the
    weighted Binder cumulant equals 2/(3N) within its error."""
    N, R, runs = L * L, 8000, 12
    recs = []
    for r in range(runs):
        o = O.OracleRun(L, model, R, R + 1000, 1, [0.0], 21, r, 4)
        recs.append(o.records())
    Jr, Jd = O.couplings(L, model, 21, 4)
    ee, mm = _beta0_moments(L, Jr, Jd)
    targets = {"sumE3": ee[2] * N ** 3, "sumE4": ee[3] * N ** 4, "sumAbsM3": mm[2] * N ** 3,
               "sumM4": mm[3] * N ** 4}
    for f, t in targets.items():
        per_run = np.array([float(O.i128(rc[f][0])) / R for rc in recs])
        se = per_run.std(ddof=1) / math.sqrt(runs)
        z = (per_run.mean() - float(t)) / se
        assert abs(z) < 5, (f, per_run.mean(), float(t), z)
    # the 128-bit sums agree with the 64-bit ones where both are defined
    for rc in recs:
        assert O.i128(rc["sumM4"][0]) >= O.i128(rc["sumAbsM3"][0]) >= rc["sumAbsM"][0] >= 0
    wa, _, _ = O.weighted_average(np.stack(recs), N, 0)
    u4 = np.array([O.weighted_average(rc[None], N, 0)[0]["W_U4"][0] for rc in recs])
    assert abs(wa["W_U4"][0] - 2 / (3 * N)) < 5 * u4.std(ddof=1) / math.sqrt(runs) + 1e-3


def _central(vals, k):
    mean = sum(vals) / len(vals)
    return sum((v - mean) ** k for v in vals) / len(vals)


@pytest.mark.parametrize("model,beta_f", [(0, 0.42), (1, 1.2)])
def test_single_run_central_moments_are_the_population_moments(model, beta_f):
    L, R = 8, 700
    N = L * L
    o = O.OracleRun(L, model, R, 2 * R, 3, W.schedule(beta_f, 6), 5, 2, 1)
    o.run_to_end()
    rec = o.records()
    _, E, M, _ = o.population()
    e = [Fraction(int(x), N) for x in E]
    am = [Fraction(abs(int(x)), N) for x in M]
    wa, _, _ = O.weighted_average(rec[None], N, 0)
    last = wa[-1]
    assert last["sum_w"] == 1.0
    for key, vals in (("e", e), ("m", am)):
        raw = [float(sum(v ** l for v in vals) / len(vals)) for l in range(5)]
        for k in (3, 4):
            exact = float(_central(vals, k))
            cond = sum(math.comb(k, l) * abs(raw[1]) ** (k - l) * abs(raw[l]) for l in range(k + 1))
            got = last[f"Wk{k}_{key}"]
            assert abs(got - exact) <= 64 * 2.0 ** -52 * cond, (key, k, got, exact)
    mp2 = sum(Fraction(int(x) ** 2, N * N) for x in M) / len(M)
    mp4 = sum(Fraction(int(x) ** 4, N ** 4) for x in M) / len(M)
    u4 = float(1 - mp4 / (3 * mp2 * mp2))
    assert last["W_U4"] == pytest.approx(u4, rel=1e-13, abs=1e-15)
    assert last["W_U4_conf"] == pytest.approx(u4, rel=1e-13, abs=1e-15)
    for f, p in (("W_e3", 3), ("W_e4", 4)):
        assert last[f] == pytest.approx(float(sum(v ** p for v in e) / len(e)), rel=1e-14)
    for f, p in (("W_m3", 3), ("W_m4", 4)):
        assert last[f] == pytest.approx(float(sum(v ** p for v in am) / len(am)), rel=1e-14)


@pytest.mark.slow
def test_weighted_central_moments_and_binder_match_exact_L4():
    """Whole method: 16 ferromagnet runs at L = 4 annealed to beta = 0.6; the
    weighted fourth central moment of e, W[e^4], W[m^4] and the Binder cumulant
    agree with enumeration within five standard errors of the runs."""
    L, N, R, M = 4, 16, 1500, 16
    betas = W.schedule(0.6, 13)
    Jr, Jd = O.couplings(L, 0, 0, 0)
    e, m = O.bruteforce_moments(L, Jr, Jd, betas[-1])
    k4 = e[3] - 4 * e[0] * e[2] + 6 * e[0] ** 2 * e[1] - 3 * e[0] ** 4
    u4 = 1 - m[3] / (3 * m[1] ** 2)
    recs = []
    for r in range(M):
        o = O.OracleRun(L, 0, R, 2 * R, 5, betas, 3, r, 0)
        o.run_to_end()
        recs.append(o.records())
    recs = np.stack(recs)
    wa, _, _ = O.weighted_average(recs, N, 0)
    single = np.stack([O.weighted_average(recs[k][None], N, 0)[0][-1] for k in range(M)])
    for f, exact in (("Wk4_e", k4), ("W_e4", e[3]), ("W_m4", m[3]), ("W_U4", u4), ("W_m3", m[2]), ("W_e3", e[2])):
        se = single[f].std(ddof=1) / math.sqrt(M)
        assert abs(wa[f][-1] - exact) < 5 * se + 2.0 / R * abs(exact), (f, wa[f][-1], exact, se)
