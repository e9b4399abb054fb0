"""Analysis of weighted averages over many PA runs (Sec. V.B-V.D).

The weighted averages themselves run on the GPU (pa_weighted_average_runs
over records resident in an engine); this module partitions runs into groups
of M, compares the group estimates with exact values, and provides the
paper's statistics:
  - exact 2D Ising ferromagnet values on the periodic L x L lattice from
    Kaufman's finite-lattice partition function (Sec. V.A.3 names it as the
    exact reference): ln Z, e, c, f = -ln Z / (beta N);
  - bias of a weighted estimator as a function of M (Sec. V.B.3: runs are
    partitioned into S = floor(n / M) groups of M, the group estimates are
    averaged);
  - least-squares fits of a M^-b to bias data with jackknife errors
    (Table III), and bootstrap errors, which the paper uses for the
    ferromagnet's bias (Sec. V.B.3);
  - the root-mean-square deviation RMSD = sqrt(bias^2 + variance) (Eq. RMSD);
  - the predicted variance of free-energy weights
    var w ~ (exp(var beta F) - 1) / M^2 (Eq. varWpred).
"""
from __future__ import annotations

import math

import numpy as np

from . import _lib

LD = np.longdouble


# --------------------------------------------------------------------------- exact ferromagnet
def kaufman_lnZ(L: int, beta) -> np.ndarray:
    """ln Z of the periodic L x L Ising ferromagnet (J = 1) at inverse temperature(s) beta.

    Z = 1/2 (2 sinh 2K)^(N/2) (Z1 + Z2 + Z3 + Z4) with
    Z1 = prod_r 2 cosh(L g_{2r+1} / 2), Z2 = prod_r 2 sinh(L g_{2r+1} / 2),
    Z3 = prod_r 2 cosh(L g_{2r} / 2),   Z4 = prod_r 2 sinh(L g_{2r} / 2), r = 0..L-1,
    cosh g_k = cosh 2K coth 2K - cos(pi k / L) (k >= 1), g_0 = 2K + ln tanh K.
    Evaluated in long double with signed logarithms."""
    betas = np.atleast_1d(np.asarray(beta, dtype=np.float64))
    out = np.empty(len(betas))
    k = np.arange(2 * L, dtype=LD)
    for n, b in enumerate(betas):
        if b == 0.0:  # Z(0) = 2^N
            out[n] = L * L * math.log(2.0)
            continue
        K = LD(b)
        c2 = np.cosh(2 * K) / np.tanh(2 * K)
        g = np.arccosh(c2 - np.cos(LD(np.pi) * k / LD(L)))
        g[0] = 2 * K + np.log(np.tanh(K))
        go, ge = g[1::2], g[0::2]
        l1 = np.sum(np.log(2 * np.cosh(L * go / 2)))
        l2 = np.sum(np.log(2 * np.sinh(L * go / 2)))
        l3 = np.sum(np.log(2 * np.cosh(L * ge / 2)))
        s4 = 2 * np.sinh(L * ge / 2)
        sign4 = np.prod(np.sign(s4))
        l4 = np.sum(np.log(np.abs(s4)))
        top = max(l1, l2, l3, l4)
        total = np.exp(l1 - top) + np.exp(l2 - top) + np.exp(l3 - top) + sign4 * np.exp(l4 - top)
        out[n] = float(-np.log(LD(2)) + LD(L * L) / 2 * np.log(2 * np.sinh(2 * K)) + top + np.log(total))
    return out


def exact_ferro(L: int, betas, h: float = 1e-4) -> dict:
    """Exact e, c, f per spin and ln Z at the given inverse temperatures
    (e = -d ln Z / d beta / N, c = beta^2 d^2 ln Z / d beta^2 / N by central
    differences of Kaufman's ln Z)."""
    b = np.asarray(betas, dtype=np.float64)
    N = L * L
    lz = kaufman_lnZ(L, b)
    lp, lm = kaufman_lnZ(L, b + h), kaufman_lnZ(L, np.maximum(b - h, 0.0))
    hm = np.where(b - h < 0, b, h)  # shorter lower step near beta = 0
    with np.errstate(divide="ignore", invalid="ignore"):
        e = np.where(b > 0, -(lp - lm) / (h + hm) / N, 0.0)          # <H>_0 = 0 at infinite temperature
        c = np.where(b > 0, b * b * 2 * (hm * lp - (h + hm) * lz + h * lm) / (h * hm * (h + hm)) / N, 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(b > 0, -lz / (b * N), np.nan)
    return {"beta": b, "lnZ": lz, "e": e, "c": c, "f": f}


# --------------------------------------------------------------------------- statistics
def jackknife(values, stat=np.mean):
    """Jackknife estimate and standard error of stat over the first axis."""
    v = np.asarray(values)
    n = len(v)
    if n < 2:
        return float(stat(v)), float("nan")
    loo = np.array([stat(np.delete(v, i, axis=0)) for i in range(n)])
    full = stat(v)
    err = math.sqrt((n - 1) / n * float(np.sum((loo - loo.mean(axis=0)) ** 2)))
    return float(full), err


def bootstrap(values, stat=np.mean, n_boot=2000, seed=0):
    """Bootstrap estimate and standard error of stat over the first axis: stat
    of the full sample, and the standard deviation of stat over n_boot
    resamples drawn with replacement (seeded, so the error is reproducible)."""
    v = np.asarray(values)
    n = len(v)
    if n < 2:
        return float(stat(v)), float("nan")
    rng = np.random.default_rng(seed)
    reps = np.array([stat(v[rng.integers(0, n, size=n)]) for _ in range(n_boot)])
    return float(stat(v)), float(np.std(reps, ddof=1))


def fit_power_law(M, bias, sigma=None):
    """Least-squares fit of |bias| = a M^-b on log-log axes (weights 1/sigma_log^2).
    Returns (a, b, sigma_b) with the standard fit error of b."""
    M = np.asarray(M, dtype=np.float64)
    y = np.log(np.abs(np.asarray(bias, dtype=np.float64)))
    x = np.log(M)
    if sigma is None:
        w = np.ones_like(y)
    else:
        s = np.asarray(sigma, dtype=np.float64) / np.abs(np.asarray(bias, dtype=np.float64))
        w = 1.0 / np.maximum(s, 1e-300) ** 2
    A = np.vstack([np.ones_like(x), -x]).T
    Aw = A * w[:, None]
    cov = np.linalg.inv(A.T @ Aw)
    coef = cov @ (Aw.T @ y)
    if sigma is None:  # scale by the residual variance
        res = y - A @ coef
        dof = max(1, len(y) - 2)
        cov = cov * float(res @ res) / dof
    return float(math.exp(coef[0])), float(coef[1]), float(math.sqrt(cov[1, 1]))


def rmsd(estimates, exact):
    """Eq. RMSD: sqrt(bias^2 + variance) of estimates (first axis: samples)."""
    est = np.asarray(estimates, dtype=np.float64)
    bias = est.mean(axis=0) - exact
    return np.sqrt(bias ** 2 + est.var(axis=0))


def varw_prediction(minus_betaF, M):
    """Eq. varWpred: var w ~ (exp(var[beta F]) - 1) / M^2 from a sample of -beta F values."""
    v = float(np.var(np.asarray(minus_betaF, dtype=np.float64)))
    return (math.exp(v) - 1.0) / (M * M)


# --------------------------------------------------------------------------- weighted estimators over groups
OBSERVABLES = ("W_e", "W_e2", "W_m", "W_m2", "Wvar_c", "Wvar_chi", "W_c", "W_chi", "W_minus_betaF")


def grouped_estimates(engine, runs, M, kind=0):
    """Weighted averages of every group of M consecutive runs (S = floor(len/M)
    groups), computed on the GPU from the engine's resident records.
    Returns a structured array [S][n_beta] (pa_wavg)."""
    runs = np.asarray(runs, dtype=np.uint32)
    S = len(runs) // M
    if S == 0:
        raise ValueError("fewer runs than M")
    return engine.weighted_average(runs[:S * M], M, kind)


def bias_vs_M(engine, runs, Ms, exact_fn, obs="W_e", kind=0, steps=None, relative=False, errors="spread",
              n_boot=2000, seed=0):
    """Bias of a weighted estimator for each M: mean over the S groups of the
    group estimate minus the exact value, averaged in absolute value over the
    selected temperature indices.  exact_fn(beta array) -> exact values.
    Returns rows (M, S, bias, stderr); stderr is the standard error of the
    signed bias averaged over the groups and temperatures: "spread", from the
    spread of the groups' temperature-averaged biases; "bootstrap", over
    resamples of the S groups (with replacement); "jackknife", over the S groups
    left out one at a time (equal to the spread's for this mean)."""
    if errors not in ("spread", "bootstrap", "jackknife"):
        raise ValueError("errors: spread, bootstrap or jackknife")
    rows = []
    for M in Ms:
        est = grouped_estimates(engine, runs, M, kind)
        beta = est["beta"][0]
        sel = np.arange(len(beta)) if steps is None else np.asarray(steps)
        ex = np.asarray(exact_fn(beta[sel]), dtype=np.float64)
        vals = est[obs][:, sel].astype(np.float64)
        diff = vals - ex[None, :]
        if relative:
            diff = diff / np.abs(ex)[None, :]
        per_group = np.mean(diff, axis=1)            # bias of one group, averaged over the temperatures
        b = np.mean(np.abs(np.mean(diff, axis=0)))   # |mean bias| per temperature, averaged
        stat = lambda d: float(np.mean(d))
        if errors == "bootstrap":
            se = bootstrap(diff, stat, n_boot=n_boot, seed=seed)[1]
        elif errors == "jackknife":
            se = jackknife(diff, stat)[1]
        else:
            se = float(np.std(per_group, ddof=1) / math.sqrt(len(per_group))) if len(per_group) > 1 else float("nan")
        rows.append((int(M), int(len(per_group)), float(b), float(se)))
    return rows


# --------------------------------------------------------------------------- command line
def main(argv=None):
    """Bias of weighted estimators versus M for a batch of ferromagnet runs:

        python -m paper_2207_05535_gb300.analysis --L 8 --R 500 --theta 2 --runs 4096 --beta-f 0.5 --temps 51
    """
    import argparse
    import json
    import time

    from . import build
    from . import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=8)
    ap.add_argument("--R", type=int, default=500)
    ap.add_argument("--theta", type=int, default=2)
    ap.add_argument("--runs", type=int, default=4096)
    ap.add_argument("--beta-f", type=float, default=0.5)
    ap.add_argument("--temps", type=int, default=51)
    ap.add_argument("--Ms", default="1,2,4,8,16,32,64,128")
    ap.add_argument("--window", default="0.42,0.46", help="beta range the bias is averaged over")
    ap.add_argument("--errors", default="bootstrap", choices=["bootstrap", "jackknife", "spread"],
                    help="standard error of the bias (the paper uses the bootstrap for the ferromagnet)")
    ap.add_argument("--fit-min-snr", type=float, default=2.0,
                    help="fit a M^-b only to the M whose bias exceeds this many standard errors (the rest is the "
                         "statistical floor of all runs together)")
    a = ap.parse_args(argv)
    build.build()
    descs = W.ferro_runs(L=a.L, R=a.R, theta=a.theta, beta_f=a.beta_f, n=a.temps, M=a.runs, seed=1)
    t0 = time.perf_counter()
    eng = _lib.Engine(descs)
    eng.run_to_end()
    t_anneal = time.perf_counter() - t0
    beta = descs[0].betas
    lo, hi = (float(x) for x in a.window.split(","))
    steps = np.nonzero((beta >= lo - 1e-12) & (beta <= hi + 1e-12))[0]
    if len(steps) == 0:
        steps = np.array([len(beta) - 1])
    Ms = [int(x) for x in a.Ms.split(",") if int(x) <= a.runs]
    runs = np.arange(a.runs)
    t1 = time.perf_counter()
    out = {}
    for obs, key, rel in (("W_e", "e", False), ("Wvar_c", "c", True), ("W_minus_betaF", "lnZ", False)):
        rows = bias_vs_M(eng, runs, Ms, lambda b, k=key: exact_ferro(a.L, b)[k], obs=obs, steps=steps,
                         relative=rel, errors=a.errors)
        use = [r for r in rows if r[2] > a.fit_min_snr * r[3]]
        fit = fit_power_law([r[0] for r in use], [r[2] for r in use], [r[3] for r in use]) if len(use) >= 3 else None
        out[obs] = {"rows": rows, "fit_a_b_sigma": fit, "fit_M": [r[0] for r in use]}
    t_an = time.perf_counter() - t1
    recs = np.stack([eng.records(k) for k in range(min(a.runs, 4096))])
    i_last = len(beta) - 1
    vw = varw_prediction(recs[:, i_last]["minus_betaF"], 16)
    eng.close()
    print(json.dumps({"config": vars(a), "beta_steps": [float(beta[s]) for s in steps], "bias": out,
                      "varw_pred_M16_last_beta": vw, "anneal_s": t_anneal, "analysis_s": t_an}))


if __name__ == "__main__":
    main()
