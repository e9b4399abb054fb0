"""Test helpers: run the oracle on the same descriptors the engine gets."""
import numpy as np

import oracle as O


def oracle_runs(descs, idx=None):
    """Run the oracle for descs[k], k in idx (default all), to the end; paired
    populations are stepped in lockstep and their two-population overlaps
    measured at every temperature.  Returns {k: OracleRun}."""
    idx = list(range(len(descs))) if idx is None else list(idx)
    want = set(idx)
    for k in idx:
        if descs[k].overlap & 2 and descs[k].paired >= 0:
            want.add(descs[k].paired)
    runs = {k: O.OracleRun.from_desc(descs[k]) for k in sorted(want)}

    def pair_measure():
        for k, r in runs.items():
            p = descs[k].paired
            if descs[k].overlap & 2 and p > k and p in runs:
                r.measure_pair(runs[p])

    pair_measure()
    n = max(d.n_beta for d in descs)
    for i in range(1, n):
        for k, r in runs.items():
            if i < descs[k].n_beta:
                rc = r.step()
                if rc:
                    raise RuntimeError(f"oracle step failed for run {k}: {rc}")
        pair_measure()
    return runs


def compare_records(gpu, ora, rtol=1e-12):
    """Integers bit-exact; ln Q and -beta F within rtol (relative, floor 1)."""
    int_fields = ["sumE", "sumE2", "sumAbsM", "sumM2", "sum_c2", "sum_absq", "sum_absq_pair", "R", "R_target",
                  "n_fam", "max_fam", "n_q", "n_q_pair", "N", "status", "sumE3", "sumE4", "sumAbsM3", "sumM4",
                  "sum_absq_wang", "n_q_wang", "wang_swaps"]
    for f in int_fields:
        assert np.array_equal(gpu[f], ora[f]), (f, np.nonzero(gpu[f] != ora[f])[0][:5])
    assert np.array_equal(gpu["beta"], ora["beta"])
    for f in ("lnQ", "minus_betaF"):
        scale = np.maximum(1.0, np.abs(ora[f]))
        err = np.abs(gpu[f] - ora[f]) / scale
        assert err.max() <= rtol, (f, err.max(), np.argmax(err))


def wavg_scale(o, f, N):
    """Magnitude against which the rounding of weighted average f is judged.
    Differences of O(1) terms (variances, central moments by binomial
    expansion, 1 - ratio) are judged relative to the terms combined."""
    import math
    scale = np.maximum(np.abs(o[f]), 1e-300)
    if f in ("Wvar_c", "Wvar_chi", "W_c", "W_chi"):
        scale = np.maximum(scale, np.abs(o["beta"]) ** 2 * N * (np.abs(o["W_e2"]) + np.abs(o["W_m2"])) + 1e-300)
    if f.startswith("Wk"):
        k, obs = int(f[2]), f[-1]
        raw = [np.ones_like(o["W_e"])] + [o[n] for n in ((f"W_{obs}", f"W_{obs}2", f"W_{obs}3", f"W_{obs}4"))]
        cond = sum(math.comb(k, l) * np.abs(raw[1]) ** (k - l) * np.abs(raw[l]) for l in range(k + 1))
        scale = np.maximum(scale, cond)
    if f in ("W_U4", "W_U4_conf"):
        scale = np.maximum(scale, 1.0)
    return scale


def wavg_close(g, o, names, N, rtol=1e-12):
    for f in names:
        if f in ("W_U4_conf",) and np.any(np.isnan(o[f])):
            assert np.array_equal(np.isnan(g[f]), np.isnan(o[f])), f
            ok = ~np.isnan(o[f])
            err = np.abs(g[f][ok] - o[f][ok]) / wavg_scale(o, f, N)[ok]
        else:
            err = np.abs(g[f] - o[f]) / wavg_scale(o, f, N)
        assert np.all(err <= rtol), (f, err.max())
