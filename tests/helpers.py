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
                  "n_fam", "max_fam", "n_q", "n_q_pair", "N", "status"]
    for f in int_fields:
        assert np.array_equal(gpu[f], ora[f]), (f, np.nonzero(gpu[f] != ora[f])[0][:5])
    assert np.array_equal(gpu["beta"], ora["beta"])
    for f in ("lnQ", "minus_betaF"):
        scale = np.maximum(1.0, np.abs(ora[f]))
        err = np.abs(gpu[f] - ora[f]) / scale
        assert err.max() <= rtol, (f, err.max(), np.argmax(err))
