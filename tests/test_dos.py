"""The package's transfer-matrix density of states (input of theta = infinity
runs) against the oracle's independent transfer matrix and the stored exact
L = 8 ferromagnet density of states."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2207_05535_gb300 import dos


@pytest.mark.parametrize("L,model,dis", [(4, 0, 0), (4, 1, 3), (6, 0, 0), (6, 1, 2)])
def test_equals_oracle_transfer_matrix(L, model, dis):
    Jr, Jd = O.couplings(L, model, 1, dis)
    ref = np.array([float(c) for c in O.dos_transfer(L, Jr, Jd)])
    g = dos.count_unsatisfied(L, Jr, Jd)
    assert np.array_equal(g, ref) and g.sum() == 2.0 ** (L * L)
    lg = dos.log_dos(L, Jr, Jd)
    assert np.all(np.isneginf(lg[ref == 0])) and np.allclose(np.exp(lg[ref > 0]), ref[ref > 0], rtol=1e-14)


def test_L8_ferromagnet_equals_stored_exact_counts():
    with open(os.path.join(os.path.dirname(__file__), "golden", "dos_fm_L8.json")) as f:
        gE = {int(k): int(v) for k, v in json.load(f)["g_by_E"].items()}
    ref = np.array([float(gE.get(2 * u - 128, 0)) for u in range(129)])
    g = dos.count_unsatisfied(8)
    assert np.all((g == 0) == (ref == 0))
    assert np.max(np.abs(g - ref) / np.maximum(ref, 1)) < 1e-12
