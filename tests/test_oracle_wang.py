"""Pins of the oracle's Wang pairing (Sec. III.D, independent pairings from
permutations, with the random search pattern sigma).

  - The result is a permutation pi* of the replicas in which no replica is
    paired with one of its own family.
  - By Hall's theorem such a permutation exists exactly when no family holds
    more than half of the replicas: the search succeeds then and fails otherwise.
  - The paper reports that the random search pattern makes pi* uniform over the
    valid permutations (it is not with sigma = identity).  Enumerating every
    (pi, sigma) pair shows this holds exactly for the family structures used
    here, though not for every structure; the oracle's draws must be uniform
    over the valid set, which is listed independently with itertools.
  - At beta_0 = 0 the replicas are independent uniform configurations, so the
    Hamming distance of every pair is Binomial(N, 1/2).
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O


def _families(sizes):
    return np.repeat(np.arange(len(sizes)), sizes).astype(np.uint32)


@pytest.mark.parametrize("seed", range(6))
def test_pairs_are_permutations_without_shared_families(seed):
    rng = np.random.default_rng(seed)
    for _ in range(40):
        R = int(rng.integers(2, 300))
        sizes = []
        while sum(sizes) < R:
            sizes.append(int(rng.integers(1, max(2, R // 3))))
        sizes[-1] -= sum(sizes) - R
        sizes = [c for c in sizes if c > 0]
        if max(sizes) * 2 > R:
            continue
        fam = _families(sizes)
        pi, swaps = O.wang_pairing(3, int(rng.integers(1 << 30)), 5, fam)
        assert pi is not None
        assert np.array_equal(np.sort(pi), np.arange(R))
        assert np.all(fam[pi] != fam)
        assert swaps <= R


@pytest.mark.parametrize("sizes,ok", [([2, 2], True), ([3, 1], False), ([1, 1], True), ([1], False), ([4, 2, 2], True),
                                      ([5, 2, 2], False), ([50, 30, 20], True), ([51, 49], False)])
def test_pairing_exists_exactly_when_no_family_exceeds_half(sizes, ok):
    for run in range(5):
        pi, _ = O.wang_pairing(1, run, 2, _families(sizes))
        assert (pi is not None) == ok


@pytest.mark.parametrize("fam", [[0, 1, 1, 1, 2, 2], [0, 1, 1, 2, 2, 2], [0, 0, 1, 1, 2]])
def test_random_search_pattern_gives_uniform_pairings(fam):
    R = len(fam)
    valid = [p for p in itertools.permutations(range(R)) if all(fam[k] != fam[p[k]] for k in range(R))]
    index = {p: n for n, p in enumerate(valid)}
    counts = np.zeros(len(valid))
    for run in range(40000):
        pi, _ = O.wang_pairing(9, run, 4, fam)
        counts[index[tuple(int(x) for x in pi)]] += 1
    assert stats.chisquare(counts).pvalue > 1e-4


def test_overlaps_of_wang_pairs_at_infinite_temperature():
    L, N, R = 4, 16, 3000
    o = O.OracleRun(L, 0, R, R + 500, 2, [0.0, 0.3, 0.6], 4, 1, 0, overlap=4)
    rec = o.record(0)
    h = o.qhist_wang(0)
    assert rec["n_q_wang"] == R and h.sum() == R
    p = np.array([math.comb(N, d) / 2 ** N for d in range(N + 1)])
    assert stats.chisquare(h, p * R).pvalue > 1e-4
    mean_absq = float(np.sum(p * np.abs(N - 2 * np.arange(N + 1)))) / N
    assert abs(rec["sum_absq_wang"] / (N * R) - mean_absq) < 5 * 0.25 / math.sqrt(R)
    o.run_to_end()
    for i in range(3):
        r = o.record(i)
        assert r["n_q_wang"] in (0, r["R"]) and o.qhist_wang(i).sum() == r["n_q_wang"]
    wa, _, _, Pw = O.weighted_average(o.records()[None], N, 0, qh_wang=np.stack([o.qhist_wang(i) for i in range(3)])[None])
    recs = o.records()
    ok = recs["n_q_wang"] > 0
    assert np.allclose(wa["W_absq_wang"][ok], recs["sum_absq_wang"][ok] / (N * recs["n_q_wang"][ok]), rtol=1e-14)
    assert np.allclose(Pw[ok].sum(axis=1), 1.0, rtol=1e-14)
