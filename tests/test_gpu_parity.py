"""Parity of the CUDA engine (through the C ABI) with the CPU oracle.

Integers (spins, energies, magnetisations, family ids, population sizes,
histograms, integer sums) must match bit for bit; ln Q and -beta F within
1e-12 relative (floor 1), weighted FP64 averages within 1e-12 relative
(floor given by the magnitude of the terms combined).
"""
import numpy as np
import pytest

import oracle as O
from paper_2207_05535_gb300 import _lib
from paper_2207_05535_gb300 import workloads as W
from tests.helpers import compare_records, oracle_runs, wavg_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2207_05535_gb300 import build
    build.build()
    _lib.load()


def check_run(eng, descs, ora, k):
    d = descs[k]
    rec = eng.records(k, qhist=bool(d.overlap))
    if d.overlap:
        rec, qa, qb = rec
    o = ora[k]
    orecs = o.records()
    assert o.cur_step == d.n_beta - 1
    compare_records(rec, orecs)
    s, E, M, fam, step = eng.population(k)
    os_, oE, oM, ofam = o.population()
    assert step == d.n_beta - 1
    assert np.array_equal(s, os_), "spins differ"
    assert np.array_equal(E, oE) and np.array_equal(M, oM) and np.array_equal(fam, ofam)
    if d.overlap:
        for i in range(d.n_beta):
            ha, hb = o.qhist(i)
            if d.overlap & W.Q_SHIFT:
                assert np.array_equal(qa[i], ha), ("qhist", i)
            if d.overlap & W.Q_PAIR:
                assert np.array_equal(qb[i], hb), ("qhist pair", i)


def run_case(descs, use_graph=True, idx=None):
    ora = oracle_runs(descs, idx)
    with _lib.Engine(descs) as eng:
        eng.run_to_end(use_graph)
        for k in (idx if idx is not None else range(len(descs))):
            check_run(eng, descs, ora, k)
    return ora


# ------------------------------------------------------------------ init
@pytest.mark.parametrize("L,model,R", [(4, 0, 37), (6, 1, 130), (8, 0, 64), (10, 1, 33), (16, 1, 257), (32, 0, 9),
                                       (64, 1, 5), (128, 0, 3), (256, 1, 2)])
def test_initial_population_bit_exact(L, model, R):
    d = [W.RunDesc(L, model, R, 1, np.array([0.0]), seed=3, run_id=7, disorder_id=2)]
    run_case(d)


# ------------------------------------------------------------------ anneal
def test_ferromagnet_L8_several_runs():
    descs = W.ferro_runs(L=8, R=500, theta=3, beta_f=0.5, n=11, M=3, seed=1)
    run_case(descs)


def test_ferromagnet_L8_without_graph():
    descs = W.ferro_runs(L=8, R=200, theta=2, beta_f=0.6, n=6, M=2, seed=5)
    run_case(descs, use_graph=False)


def test_glass_L16_pairs_with_overlaps():
    descs = W.glass_pairs(L=16, R=300, theta=2, beta_f=3.0, n=9, n_samples=2, seed=1)
    run_case(descs)


@pytest.mark.parametrize("L", [4, 6, 10, 12, 14])
def test_glass_ragged_lattices(L):
    """L/2 odd or smaller than a Philox group: ragged colour planes."""
    b = W.schedule(2.0, 6)
    descs = [W.RunDesc(L, W.EA_PMJ, 150, 3, b, seed=2, run_id=r, disorder_id=1, overlap=W.Q_SHIFT)
             for r in range(2)]
    run_case(descs)


def test_large_lattices_multi_group_threads():
    descs = [W.RunDesc(64, W.FERRO, 40, 2, W.schedule(0.44, 4), seed=1, run_id=0),
             W.RunDesc(128, W.EA_PMJ, 9, 1, W.schedule(1.0, 3), seed=1, run_id=1, disorder_id=4,
                       overlap=W.Q_SHIFT),
             W.RunDesc(256, W.FERRO, 5, 1, W.schedule(0.44, 3), seed=1, run_id=2)]
    run_case(descs)


def test_mixed_sizes_in_one_engine():
    """Runs of different L, R and schedule length share one engine; each must
    equal its oracle run (and so its result alone)."""
    descs = [W.RunDesc(8, W.FERRO, 100, 2, W.schedule(0.5, 5), run_id=0),
             W.RunDesc(12, W.EA_PMJ, 333, 1, W.schedule(2.0, 8), run_id=1, disorder_id=3, overlap=W.Q_SHIFT),
             W.RunDesc(16, W.FERRO, 64, 3, W.schedule(0.44, 3), run_id=2),
             W.RunDesc(8, W.EA_PMJ, 1, 2, W.schedule(1.0, 4), run_id=3)]
    run_case(descs)


def test_multinomial_resampling():
    b = W.schedule(2.5, 8)
    descs = [W.RunDesc(8, W.EA_PMJ, 300, 2, b, seed=4, run_id=r, disorder_id=2, resample=W.MULTINOMIAL,
                       overlap=W.Q_SHIFT) for r in range(2)]
    descs.append(W.RunDesc(16, W.FERRO, 1000, 1, W.schedule(0.6, 6), seed=4, run_id=5, resample=W.MULTINOMIAL))
    run_case(descs)


def test_populations_split_over_several_ctas():
    """Populations of more than 16384 replicas are measured and (nearest-integer)
    resampled by several CTAs each, with families crossing the CTAs'
    boundaries; a small run and a multinomial run share the same launches."""
    descs = [W.RunDesc(8, W.FERRO, 40000, 1, W.schedule(0.6, 7), seed=6, run_id=0),
             W.RunDesc(6, W.EA_PMJ, 20000, 1, W.schedule(2.5, 8), seed=6, run_id=1, disorder_id=2),
             W.RunDesc(8, W.FERRO, 300, 2, W.schedule(0.5, 7), seed=6, run_id=2),
             W.RunDesc(8, W.EA_PMJ, 8300, 1, W.schedule(2.0, 6), seed=6, run_id=3, disorder_id=1,
                       resample=W.MULTINOMIAL)]
    run_case(descs)


def test_degenerate_schedules():
    """theta = 0, repeated temperatures (dbeta = 0), one temperature, R = 1."""
    descs = [W.RunDesc(8, W.FERRO, 50, 0, W.schedule(1.0, 5), run_id=0),
             W.RunDesc(8, W.EA_PMJ, 50, 2, np.array([0.0, 0.3, 0.3, 0.3, 0.9]), run_id=1, disorder_id=1),
             W.RunDesc(6, W.FERRO, 20, 4, np.array([0.0]), run_id=2),
             W.RunDesc(10, W.FERRO, 1, 3, W.schedule(2.0, 6), run_id=3)]
    run_case(descs)


def test_capacity_overflow_is_reported_not_written():
    d = W.RunDesc(8, W.EA_PMJ, 200, 1, W.schedule(3.0, 30), run_id=0, disorder_id=1, R_cap=201)
    o = O.OracleRun.from_desc(d)
    rc, step = 0, 0
    while not rc and o.cur_step + 1 < d.n_beta:
        rc = o.step()
        step = o.cur_step
    assert rc == 3, "choose a case where the oracle overflows"
    with _lib.Engine([d]) as eng:
        eng.step(d.n_beta - 1)
        with pytest.raises(_lib.PAError) as ei:
            eng.sync()
        assert ei.value.code == 3
        rec = _lib.pa_measure(eng.h, 0, step + 1) if step + 1 < d.n_beta else None
        if rec is not None:
            assert rec["status"] == 3


# ------------------------------------------------------------------ weighted averages
def _wavg_close(g, o, N=64):
    wavg_close(g, o, _lib.WAVG_DTYPE.names, N)


def test_weighted_averages_from_host_records():
    descs = W.glass_pairs(L=8, R=200, theta=2, beta_f=2.0, n=7, n_samples=3, seed=2)
    ora = oracle_runs(descs)
    recs = np.stack([ora[k].records() for k in range(len(descs))])
    qh = np.stack([np.stack([ora[k].qhist(i)[0] for i in range(7)]) for k in range(len(descs))])
    qp = np.stack([np.stack([ora[k].qhist(i)[1] for i in range(7)]) for k in range(len(descs))])
    for kind in (0, 1):
        o, oPq, oPp = O.weighted_average(recs, 64, kind, qh=qh, qh_pair=qp)
        g, gPq, gPp = _lib.pa_weighted_average(recs, 64, kind, qh=qh, qh_pair=qp)
        _wavg_close(g, o)
        assert np.allclose(gPq, oPq, rtol=1e-12, atol=1e-15) and np.allclose(gPp, oPp, rtol=1e-12, atol=1e-15)


def test_weighted_averages_of_resident_runs():
    descs = W.glass_pairs(L=8, R=150, theta=2, beta_f=2.0, n=6, n_samples=3, seed=3)
    ora = oracle_runs(descs)
    with _lib.Engine(descs) as eng:
        eng.run_to_end()
        idx = np.arange(len(descs), dtype=np.uint32)
        for kind in (0, 1):
            g, gPq, gPp = eng.weighted_average(idx, 2, kind, q=True)
            for grp in range(3):
                recs = np.stack([ora[2 * grp].records(), ora[2 * grp + 1].records()])
                qh = np.stack([np.stack([ora[k].qhist(i)[0] for i in range(6)]) for k in (2 * grp, 2 * grp + 1)])
                qp = np.stack([np.stack([ora[k].qhist(i)[1] for i in range(6)]) for k in (2 * grp, 2 * grp + 1)])
                o, oPq, oPp = O.weighted_average(recs, 64, kind, qh=qh, qh_pair=qp)
                _wavg_close(g[grp], o)
                assert np.allclose(gPq[grp], oPq, rtol=1e-12, atol=1e-15)
                assert np.allclose(gPp[grp], oPp, rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------------ full-size workload
@pytest.mark.slow
def test_glass_L16_R5000_full_size_sampled_runs():
    """The full +-J glass workload (L=16, R=5000, 101 temperatures, theta=10,
    100 disorder samples x 2 populations) in the launch configuration the
    benchmark times; the oracle recomputes one disorder sample (both of its
    populations, with their two-population overlaps) in full."""
    descs = W.glass_L16_R5000()
    sample = 37
    ora = oracle_runs(descs, [2 * sample, 2 * sample + 1])
    with _lib.Engine(descs) as eng:
        eng.run_to_end(True)
        for k in (2 * sample, 2 * sample + 1):
            check_run(eng, descs, ora, k)
        # every run: population sizes stay near R and the records are complete
        for k in range(0, len(descs), 17):
            rec = eng.records(k)
            assert np.all(rec["status"] == 0) and np.all(rec["R"] > 4000)


@pytest.mark.parametrize("L", [4, 6, 8, 10, 12, 14, 16, 18, 30, 32, 34, 46, 50, 62, 64, 100, 128, 254, 256])
def test_bitsliced_and_generic_sweeps_agree(L):
    """The bit-sliced kernels (L/2 a power of two; rows padded to a pitch;
    rows repacked without padding) and the byte-plane kernel flip the same
    spins: whole anneals agree bit for bit for the ferromagnet and the glass.
    Nine steps take the autotuned engine through every candidate shape of its
    lattice size (one warm-up step, then two steps per candidate)."""
    R = max(4, 20000 // (L * L) * 8)
    b = W.schedule(1.5, 10)
    descs = [W.RunDesc(L, W.FERRO, R, 2, b, seed=3, run_id=0),
             W.RunDesc(L, W.EA_PMJ, R, 2, b, seed=3, run_id=1, disorder_id=9, overlap=W.Q_SHIFT)]
    out = []
    for flags in (0, _lib.PA_CREATE_GENERIC_SWEEP, _lib.PA_CREATE_NO_AUTOTUNE):
        with _lib.Engine(descs, flags=flags) as eng:
            eng.run_to_end()
            out.append([(eng.records(k), eng.population(k)) for k in range(2)])
    for other in out[1:]:
        for (ra, pa), (rb, pb) in zip(out[0], other):
            assert np.array_equal(ra, rb)
            for x, y in zip(pa, pb):
                assert np.array_equal(np.asarray(x), np.asarray(y))


def test_uneven_batch_work_list():
    """Runs of very different R share each lattice size's work list (one launch
    per kernel): every run equals its oracle run."""
    b = W.schedule(1.0, 5)
    descs = []
    for k, (L, R) in enumerate([(16, 5), (16, 2000), (16, 37), (32, 3), (32, 500), (8, 1), (8, 1000), (64, 17)]):
        descs.append(W.RunDesc(L, W.FERRO if k % 2 else W.EA_PMJ, R, 2, b, seed=8, run_id=k, disorder_id=k))
    run_case(descs)


def test_philox_calibration_reports_a_plausible_rate():
    split = _lib.pa_calibrate_philox(False, reps=2)
    wide = _lib.pa_calibrate_philox(True, reps=2)
    assert 1e10 < split < 1e13 and 1e10 < wide < 1e13


def test_tuned_shapes_are_reused_by_later_engines():
    b = W.schedule(1.0, 8)
    descs = [W.RunDesc(64, W.FERRO, 100, 2, b, seed=9, run_id=r) for r in range(3)]
    with _lib.Engine(descs) as a:
        assert _lib.pa_tuning_pending(a.h) in (0, 1)  # 0 if an earlier engine of the process chose the shape
        a.step(7, False)  # one warm-up step, two per candidate shape, then tuned
        assert _lib.pa_tuning_pending(a.h) == 0
        shape_a = _lib.pa_sweep_shapes(a.h)
        rec_a = a.records(0)
    assert shape_a[0][3] == 1
    with _lib.Engine(descs) as e:
        assert _lib.pa_sweep_shapes(e.h) == shape_a  # chosen, without timing, before any step
        counts = []
        for _ in range(3):
            l0 = e.launches
            e.step(1, False)
            counts.append(e.launches - l0)
        assert counts[0] == counts[1] == counts[2]   # no candidate launches on the first step
        e.step(4, False)
        assert np.array_equal(e.records(0), rec_a)
