"""The C-ABI library: builds, loads, exports every symbol of include/pa.h, its
structs match the Python mirrors, and argument validation runs before any CUDA
call (so these tests need no GPU)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2207_05535_gb300 import _lib, build
from paper_2207_05535_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# CUDA headers of the toolkit whose nvcc builds the engine (<toolkit>/bin/nvcc -> <toolkit>/include)
CUDA_INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(build.nvcc()))), "include")
HEADER = os.path.join(ROOT, "include", "pa.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pa_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}$", out, re.M), n


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "pa.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(pa_run_desc), sizeof(pa_step_record), sizeof(pa_wavg),
         offsetof(pa_step_record, R), offsetof(pa_step_record, status), offsetof(pa_wavg, W_minus_betaF),
         offsetof(pa_step_record, sumE3), offsetof(pa_step_record, sumM4), offsetof(pa_wavg, W_e3),
         offsetof(pa_wavg, W_U4_conf), offsetof(pa_run_desc, log_g));
  return 0;
}
''')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals[0] == C.sizeof(_lib.pa_run_desc)
    assert vals[1] == _lib.RECORD_DTYPE.itemsize
    assert vals[2] == _lib.WAVG_DTYPE.itemsize
    assert vals[3] == _lib.RECORD_DTYPE.fields["R"][1]
    assert vals[4] == _lib.RECORD_DTYPE.fields["status"][1]
    assert vals[5] == _lib.WAVG_DTYPE.fields["W_minus_betaF"][1]
    assert vals[6] == _lib.RECORD_DTYPE.fields["sumE3"][1]
    assert vals[7] == _lib.RECORD_DTYPE.fields["sumM4"][1]
    assert vals[8] == _lib.WAVG_DTYPE.fields["W_e3"][1]
    assert vals[9] == _lib.WAVG_DTYPE.fields["W_U4_conf"][1]
    assert vals[10] == _lib.pa_run_desc.log_g.offset


def test_status_strings(lib):
    for code in range(9):
        assert _lib.pa_status_string(code)


@pytest.mark.parametrize("bad", [
    dict(L=7), dict(L=2), dict(L=258), dict(R=0), dict(R_cap=10, R=20), dict(model=3), dict(resample=5),
    dict(betas=np.array([0.0, 0.5, 0.4])), dict(betas=np.array([])), dict(overlap=8),
    dict(theta=W.THETA_INF), dict(theta=W.THETA_INF, log_g=np.zeros(129), overlap=1),
    dict(theta=W.THETA_INF, log_g=np.full(129, -np.inf)), dict(theta=W.THETA_INF, log_g=np.full(129, np.nan)),
    dict(theta=W.THETA_INF, log_g=np.where(np.arange(129) < 2, 0.0, -np.inf)),
    dict(theta=(1 << 22) + 1), dict(overlap=W.Q_WANG, R=9000), dict(overlap=W.Q_WANG, R=8000, R_cap=8193),
])
def test_invalid_descriptors_rejected_before_any_device_work(lib, bad):
    args = dict(L=8, model=W.FERRO, R=16, theta=1, betas=np.array([0.0, 0.1]))
    cap = bad.pop("R_cap", 0)
    args.update(bad)
    d = W.RunDesc(**args)
    if cap:
        d.R_cap = cap
    with pytest.raises(_lib.PAError) as ei:
        _lib.pa_create([d])
    assert ei.value.code == 1


def test_paired_runs_must_be_mutual(lib):
    b = W.schedule(1.0, 3)
    a = W.RunDesc(8, W.EA_PMJ, 16, 1, b, overlap=W.Q_PAIR, paired=1)
    c = W.RunDesc(8, W.EA_PMJ, 16, 1, b, overlap=W.Q_PAIR, paired=0, run_id=1)
    bad = W.RunDesc(10, W.EA_PMJ, 16, 1, b, overlap=W.Q_PAIR, paired=0, run_id=1)
    with pytest.raises(_lib.PAError):
        _lib.pa_create([a, bad])
    with pytest.raises(_lib.PAError):
        _lib.pa_create([W.RunDesc(8, W.EA_PMJ, 16, 1, b, overlap=W.Q_PAIR, paired=0)])
    del c


def test_oracle_and_engine_records_share_the_abi_layout():
    import oracle as O
    assert O.RECORD_DTYPE == _lib.RECORD_DTYPE
    assert O.WAVG_DTYPE == _lib.WAVG_DTYPE


def test_binding_argument_counts_match_the_header(lib):
    """Every declaration in pa.h has as many parameters as its ctypes binding."""
    with open(os.path.join(ROOT, "include", "pa.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    decls = {m.group(1): m.group(2) for m in re.finditer(r"\b(pa_\w+)\s*\(([^;{]*?)\)\s*;", text)}
    for name in _lib.EXPORTS:
        assert name in decls, name
        params = [p for p in decls[name].split(",") if p.strip() and p.strip() != "void"]
        assert len(getattr(lib, name).argtypes) == len(params), name


def _documented_plane_words(L):
    """P(L) as the pool units of include/pa.h state it."""
    Lh = L // 2
    if Lh & (Lh - 1) == 0:
        pitch = Lh
    elif Lh < 32:
        pitch = min(p for p in (4, 8, 16, 32) if p >= Lh and L * p % 32 == 0)
    else:
        pitch = -(-Lh // 32) * 32
    return -(-L * pitch // 32)


def test_pool_sizes_follow_the_documented_units(lib):
    for L in range(4, 257, 2):
        for R, resample in ((100, W.NEAREST), (40000, W.NEAREST), (300, W.MULTINOMIAL)):
            d = W.RunDesc(L, W.FERRO, R, 2, W.schedule(1.0, 11), resample=resample)
            c = _lib.pa_pool_sizes([d])
            N, P = L * L, _documented_plane_words(L)
            S = -(-2 * P // 4) * 4
            assert d.R_cap == (R if resample == W.MULTINOMIAL else W.default_cap(R))
            assert (c.max_runs, c.replica_capacity, c.record_capacity, c.qhist_words) == (1, d.R_cap, 11, 0)
            assert c.spin_words == d.R_cap * S, L
            assert c.coupling_words == 2 * S + 8 * P, L
            assert c.scratch_words == (3 * ((N + 2) // 2) + N + 5
                                       + max((d.R_cap + 1) // 2, 128, 4 * -(-d.R_cap // 16384))), (L, R)
            n_db = len({x.tobytes() for x in np.diff(d.betas)})  # distinct dbeta bit patterns
            assert c.table_doubles == n_db * (N + 1), L


def test_pool_sizes_share_tables_and_count_overlaps(lib):
    b = W.schedule(1.0, 5)
    n_db = len({x.tobytes() for x in np.diff(b)})
    a = W.RunDesc(8, W.EA_PMJ, 50, 1, b, overlap=W.Q_SHIFT | W.Q_PAIR, paired=1)
    p = W.RunDesc(8, W.EA_PMJ, 50, 1, b, run_id=1, overlap=W.Q_SHIFT | W.Q_PAIR, paired=0)
    f16 = W.RunDesc(16, W.FERRO, 50, 1, b)
    alone = W.RunDesc(8, W.EA_PMJ, 50, 1, b, overlap=W.Q_SHIFT)  # a's needs without its partner
    one = [_lib.pa_pool_sizes([r]) for r in (alone, f16)]
    assert one[0].qhist_words == 5 * 65
    both = _lib.pa_pool_sizes([a, p, f16])
    assert both.max_runs == 3
    assert both.qhist_words == 2 * 5 * 65
    assert both.replica_capacity == 2 * one[0].replica_capacity + one[1].replica_capacity
    assert both.spin_words == 2 * one[0].spin_words + one[1].spin_words
    assert both.table_doubles == n_db * (65 + 257)  # one table per distinct (N, dbeta), shared by the pair
    # theta = infinity: n_beta (2N + 2) per distinct (ln g, schedule), on top of the weight tables
    g = np.full(2 * 16 + 1, -np.inf)
    g[0::2] = 0.0
    t1 = W.RunDesc(4, W.FERRO, 50, W.THETA_INF, b, log_g=g)
    t2 = W.RunDesc(4, W.FERRO, 50, W.THETA_INF, b, run_id=1, log_g=g)
    t3 = W.RunDesc(4, W.FERRO, 50, W.THETA_INF, W.schedule(0.5, 5), run_id=2, log_g=g)
    n_db3 = len({x.tobytes() for x in np.diff(W.schedule(0.5, 5))})
    c = _lib.pa_pool_sizes([t1, t2, t3])
    assert c.table_doubles == (n_db + n_db3) * 17 + 2 * 5 * 34


def test_pool_sizes_reject_what_pa_create_rejects(lib):
    with pytest.raises(_lib.PAError) as ei:
        _lib.pa_pool_sizes([W.RunDesc(9, W.FERRO, 10, 1, W.schedule(1.0, 3))])  # odd L
    assert ei.value.code == 1
    d = _lib.make_descs([W.RunDesc(8, W.FERRO, 10, 1, W.schedule(1.0, 3))])
    assert lib.pa_pool_sizes(d, 1, None) == 1


def test_benchmark_plane_words_follow_the_engine_layout(tmp_path):
    """bench.py's byte counts use the engine's colour-plane size (row pitch)."""
    import bench
    prog = tmp_path / "pw.cpp"
    prog.write_text(r'''
#include <cstdio>
#include <cuda_runtime.h>
#include "pa_internal.cuh"
int main() {
  for (unsigned L = 4; L <= 256; L += 2) std::printf("%u %u\n", L, pa::plane_words_of(L));
  return 0;
}
''')
    exe = tmp_path / "pw"
    subprocess.run(["g++", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I",
                    os.path.join(ROOT, "paper_2207_05535_gb300", "csrc"), "-I", CUDA_INCLUDE, str(prog),
                    "-o", str(exe)], check=True)
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n"):
        if line:
            L, pw = (int(x) for x in line.split())
            assert bench.plane_words(L) == pw, L


def test_run_scratch_regions_fit_and_do_not_overlap(tmp_path):
    """A run's scratch (histograms, level tables, and the tail shared by the
    multinomial member list, the per-CTA totals and the per-CTA family
    statistics) holds every region the kernels index, for any lattice size and
    capacity; the CTA count of a run covers its replicas."""
    prog = tmp_path / "scr.cpp"
    prog.write_text(r'''
#include <cstdio>
#include <cuda_runtime.h>
#include "pa_internal.cuh"
int main() {
  const unsigned caps[] = {1u, 2u, 31u, 4096u, 16383u, 16384u, 16385u, 100000u, 1000000u, 5000000u, 4200000000u};
  for (unsigned L = 4; L <= 256; L += 2)
    for (unsigned cap : caps) {
      const unsigned N = L * L;
      std::printf("%u %u %llu %llu %llu %llu %llu %u %u %u %u %llu\n", N, cap,
                  (unsigned long long)pa::scr_mhist_off(N), (unsigned long long)pa::scr_table_off(N),
                  (unsigned long long)pa::scr_level_off(N), (unsigned long long)pa::scr_tail_off(N),
                  (unsigned long long)pa::scratch_words(N, cap), pa::run_ctas(cap), pa::CTA_REPLICAS,
                  pa::MAX_RUN_CTAS, pa::resample_nearest_launches(cap),
                  (unsigned long long)pa::MEASURE_PART_WORDS);
    }
  return 0;
}
''')
    exe = tmp_path / "scr"
    subprocess.run(["g++", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I",
                    os.path.join(ROOT, "paper_2207_05535_gb300", "csrc"), "-I", CUDA_INCLUDE, str(prog),
                    "-o", str(exe)], check=True)
    rows = [list(map(int, line.split())) for line in
            subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n") if line]
    assert rows
    for N, cap, mh, tab, lev, tail, words, nc, per_cta, max_ctas, launches, part_words in rows:
        n1 = N + 1
        assert 4 * n1 <= 8 * mh  # energy histogram, u32
        assert 4 * n1 <= 8 * (tab - mh)  # magnetisation histogram, u32
        assert 8 * n1 <= 8 * (lev - tab)  # CDF / thresholds, f64 / u64
        assert 4 * n1 <= 8 * (tail - lev)  # fill counters / floors, u32
        room = 8 * (words - tail)
        assert room >= 4 * cap  # multinomial member list
        assert room >= 4 * max_ctas  # per-CTA replica totals
        assert room >= 8 * part_words * nc  # per-CTA family statistics
        assert 1 <= nc <= max_ctas
        assert nc == max_ctas or nc * per_cta >= cap
        assert (nc - 1) * per_cta < cap or nc == 1
        assert launches == (1 if nc == 1 else 2)


def test_measured_traffic_is_keyed_by_each_kernels_own_source(tmp_path, monkeypatch):
    """bench.py reports an ncu traffic figure only for the source it was taken
    on: an edit in one kernel's section changes that kernel's hash and no other,
    an edit in the shared header changes both."""
    import shutil

    import bench
    src = os.path.join(ROOT, "paper_2207_05535_gb300", "csrc")
    dst = tmp_path / "paper_2207_05535_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("pa_internal.cuh", "pa_kernels.cu"):
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    base = {k: bench.source_sha(k) for k in bench.KERNEL_SECTIONS}

    def edit(name, marker, text):
        p = dst / name
        body = p.read_text()
        i = body.index(marker) + len(marker)
        p.write_text(body[:i] + text + body[i:])

    edit("pa_kernels.cu", "// Measurement (Sec. III.B", " ")
    assert bench.source_sha("sweep") == base["sweep"] and bench.source_sha("measure") != base["measure"]
    edit("pa_kernels.cu", "// Overlaps (Sec. III.D)", " ")  # the end marker of the sweep section: outside it
    assert bench.source_sha("sweep") == base["sweep"]
    edit("pa_kernels.cu", "// Fused gather + theta checkerboard", " ")
    assert bench.source_sha("sweep") != base["sweep"]
    mid = {k: bench.source_sha(k) for k in bench.KERNEL_SECTIONS}
    edit("pa_internal.cuh", "#pragma once", "\n")
    assert all(bench.source_sha(k) != mid[k] for k in bench.KERNEL_SECTIONS)
    monkeypatch.undo()
    for t in bench.TRAFFIC:
        assert bench.measured_traffic(t["kernel"], "no such workload") is None
