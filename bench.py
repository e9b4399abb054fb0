#!/usr/bin/env python
"""Benchmark: attempted spin updates per ns of population annealing on GB300.

Default workload (the largest single-GPU configuration): 4096 independent 2D
Ising ferromagnet runs in one batch, L drawn from {16, 32, 64, 128} and R from
{1e3, 1e4, 5e4} by seed, beta 0 -> 1 in 101 temperatures, theta = 10
checkerboard Metropolis sweeps per temperature, nearest-integer resampling;
about 120 GB of bit-packed populations resident in HBM.  One "step" is one
anneal temperature of the whole batch (resampling, sweeps and measurement of
every run); the warm-up and the timed steps walk the schedule from beta_0 on
(the timed temperature range is in `config`).  `--workload` selects the other
workloads, where one step is one whole anneal (small batches) or the serving
stream.  Inputs are seeded and synthetic (the paper's instances are not
available).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload W]

Prints one JSON line on rank 0.  `value` is device-timed with the populations
resident in HBM; `e2e` times the same work through the C ABI from host
descriptors to host results (engine creation and uploads, the K steps, each
followed by a copy of every run's new record to pinned host memory).
`--impl reference` times the CPU oracle on the host cores over a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "attempted spin updates/ns and PA runs/s (batched+served vs plain) at oracle-exact"
UNIT = "attempted spin updates/ns"
WORKLOADS = {
    "glass_L16_R5000": ("2D +-J EA glass L=16 periodic, R=5000, beta 0->3 in 101 steps, theta=10, nearest-integer "
                        "resampling, 100 disorder samples x 2 populations, index-shift + two-population overlaps, "
                        "free-energy-weighted averages over the two populations of each sample"),
    "ising_L8_R500": ("2D Ising FM L=8 periodic, R=500, beta 0->0.5 in 51 steps, theta=10, nearest-integer "
                      "resampling, M=20 runs from seed 1, free-energy-weighted averages over the 20 runs"),
    "uneven_4096": ("4096 independent 2D Ising FM runs, L drawn from {16,32,64,128}, R from {1e3,1e4,5e4} by seed, "
                    "beta 0->1 in 101 steps, theta=10, one launch per kernel per step over all runs"),
    "ferro_L8_theta_inf": ("2D Ising FM L=8 periodic, theta = infinity (energies drawn from the exact density of "
                           "states, Sec. V.B), R=2e4, beta 0->0.6 in 61 steps, nearest-integer resampling, 200 runs, "
                           "free-energy-weighted averages over groups of 20 runs"),
    "ising_L256_R1e5": ("2D Ising FM L=256 periodic, R=1e5, beta 0->0.44 in 201 steps, theta=20, "
                        "M=16 runs, free-energy-weighted averages over the runs"),
    "serving": ("Poisson stream of PA jobs at 200/s (FM or +-J glass with equal odds, L even uniform in 8..64, "
                "R log-uniform in 1e3..5e4, 50..300 temperatures, beta_f 1 (FM) / 3 (glass), theta=10), "
                "continuous batching in one server engine with a 64 GB pool budget"),
}
# Workloads whose bench step is one temperature of the whole batch (a whole
# anneal takes minutes); the others time whole anneals.
TEMPERATURE_STEP = {"uneven_4096", "ising_L256_R1e5"}
# Algorithmic work of one attempted update on the binding unit, the 32-bit
# integer multiplier: a quarter of a Philox4x32-10 call, whose 10 rounds hold
# two 32x32->64 multiplies each, i.e. 20 wide multiplies = 40 multiply-add
# slots per call, 10 per update.  The multiplier retires 64 multiply-add lanes
# per clock per SM.
ALGO_MULADD_PER_UPDATE = 10.0
ALGO_MULADD_PER_DRAW = 40.0  # theta = infinity: one Philox4x32-10 call per energy draw
INF_WORKLOADS = {"ferro_L8_theta_inf"}
METRIC_INF = "energy draws/ns of theta = infinity PA (Sec. V.B) at oracle-exact"
UNIT_INF = "energy draws/ns"


def metric_unit(wl):
    return (METRIC_INF, UNIT_INF) if wl in INF_WORKLOADS else (METRIC, UNIT)


def plane_words(L):
    """Words of one colour plane of a replica (rows padded to the engine's row pitch)."""
    Lh = L // 2
    if Lh & (Lh - 1) == 0:
        pitch = Lh
    elif Lh < 32:
        pitch = next(P for P in (4, 8, 16, 32) if P >= Lh and (L * P) % 32 == 0)
    else:
        pitch = (Lh + 31) // 32 * 32
    return (L * pitch + 31) // 32


def work_units(d, R):
    """Work of one temperature at population R: attempted spin updates (theta N R),
    or R energy draws for theta = infinity runs."""
    return R if d.theta == 0xFFFFFFFF else d.theta * d.N * R
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu
# capture of the kernel, valid only for the kernel source it was taken on.
# The uneven batch: the four lattice-size groups' sweep launches of one temperature
# (temperature 7, full size, one ncu pass), read + write summed: bytes per step.
TRAFFIC = [{"kernel": "sweep", "workload": "uneven_4096", "source_sha256_16": "009194d71dfeaa51",
            "bytes_per_launch": 81.124e9,
            "captured": "L=128: 15.06 + 40.83 GB, L=64: 7.15 + 10.86 GB, L=32: 2.53 + 3.06 GB, L=16: 0.80 + 0.83 GB "
                        "(dram__bytes_read.sum + dram__bytes_write.sum)"}]
MULADD_LANES_PER_SM = 64


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="uneven_4096", choices=sorted(WORKLOADS))
    ap.add_argument("--samples", type=int, default=100, help="glass: disorder samples (2 populations each)")
    ap.add_argument("--runs", type=int, default=0, help="ising/uneven: number of runs (0 = the workload's)")
    ap.add_argument("--window", type=float, default=10.0, help="serving: seconds of arrivals")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean arrivals per second")
    ap.add_argument("--rates", default="", help="serving: comma-separated arrival rates to sweep for the largest "
                                                "sustainable rate (then 50 %% and 80 %% of it are measured too)")
    ap.add_argument("--wang", action="store_true", help="also measure Wang pairing overlaps (Sec. III.D)")
    ap.add_argument("--max-temps", type=int, default=0,
                    help="anneal only the first T temperatures of the schedule (0 = all); reported in config")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the small whole-anneal workloads in `extra`")
    return ap.parse_args()


# ---------------------------------------------------------------- CPU oracle
def _workload_descs(wl, runs=0):
    from paper_2207_05535_gb300 import workloads as W
    if wl == "glass_L16_R5000":
        return W.glass_L16_R5000()
    if wl == "serving":
        return [d for _, d in W.serving_stream(duration=2.0)]
    if wl == "ising_L8_R500":
        return W.ising_L8_R500(M=runs or 20)
    if wl == "uneven_4096":
        return W.batched_uneven(n_runs=runs or 4096)
    if wl == "ferro_L8_theta_inf":
        from paper_2207_05535_gb300 import dos
        return W.ferro_theta_inf(dos.log_dos(8), M=runs or 200)
    return W.ising_L256_R1e5(M=runs or 16)


def _oracle_job(args):
    descs, n_temps, r_max = args
    sys.path.insert(0, ROOT)
    import dataclasses
    import oracle as O
    t0 = time.perf_counter()
    upd = 0
    for d in descs:  # runs one after another in this process
        if r_max and d.R > r_max:
            d = dataclasses.replace(d, R=r_max, R_cap=0)
        r = O.OracleRun.from_desc(d)
        for i in range(1, n_temps):
            assert r.step() == 0
            upd += work_units(d, int(r.record(i)["R"]))
    return upd, time.perf_counter() - t0


# bounded oracle samples per workload: (temperatures, population cap, runs per process)
ORACLE_SAMPLE = {"glass_L16_R5000": (25, 0, 1), "ising_L8_R500": (51, 0, 1), "uneven_4096": (2, 2000, 1),
                 "ising_L256_R1e5": (2, 200, 1), "serving": (6, 2000, 1), "ferro_L8_theta_inf": (61, 0, 12)}


def oracle_sample(wl="glass_L16_R5000", n_temps=None, procs=None):
    """The oracle as it stands on all host cores: each process anneals one run
    of the workload (population capped for the largest workloads) through its
    first n_temps temperatures."""
    procs = procs or os.cpu_count() or 1
    nt, r_max, reps = ORACLE_SAMPLE[wl]
    n_temps = n_temps or nt
    descs = _workload_descs(wl)
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_job, [([descs[(k * reps + q) % len(descs)] for q in range(reps)], n_temps, r_max)
                                     for k in range(procs)])
    wall = time.perf_counter() - t0
    upd = sum(u for u, _ in res)
    cap = f", populations capped at R={r_max}" if r_max else ""
    unit = metric_unit(wl)[1]
    return {"value": upd / (wall * 1e9), "unit": unit, "cores": procs, "kind": "oracle",
            "sample": f"{procs * reps} runs of the workload ({reps} per process) through their first {n_temps} "
                      f"temperatures{cap} ({upd:.3e} {unit.split('/')[0]}, {wall:.1f} s wall)"}


# ---------------------------------------------------------------- clocks
class Clocks:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 7:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[3 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# Sections of the kernel file each roofline kernel compiles from (beside the
# shared header and the helpers before the resampling section).
KERNEL_SECTIONS = {"sweep": (b"// Fused gather + theta checkerboard", b"// Overlaps (Sec. III.D)"),
                   "measure": (b"// Measurement (Sec. III.B", b"// A record's 128-bit sum as a double")}


def source_sha(kernel):
    """Hash of the source a kernel compiles from: the shared header, the shared
    helpers at the top of the kernel file and the kernel's own section."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2207_05535_gb300", "csrc")
    with open(os.path.join(csrc, "pa_internal.cuh"), "rb") as f:
        head = f.read()
    with open(os.path.join(csrc, "pa_kernels.cu"), "rb") as f:
        body = f.read()
    a, b = KERNEL_SECTIONS[kernel]
    common = body[:body.find(b"// Resampling (Sec. II.B")]
    return hashlib.sha256(head + common + body[body.find(a):body.find(b)]).hexdigest()[:16]


def measured_traffic(kernel, wl):
    """DRAM bytes per launch from an ncu capture, or None when the kernel's
    source changed since the capture (or it was taken on another workload)."""
    for t in TRAFFIC:
        if t["kernel"] == kernel and t["workload"] == wl and source_sha(kernel) == t["source_sha256_16"]:
            return t["bytes_per_launch"]
    return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------- main
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        W_, K = args.warmup, args.steps
        nt = ORACLE_SAMPLE[args.workload][0]
        for _ in range(W_):
            oracle_sample(args.workload, n_temps=2)
        vals, tot = [], 0.0
        for _ in range(K):
            t0 = time.perf_counter()
            s = oracle_sample(args.workload, n_temps=max(2, min(nt, 4)))
            tot += time.perf_counter() - t0
            vals.append(s["value"])
        v = statistics.median(vals)
        print(json.dumps({
            "impl": "reference", "metric": metric_unit(args.workload)[0], "value": v,
            "unit": metric_unit(args.workload)[1], "n_gpus": args.gpus, "steps": K,
            "warmup": W_, "ms_per_step": 1e3 * tot / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32/f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "name": args.workload,
                       "sample": "bounded oracle sample per step"},
            "cpu_baseline": {"value": v, "unit": metric_unit(args.workload)[1], "cores": s["cores"], "kind": "oracle",
                             "sample": s["sample"]},
            "e2e": {"value": v, "unit": metric_unit(args.workload)[1], "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}), flush=True)
        return

    # CPU baseline first: a spawn pool, before any CUDA context exists
    cpu = None
    if rank == 0 and world >= 1 and args.gpus == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(args.workload)

    import numpy as np
    import torch
    from paper_2207_05535_gb300 import _lib, build
    from paper_2207_05535_gb300 import workloads as W

    build.build()
    _lib.load()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    wl = args.workload
    if wl == "serving":
        return serving_main(args, rank, world, cpu)
    if wl in TEMPERATURE_STEP:
        return temperature_main(args, rank, world, local, cpu, dist, barrier)
    # weak scaling: every rank anneals its own batch (disorder samples / runs offset by rank)
    if wl == "glass_L16_R5000":
        descs, M_avg = W.glass_L16_R5000(n_samples=args.samples), 2
    elif wl == "ising_L8_R500":
        descs = W.ising_L8_R500(M=args.runs or 20)
        M_avg = len(descs)
    elif wl == "uneven_4096":
        descs, M_avg = W.batched_uneven(n_runs=args.runs or 4096), 0
    elif wl == "ferro_L8_theta_inf":
        descs, M_avg = _workload_descs(wl, args.runs), 20
    else:
        descs = W.ising_L256_R1e5(M=args.runs or 16)
        M_avg = len(descs)
    if args.max_temps:
        for d in descs:
            d.betas = d.betas[:args.max_temps]
    if args.wang:  # add Wang et al.'s pairing (Sec. III.D) to every run's overlap measurements
        for d in descs:
            d.overlap |= W.Q_WANG
    from paper_2207_05535_gb300 import replicas
    descs = replicas.shard(descs, rank)
    n_ticks = max(d.n_beta for d in descs) - 1
    idx = np.arange(len(descs), dtype=np.uint32)
    stream = torch.cuda.Stream()
    eng = _lib.Engine(descs, stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)

    def one_step(use_graph=True):
        eng.reset()
        eng.step(n_ticks, use_graph)
        if M_avg:
            return eng.weighted_average(idx, M_avg, 0)
        eng.sync()

    for _ in range(args.warmup):
        one_step()
    eng.sync()

    # ---- timed region: K whole anneals, device-timed, L2 flushed between steps
    clocks = Clocks(local) if rank == 0 else None
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = eng.launches
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            ev[k][0].record(stream)
        one_step()
        ev[k][1].record(stream)
    barrier()
    launches = eng.launches - l0
    ms = sum(a.elapsed_time(b) for a, b in ev)
    clk = clocks.stop() if clocks else None
    updates = 0
    runs_done = 0
    for k in range(len(descs)):
        rec = eng.records(k)
        updates += int(sum(work_units(descs[k], int(r)) for r in rec["R"][1:]))
        runs_done += 1
    t_max, upd_all = replicas.reduce_timing(ms, updates * args.steps, dist, device="cuda")
    value = upd_all / (t_max * 1e6)
    runs_per_s = world * runs_done * args.steps / (t_max / 1e3)

    # ---- per-kernel device time (eager launches bracketed by events), same work
    _lib.pa_set_profiling(eng.h, True)
    kt_tot = {}
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        _lib.pa_kernel_times(eng.h)
        one_step(use_graph=False)
        for kk, (t, n) in _lib.pa_kernel_times(eng.h).items():
            a, b = kt_tot.get(kk, (0.0, 0))
            kt_tot[kk] = (a + t, b + n)
    _lib.pa_set_profiling(eng.h, False)
    sweep_ms, sweep_n = kt_tot["sweep"]
    small_ms = kt_tot.get("small", (0.0, 0))[0]
    small = small_ms > sweep_ms  # runs on the one-launch-per-step path: its kernel holds the sweeps
    if small:
        sweep_ms = small_ms
    pk, pk_kind = peaks()
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    peak_tops = 152 * MULADD_LANES_PER_SM * sm_mhz * 1e6 / 1e12  # integer multiply-add slots, T/s
    # the multiplier roof, checked live: Philox4x32-10 alone (40 multiply-add slots per call)
    cal = {"calls_per_s_split": _lib.pa_calibrate_philox(False), "calls_per_s_wide": _lib.pa_calibrate_philox(True)}
    cal["frac_of_peak_split"] = cal["calls_per_s_split"] * 40 / (peak_tops * 1e12)
    inf = wl in INF_WORKLOADS
    slots = ALGO_MULADD_PER_DRAW if inf else ALGO_MULADD_PER_UPDATE
    achieved_tops = updates * slots / (sweep_ms / args.steps * 1e-3) / 1e12
    metric, unit = metric_unit(wl)
    total_kernel_ms = sum(t for t, _ in kt_tot.values())
    sweep_roof = {"bound": "alu", "kernel": "dos_sample_kernel" if inf else
                  ("anneal_small_kernel (resampling, sweeps and measurement of a step)" if small else "sweep_pow2_kernel"),
                  "achieved": achieved_tops, "peak": peak_tops, "unit": "Tmuladd/s", "frac": achieved_tops / peak_tops,
                  "traffic": None if inf or small else measured_traffic("sweep", wl),
                  "basis": (f"{ALGO_MULADD_PER_DRAW:g} integer multiply-add slots per energy draw "
                            f"(one Philox4x32-10 call)" if inf else
                            f"{ALGO_MULADD_PER_UPDATE:g} integer multiply-add slots per attempted update "
                            f"(Philox4x32-10: 40 per call, 4 updates per call)") + "; peak = 152 SMs x "
                           f"{MULADD_LANES_PER_SM} lanes x {sm_mhz:g} MHz, clock from MEASURED_PEAKS.json "
                           f"({pk_kind})",
                  "updates_per_ns_sweep_only": updates / (sweep_ms / args.steps * 1e-3) / 1e9,
                  "sweep_ms_per_step": sweep_ms / args.steps,
                  "sweep_share_of_kernel_time": sweep_ms / total_kernel_ms if total_kernel_ms else None,
                  "philox_calibration": cal}
    # HBM rooflines of the measurement and the nearest-integer resampling (algorithmic bytes per anneal)
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    meas_bytes = res_bytes = 0
    for k, d in enumerate(descs):
        Rs = eng.records(k)["R"].astype(np.int64)
        meas_bytes += 12 * int(Rs.sum())
        if d.resample != W.MULTINOMIAL:
            res_bytes += int(12 * Rs[:-1].sum() + 4 * Rs[1:].sum())

    def hbm_roof(name, key, nbytes, traffic, basis):
        ms_ = kt_tot.get(key, (0.0, 0))[0] / args.steps
        if not ms_ or not nbytes:
            return None
        ach = nbytes / (ms_ * 1e-3) / 1e9
        return {"bound": "hbm", "kernel": name, "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": traffic, "bytes_per_step": nbytes, "ms_per_step": ms_,
                "basis": basis + f"; peak = HBM copy bandwidth from MEASURED_PEAKS.json ({pk_kind})"}

    # small runs are measured inside their own step kernel (anneal_small_kernel);
    # measure_kernel then runs only at beta_0
    roof_meas = None if small else hbm_roof("measure_kernel", "measure", meas_bytes,
                                                      measured_traffic("measure", wl),
                                                      "12 B read per measured replica (E, M, family)")
    roof_res = hbm_roof("resample_counts_kernel + resample_parents_kernel", "resample", res_bytes, None,
                        "per parent: E read, copy number written and read back (12 B); per child: its parent "
                        "index written (4 B)")
    dominant = max(("sweep", "measure", "resample", "small") if roof_meas else ("sweep", "resample", "small"),
                   key=lambda k_: kt_tot.get(k_, (0.0, 0))[0])
    dominant = "sweep" if dominant == "small" else dominant
    roofline = {"sweep": sweep_roof, "measure": roof_meas, "resample": roof_res}[dominant] or sweep_roof
    # overlap kernels (a10): HBM-bound; algorithmic bytes = both replicas' colour planes per pair
    ov_ms = kt_tot.get("overlap", (0.0, 0))[0] / args.steps
    ov_bytes = 0
    for k, d in enumerate(descs):
        if d.overlap:
            rec = eng.records(k)
            per_replica = 2 * plane_words(d.L) * 4
            ov_bytes += int(np.sum(2 * rec["n_q"].astype(np.int64) + rec["n_q_pair"] + 2 * rec["n_q_wang"])) * per_replica
    # resampling copy (a7), fused into the sweep's prologue: every child reads its parent's colour
    # planes and E, M, family and writes its own, plus its parent index
    gather_bytes = 0
    for k, d in enumerate(descs):
        if d.theta == 0xFFFFFFFF:
            continue
        rec = eng.records(k)
        gather_bytes += int(np.sum(rec["R"][1:].astype(np.int64))) * (2 * 2 * plane_words(d.L) * 4 + 2 * 12 + 4)
    gather = {"bytes_per_step": gather_bytes,
              "GBps_within_sweep": gather_bytes / (sweep_ms / args.steps * 1e-3) / 1e9 if sweep_ms else None,
              "basis": "children x (parent planes read + child planes written + 12 B E/M/family each way + "
                       "4 B parent index); the copy is fused into the sweep kernel, so its rate is per sweep time"}
    roof_ov = None
    if ov_ms > 0 and ov_bytes:
        ach = ov_bytes / (ov_ms * 1e-3) / 1e9
        roof_ov = {"bound": "hbm", "kernel": "overlap_kernel" + (" + wang_kernel" if args.wang else ""),
                   "achieved": ach, "peak": float(pk.get("hbm_gbs", 6800.0)), "unit": "GB/s",
                   "frac": ach / float(pk.get("hbm_gbs", 6800.0)), "bytes_per_step": ov_bytes,
                   "basis": "2 replicas x 2 colour planes read per overlap pair; peak = HBM copy bandwidth from "
                            f"MEASURED_PEAKS.json ({pk_kind})"}

    # ---- plain form: one run per engine, all on one stream (one run per launch)
    plain = None
    if not args.no_plain and rank == 0:
        import dataclasses
        # one run (one disorder sample of two paired populations for the glass) per engine and per launch
        if wl == "glass_L16_R5000":
            units = [[dataclasses.replace(descs[2 * smp + p_], paired=1 - p_) for p_ in range(2)] for smp in range(10)]
        else:
            units = [[dataclasses.replace(d)] for d in descs[:min(len(descs), 20)]]
        engines = [_lib.Engine(u, stream.cuda_stream) for u in units]
        for e in engines:
            e.reset()
            e.step(n_ticks, False)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for e in engines:
            e.reset()
            e.step(n_ticks, False)
        b.record(stream)
        torch.cuda.synchronize()
        pms = a.elapsed_time(b)
        pupd, nruns = 0, 0
        for u, e in zip(units, engines):
            for k, d_ in enumerate(u):
                rec = e.records(k)
                pupd += int(sum(work_units(d_, int(r)) for r in rec["R"][1:]))
                nruns += 1
        for e in engines:
            e.close()
        plain = {"value": pupd / (pms * 1e6), "unit": unit, "runs": nruns, "runs_per_s": nruns / (pms / 1e3),
                 "form": "one run (glass: one disorder sample of two populations) per engine and per launch, "
                         "no graph, one stream"}

    # ---- end to end through the C ABI: host descriptors in, host results out
    e2e = None
    if not args.no_e2e:
        es = []
        h2d = d2h = 0
        for k in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e = _lib.Engine(descs, stream.cuda_stream)
            e.step(n_ticks, True)
            if M_avg:
                e.weighted_average(idx, M_avg, 0)
            for r in range(len(descs)):
                e.records(r)
            a_, b_ = _lib.pa_transfer_bytes(e.h)
            e.close()
            es.append(time.perf_counter() - t0)
            h2d, d2h = a_, b_
        e2e = {"value": updates * world / (statistics.median(es) * 1e9), "unit": unit,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "includes": "pa_create (allocation, table upload, beta_0 draw) + anneal + weighted averages + "
                           "all records copied to host + pa_destroy"}

    if rank == 0:
        out = {
            "metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32/f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[wl] + ("; plus Wang pairing overlaps" if args.wang else ""), "name": wl, "runs_per_gpu": len(descs), "temperatures": n_ticks + 1,
                       ("energy_draws_per_step" if inf else "attempted_updates_per_step"): updates,
                       "l2": "flushed between steps (256 MB write)",
                       "form": "batched: all runs share each launch; small runs (L <= 32, no overlaps) anneal in one "
                               "launch per lattice size, the others in one CUDA graph replay per temperature",
                       "parallelism": f"replicas x{world} (independent runs per GPU)"},
            "runs_per_s": runs_per_s,
            "roofline": roofline,
            "roofline_sweep": sweep_roof if roofline is not sweep_roof else None,
            "roofline_measure": roof_meas,
            "roofline_resample": roof_res,

            "roofline_overlap": roof_ov,
            "resample_gather": gather,
            "kernel_ms_per_step": {k: t / args.steps for k, (t, n) in kt_tot.items()},
            "sweep_shapes": [{"L": L_, "words_per_thread": w_, "block": b_, "autotuned": bool(t_)}
                             for (L_, w_, b_, t_) in _lib.pa_sweep_shapes(eng.h)],
            "gpu_launches": launches,
            "clocks": clk,
            "plain": plain,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out), flush=True)
    eng.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def sweep_roofline(kernel, updates, sweep_ms, total_kernel_ms, traffic):
    """The sweep against the integer-multiplier roof: 10 multiply-add slots per
    attempted update over the sweep's CUDA-event time, plus the live Philox-only
    calibration of that roof."""
    from paper_2207_05535_gb300 import _lib
    pk, pk_kind = peaks()
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    peak_tops = 152 * MULADD_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    cal = {"calls_per_s_split": _lib.pa_calibrate_philox(False), "calls_per_s_wide": _lib.pa_calibrate_philox(True)}
    cal["frac_of_peak_split"] = cal["calls_per_s_split"] * 40 / (peak_tops * 1e12)
    achieved = updates * ALGO_MULADD_PER_UPDATE / (sweep_ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak_tops, "unit": "Tmuladd/s",
            "frac": achieved / peak_tops, "traffic": traffic,
            "basis": f"{ALGO_MULADD_PER_UPDATE:g} integer multiply-add slots per attempted update (Philox4x32-10: "
                     f"40 per call, 4 updates per call); peak = 152 SMs x {MULADD_LANES_PER_SM} lanes x {sm_mhz:g} MHz, "
                     f"clock from MEASURED_PEAKS.json ({pk_kind})",
            "updates_per_ns_sweep_only": updates / (sweep_ms * 1e-3) / 1e9, "sweep_ms_per_step": sweep_ms,
            "sweep_share_of_kernel_time": sweep_ms / total_kernel_ms if total_kernel_ms else None,
            "philox_calibration": cal}


def hbm_roofline(name, nbytes, ms, traffic, basis):
    pk, pk_kind = peaks()
    if not ms or not nbytes:
        return None
    hbm = float(pk.get("hbm_gbs", 6800.0))
    ach = nbytes / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": name, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": traffic, "bytes_per_step": nbytes, "ms_per_step": ms,
            "basis": basis + f"; peak = HBM copy bandwidth from MEASURED_PEAKS.json ({pk_kind})"}


def step_units(descs, recs_R, temps):
    """Attempted updates of temperatures `temps` (indices into each run's records)."""
    tot = 0
    for d, R in zip(descs, recs_R):
        for t in temps:
            tot += work_units(d, int(R[t]))
    return tot


def temperature_main(args, rank, world, local, cpu, dist, barrier):
    """One step = one temperature of the whole batch; the warm-up and the timed
    steps walk the schedule (a reset between steps, untimed, when it ends)."""
    import dataclasses
    import numpy as np
    import torch
    from paper_2207_05535_gb300 import _lib, replicas
    from paper_2207_05535_gb300 import workloads as W
    wl = args.workload
    descs = W.batched_uneven(n_runs=args.runs or 4096) if wl == "uneven_4096" else \
        W.ising_L256_R1e5(M=args.runs or 16)
    descs = replicas.shard(descs, rank)
    n_ticks = max(d.n_beta for d in descs) - 1
    K, Wm = args.steps, args.warmup
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)
    eng = _lib.Engine(descs, stream.cuda_stream)
    every = np.arange(len(descs), dtype=np.uint32)
    cur = [0]  # temperature index every run has reached

    def fit(n):  # make room for n more temperatures in this pass (untimed reset otherwise)
        if cur[0] + n > n_ticks:
            eng.reset()
            eng.sync()
            cur[0] = 0

    def R_of_steps():
        return [eng.records(k)["R"] for k in range(len(descs))]

    # warm-up: the first steps of each lattice size also time its candidate sweep shapes
    # (pa_tuning_pending); then W more steps, all walking the schedule
    tuning_steps = 0
    while _lib.pa_tuning_pending(eng.h) and tuning_steps < n_ticks:
        fit(1)
        eng.step(1, True)
        cur[0] += 1
        tuning_steps += 1
    for _ in range(Wm):
        fit(1)
        eng.step(1, True)
        cur[0] += 1
    eng.sync()
    fit(K)
    first = cur[0] + 1

    # ---- timed region: K temperatures, device-timed, L2 flushed before each
    clocks = Clocks(local) if rank == 0 else None
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    l0 = eng.launches
    for k in range(K):
        with torch.cuda.stream(stream):
            flush.zero_()
            ev[k][0].record(stream)
        eng.step(1, True)
        ev[k][1].record(stream)
    barrier()
    launches = eng.launches - l0
    cur[0] += K
    ms = sum(a.elapsed_time(b) for a, b in ev)
    clk = clocks.stop() if clocks else None
    temps = list(range(first, first + K))
    Rs = R_of_steps()
    updates = step_units(descs, Rs, temps)
    t_max, upd_all = replicas.reduce_timing(ms, updates, dist, device="cuda")
    value = upd_all / (t_max * 1e6)

    # ---- per-kernel device time: eager launches bracketed by events, the next temperatures
    Kp = min(K, 5)
    fit(Kp)
    p_first = cur[0] + 1
    _lib.pa_set_profiling(eng.h, True)
    _lib.pa_kernel_times(eng.h)
    for k in range(Kp):
        with torch.cuda.stream(stream):
            flush.zero_()
        eng.step(1, False)
    kt = _lib.pa_kernel_times(eng.h)
    _lib.pa_set_profiling(eng.h, False)
    cur[0] += Kp
    Rp = R_of_steps()
    p_temps = list(range(p_first, p_first + Kp))
    p_updates = step_units(descs, Rp, p_temps)
    kt_step = {k_: t / Kp for k_, (t, n) in kt.items()}
    total_kernel_ms = sum(kt_step.values())
    sweep_roof = sweep_roofline("sweep_pow2_kernel", p_updates / Kp, kt_step["sweep"], total_kernel_ms,
                                measured_traffic("sweep", wl))
    meas_bytes = 12 * sum(int(R[t]) for R in Rp for t in p_temps) // Kp
    res_bytes = sum(12 * int(R[t - 1]) + 4 * int(R[t]) for R in Rp for t in p_temps) // Kp
    roof_meas = hbm_roofline("measure_kernel", meas_bytes, kt_step.get("measure"), measured_traffic("measure", wl),
                             "12 B read per measured replica (E, M, family)")
    roof_res = hbm_roofline("resample_counts_kernel + resample_parents_kernel", res_bytes, kt_step.get("resample"),
                            None, "per parent: E read, copy number written and read back (12 B); per child: its "
                                  "parent index written (4 B)")
    gather_bytes = sum(int(R[t]) * (2 * 2 * plane_words(d.L) * 4 + 2 * 12 + 4)
                       for d, R in zip(descs, Rp) for t in p_temps) // Kp
    gather = {"bytes_per_step": gather_bytes, "GBps_within_sweep": gather_bytes / (kt_step["sweep"] * 1e-3) / 1e9,
              "basis": "children x (parent planes read + child planes written + 12 B E/M/family each way + 4 B "
                       "parent index); the copy is fused into the sweep kernel, so its rate is per sweep time"}
    shapes = [{"L": L_, "words_per_thread": w_, "block": b_, "autotuned": bool(t_)}
              for (L_, w_, b_, t_) in _lib.pa_sweep_shapes(eng.h)]
    eng.close()
    del flush

    # ---- plain form: 20 of the runs, one engine (one run) each, eager launches, one after another
    plain = None
    if not args.no_plain and rank == 0:
        units = descs[:min(len(descs), 20)]
        engines = [_lib.Engine([dataclasses.replace(d)], stream.cuda_stream) for d in units]
        for e in engines:
            for _ in range(min(Wm, n_ticks - K)):
                e.step(1, False)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for k in range(K):
            for e in engines:
                e.step(1, False)
        b.record(stream)
        torch.cuda.synchronize()
        pms = a.elapsed_time(b)
        p0 = min(Wm, n_ticks - K) + 1
        pupd = step_units(units, [e.records(0)["R"] for e in engines], range(p0, p0 + K))
        for e in engines:
            e.close()
        plain = {"value": pupd / (pms * 1e6), "unit": UNIT, "runs": len(units),
                 "form": "20 of the batch's runs, one engine and eager launch sequence per run, one after another, "
                         "the same number of temperatures"}

    # ---- end to end through the C ABI: host descriptors in, every run's record of each step out
    e2e = None
    if not args.no_e2e:
        pinned = torch.empty(len(descs) * _lib.RECORD_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
        host = pinned.numpy().view(_lib.RECORD_DTYPE)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e = _lib.Engine(descs, stream.cuda_stream)
        for k in range(K):
            e.step(1, True)
            e.step_records(every, host)
        wall = time.perf_counter() - t0
        h2d, d2h = _lib.pa_transfer_bytes(e.h)
        eupd = step_units(descs, [e.records(k)["R"] for k in range(len(descs))], range(1, K + 1))
        e.close()
        e2e = {"value": eupd * world / (wall * 1e9), "unit": UNIT, "h2d_bytes_per_step": h2d / K,
               "d2h_bytes_per_step": d2h / K,
               "includes": "pa_create from host descriptors (pool allocation, descriptor/schedule/table uploads, "
                           "beta_0 draw) + K anneal steps, each followed by pa_step_records of every run into pinned "
                           "host memory; wall clock"}

    extra = None
    if rank == 0 and world == 1 and not args.no_extra:
        extra = {w_: small_workload(w_, stream) for w_ in ("ising_L8_R500", "glass_L16_R5000")}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
            "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32/f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[wl], "name": wl, "runs_per_gpu": len(descs),
                       "temperatures": n_ticks + 1, "step": "one temperature of the whole batch",
                       "tuning_steps_before_warmup": tuning_steps,
                       "timed_temperatures": [temps[0], temps[-1]], "attempted_updates_timed": updates,
                       "l2": "inputs larger than L2 (about 120 GB of populations) and a 256 MB write before each step",
                       "form": "batched: all runs in one launch per kernel, each temperature one CUDA graph replay",
                       "parallelism": f"replicas x{world} (independent runs per GPU)"},
            "roofline": sweep_roof, "roofline_measure": roof_meas, "roofline_resample": roof_res,
            "resample_gather": gather, "kernel_ms_per_step": kt_step, "sweep_shapes": shapes,
            "gpu_launches": launches, "clocks": clk, "plain": plain, "e2e": e2e, "cpu_baseline": cpu,
            "extra": extra,
        }
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def small_workload(wl, stream, K=3, Wm=2):
    """Device-timed value of a small workload (one step = one whole anneal of its
    batch, graph replays) beside its plain form (one run, or one disorder sample
    of two populations, per engine; eager launches)."""
    import dataclasses
    import numpy as np
    import torch
    from paper_2207_05535_gb300 import _lib
    from paper_2207_05535_gb300 import workloads as W
    descs = W.ising_L8_R500(M=20) if wl == "ising_L8_R500" else W.glass_L16_R5000()
    n_ticks = max(d.n_beta for d in descs) - 1
    eng = _lib.Engine(descs, stream.cuda_stream)
    for _ in range(Wm):
        eng.reset()
        eng.step(n_ticks, True)
    eng.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    for _ in range(K):
        eng.reset()
        eng.sync()
        a.record(stream)
        eng.step(n_ticks, True)
        b.record(stream)
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
    upd = sum(work_units(d, int(r)) for k, d in enumerate(descs) for r in eng.records(k)["R"][1:]) * K
    eng.close()
    if wl == "glass_L16_R5000":
        units = [[dataclasses.replace(descs[2 * s_ + p_], paired=1 - p_) for p_ in range(2)] for s_ in range(10)]
    else:
        units = [[dataclasses.replace(d)] for d in descs]
    engines = [_lib.Engine(u, stream.cuda_stream) for u in units]
    for e in engines:
        e.step(n_ticks, False)
        e.reset()
    torch.cuda.synchronize()
    a.record(stream)
    for e in engines:
        e.step(n_ticks, False)
    b.record(stream)
    torch.cuda.synchronize()
    pms = a.elapsed_time(b)
    pupd = sum(work_units(d, int(r)) for u, e in zip(units, engines) for k, d in enumerate(u)
               for r in e.records(k)["R"][1:])
    for e in engines:
        e.close()
    return {"workload": WORKLOADS[wl], "value": upd / (ms * 1e6), "unit": UNIT, "anneals_timed": K,
            "ms_per_anneal": ms / K, "plain": pupd / (pms * 1e6),
            "form": "batched: all runs share each launch (small runs: one launch for the whole anneal; the others: "
                    "one CUDA graph replay per temperature); plain: one run "
                    "(glass: one disorder sample of two populations) per engine, eager launches"}


def serving_main(args, rank, world, cpu):
    """The serving workload: a Poisson stream through one continuous-batching server."""
    import dataclasses
    import numpy as np
    import torch
    from paper_2207_05535_gb300 import _lib, serve
    from paper_2207_05535_gb300 import workloads as W
    stream = torch.cuda.Stream()
    cfg = serve.config_for_budget(64 << 30)
    arrivals = W.serving_stream(rate=args.rate, duration=args.window, seed=11 + 1000 * rank)
    # warm-up: a short stream (tunes the sweep shapes of the lattice sizes it meets)
    warm = W.serving_stream(duration=0.2, seed=99)
    for _ in range(max(1, args.warmup)):
        srv = serve.Server(cfg, stream.cuda_stream)
        serve.serve([(0.0, d) for _, d in warm], srv)
        srv.close()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0"))) if rank == 0 else None
    torch.cuda.synchronize()
    srv = serve.Server(cfg, stream.cuda_stream)
    l0 = _lib.pa_launch_count(srv.h)
    done, st = serve.serve(arrivals, srv)
    torch.cuda.synchronize()
    launches = _lib.pa_launch_count(srv.h) - l0
    srv.close()
    clk = clocks.stop() if clocks else None
    summ = serve.summarize(done, st["wall_s"])
    # plain form: the first 20 jobs one after another, one engine each
    plain = None
    if not args.no_plain:
        t0 = time.perf_counter()
        upd = 0
        for _, d in arrivals[:20]:
            e = _lib.Engine([dataclasses.replace(d)], stream.cuda_stream)
            e.run_to_end(False)
            rec = e.records(0)
            upd += int(sum(d.theta * d.N * int(r) for r in rec["R"][1:]))
            e.close()
        pt = time.perf_counter() - t0
        plain = {"value": upd / (pt * 1e9), "unit": UNIT, "runs": 20, "runs_per_s": 20 / pt,
                 "form": "the first 20 jobs one after another, one engine and launch sequence each"}
    sweep = None
    if args.rates:
        sweep = rate_sweep([float(x) for x in args.rates.split(",")], args.window, cfg, stream, rank)
    out = {"metric": METRIC, "value": summ["updates_per_ns"], "unit": UNIT, "n_gpus": world, "steps": 1,
           "warmup": args.warmup, "ms_per_step": 1e3 * st["wall_s"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "int32/f64", "data": "synthetic",
           "config": {"workload": WORKLOADS["serving"].replace("200/s", f"{args.rate:g}/s"), "name": "serving",
                      "window_s": args.window, "jobs": len(arrivals),
                      "form": "continuous batching (admit/retire between steps)"},
           "rate_sweep": sweep,
           "serving": summ, "runs_per_s": summ["jobs_per_s"], "gpu_launches": launches, "clocks": clk,
           "plain": plain, "cpu_baseline": cpu,
           "e2e": {"value": summ["updates_per_ns"], "unit": UNIT, "h2d_bytes_per_step": None,
                   "d2h_bytes_per_step": None, "includes": "wall clock of the whole stream: admissions "
                   "(descriptor and table uploads), steps, record copies, retirements"}}
    if rank == 0:
        print(json.dumps(out), flush=True)


def serve_rate(rate, window, cfg, stream, seed):
    """One Poisson stream at `rate` jobs/s for `window` s through a fresh server."""
    import numpy as np
    from paper_2207_05535_gb300 import serve
    from paper_2207_05535_gb300 import workloads as W
    arrivals = W.serving_stream(rate=rate, duration=window, seed=seed)
    srv = serve.Server(cfg, stream.cuda_stream)
    done, st = serve.serve(arrivals, srv)
    srv.close()
    summ = serve.summarize(done, st["wall_s"])
    by_arrival = sorted(done, key=lambda j: j.arrival)
    third = max(1, len(by_arrival) // 3)
    lat_first = float(np.mean([j.finished - j.arrival for j in by_arrival[:third]]))
    lat_last = float(np.mean([j.finished - j.arrival for j in by_arrival[-third:]]))
    summ.update(rate=rate, offered_jobs=len(arrivals), mean_latency_first_third_s=lat_first,
                mean_latency_last_third_s=lat_last,
                sustained=bool(summ["jobs_per_s"] >= 0.9 * rate and lat_last <= 1.5 * lat_first + 0.5))
    return summ


def rate_sweep(rates, window, cfg, stream, rank):
    """Largest sustainable arrival rate: the server keeps up (completion rate near
    the offered rate, latencies not growing over the window); then latencies at
    50 % and 80 % of it."""
    points = [serve_rate(r, window, cfg, stream, 21 + 1000 * rank) for r in sorted(rates)]
    ok = [p["rate"] for p in points if p["sustained"]]
    lam = max(ok) if ok else None
    at = {}
    if lam:
        for f in (0.5, 0.8):
            at[f"{int(f * 100)}%"] = serve_rate(f * lam, window, cfg, stream, 21 + 1000 * rank)
        at["100%"] = next(p for p in points if p["rate"] == lam)
    return {"points": points, "max_sustainable_rate": lam, "at_fraction_of_max": at,
            "criterion": "kept up: jobs finished per second of the whole stream (arrival window and drain) >= 0.9 x "
                         "the offered rate, and the mean latency of the last third of the arrivals <= 1.5 x that of "
                         "the first third + 0.5 s (no growing backlog)"}


if __name__ == "__main__":
    main()
