"""Run a synthetic batch of population-annealing runs on the GPU and print its
throughput.

    python -m paper_2207_05535_gb300.run --L 30 --runs 40 --R 10000 --temps 8 [--model fm|glass|mixed] [--wang]

Runs are independent (run_id = 0..runs-1, disorder_id = run_id), theta sweeps
per temperature, beta from 0 to --beta-f in --temps equidistant steps.
"""
from __future__ import annotations

import argparse
import json
import time

from . import _lib, build
from . import workloads as W


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=16)
    ap.add_argument("--runs", type=int, default=8)
    ap.add_argument("--R", type=int, default=1000)
    ap.add_argument("--temps", type=int, default=11)
    ap.add_argument("--theta", type=int, default=10)
    ap.add_argument("--beta-f", type=float, default=1.0)
    ap.add_argument("--model", default="mixed", choices=["fm", "glass", "mixed"])
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--generic", action="store_true", help="byte-plane sweep kernel for every size")
    ap.add_argument("--wang", action="store_true", help="measure overlaps of Wang pairs (Sec. III.D)")
    a = ap.parse_args(argv)
    build.build()
    model = {"fm": lambda k: W.FERRO, "glass": lambda k: W.EA_PMJ, "mixed": lambda k: k % 2}[a.model]
    descs = [W.RunDesc(a.L, model(k), a.R, a.theta, W.schedule(a.beta_f, a.temps), run_id=k, disorder_id=k,
                       overlap=W.Q_WANG if a.wang else W.Q_NONE)
             for k in range(a.runs)]
    flags = (_lib.PA_CREATE_NO_AUTOTUNE if a.no_autotune else 0) | (_lib.PA_CREATE_GENERIC_SWEEP if a.generic else 0)
    t0 = time.perf_counter()
    with _lib.Engine(descs, flags=flags) as eng:
        eng.run_to_end(use_graph=False)
        wall = time.perf_counter() - t0
        upd = sum(int(sum(d.theta * d.N * int(r) for r in eng.records(k)["R"][1:])) for k, d in enumerate(descs))
        shapes = _lib.pa_sweep_shapes(eng.h)
    print(json.dumps({"updates": upd, "wall_s": wall, "updates_per_ns_wall": upd / wall / 1e9,
                      "sweep_shapes": shapes}))


if __name__ == "__main__":
    main()
