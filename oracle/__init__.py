"""Plain CPU oracle for population annealing (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA engine.
"""
from .oracle import (  # noqa: F401
    ORACLE_LIB,
    OracleRun,
    build,
    bruteforce,
    bruteforce_moments,
    couplings,
    dos_transfer,
    energy,
    i128,
    wang_pairing,
    kaufman_lnZ,
    load,
    log_weights,
    metropolis_threshold,
    philox4x32_10,
    sweep_lattice,
    weighted_average,
    RECORD_DTYPE,
    WAVG_DTYPE,
    THETA_INF,
)
