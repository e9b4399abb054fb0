"""Seeded synthetic workloads: run descriptors only.

This module holds no arithmetic of the method.  It builds the inputs that both
the CUDA engine and the CPU oracle consume: lattice size, model, population
size, sweeps, the annealing schedule and the Philox key material.  Every random
decision of the method itself is drawn inside each implementation from the
counter-based generator keyed by these fields.

Schedules are equidistant, beta_i = i * beta_f / (n - 1) for n temperatures
(Sec. V.A.2 uses beta_i = i * dbeta from beta_0 = 0).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FERRO = 0
EA_PMJ = 1
NEAREST = 0
MULTINOMIAL = 1
Q_NONE = 0
Q_SHIFT = 1
Q_PAIR = 2
Q_WANG = 4
THETA_INF = 0xFFFFFFFF  # theta -> infinity: energies drawn from the exact density of states (Sec. V.B)


def schedule(beta_f: float, n: int) -> np.ndarray:
    """n equidistant inverse temperatures from 0 to beta_f inclusive."""
    if n < 1:
        raise ValueError("n >= 1")
    if n == 1:
        return np.zeros(1)
    return np.array([i * beta_f / (n - 1) for i in range(n)], dtype=np.float64)


def default_cap(R: int) -> int:
    """Capacity for nearest-integer resampling: R + 8 sqrt(R) + 64."""
    return int(R + 8 * math.ceil(math.sqrt(R)) + 64)


@dataclasses.dataclass
class RunDesc:
    L: int
    model: int
    R: int
    theta: int
    betas: np.ndarray
    seed: int = 1
    run_id: int = 0
    disorder_id: int = 0
    resample: int = NEAREST
    overlap: int = Q_NONE
    paired: int = -1          # index (within the same batch) of the paired population
    R_cap: int = 0
    log_g: np.ndarray | None = None  # theta = THETA_INF: ln g(E) at E = 2u - 2N, u = 0..2N

    def __post_init__(self):
        self.betas = np.ascontiguousarray(self.betas, dtype=np.float64)
        if self.R_cap == 0:
            self.R_cap = self.R if self.resample == MULTINOMIAL else default_cap(self.R)

    @property
    def N(self) -> int:
        return self.L * self.L

    @property
    def n_beta(self) -> int:
        return len(self.betas)

    def updates(self) -> int:
        """Nominal attempted spin updates of the whole anneal (theta N R per step;
        none for theta = THETA_INF, where energies are drawn instead)."""
        if self.theta == THETA_INF:
            return 0
        return self.theta * self.N * self.R * (self.n_beta - 1)


def ferro_runs(L=8, R=500, theta=10, beta_f=0.5, n=51, M=20, seed=1, resample=NEAREST, first_run=0):
    """Independent ferromagnet runs (2D Ising, J = 1), run_id = first_run..first_run+M-1."""
    b = schedule(beta_f, n)
    return [RunDesc(L, FERRO, R, theta, b, seed, first_run + m, 0, resample) for m in range(M)]


def glass_pairs(L=16, R=5000, theta=10, beta_f=3.0, n=101, n_samples=100, seed=1, resample=NEAREST,
                overlap=Q_SHIFT | Q_PAIR):
    """+-J glass: disorder sample d holds two independent populations (run_id 2d, 2d+1)
    that are paired for the two-population overlap."""
    b = schedule(beta_f, n)
    runs = []
    for d in range(n_samples):
        for p in range(2):
            runs.append(RunDesc(L, EA_PMJ, R, theta, b, seed, 2 * d + p, d, resample, overlap,
                                paired=2 * d + (1 - p) if overlap & Q_PAIR else -1))
    return runs


# The five workloads, by what they are.
def ising_L8_R500(M=20):
    """2D Ising FM, L=8, R=500, beta 0->0.5 in 51 steps, theta=10, M=20 runs, seed 1."""
    return ferro_runs(L=8, R=500, theta=10, beta_f=0.5, n=51, M=M, seed=1)


def glass_L16_R5000(n_samples=100, R=5000, n=101):
    """2D +-J glass, L=16, R=5000, beta 0->3 in 101 steps, theta=10, 100 samples x 2 populations."""
    return glass_pairs(L=16, R=R, theta=10, beta_f=3.0, n=n, n_samples=n_samples, seed=1)


def batched_uneven(n_runs=4096, seed=7, n=101, beta_f=1.0, theta=10, Ls=(16, 32, 64, 128),
                   Rs=(1000, 10000, 50000)):
    """Independent ferromagnet runs with L and R drawn by seed (uneven batch)."""
    rng = np.random.default_rng(seed)
    b = schedule(beta_f, n)
    Lc = rng.choice(np.array(Ls), size=n_runs)
    Rc = rng.choice(np.array(Rs), size=n_runs)
    return [RunDesc(int(Lc[m]), FERRO, int(Rc[m]), theta, b, 1, m, 0) for m in range(n_runs)]


def ising_L256_R1e5(M=16, R=100000, n=201):
    """2D Ising FM, L=256, R=1e5, beta 0->0.44 in 201 steps, theta=20, M=16 runs."""
    return ferro_runs(L=256, R=R, theta=20, beta_f=0.44, n=n, M=M, seed=1)


def ferro_theta_inf(log_g, L=8, R=20000, beta_f=0.6, n=61, M=200, seed=1, resample=NEAREST):
    """theta = infinity ferromagnet runs (Sec. V.B): at every temperature each
    replica's energy is drawn from the exact distribution of the density of states
    log_g (ln g at E = 2u - 2N, u = 0..2N) instead of Metropolis sweeps."""
    b = schedule(beta_f, n)
    return [RunDesc(L, FERRO, R, THETA_INF, b, seed, m, 0, resample, log_g=log_g) for m in range(M)]


def serving_stream(rate=200.0, duration=10.0, seed=11, Lmin=8, Lmax=64, Rmin=1000, Rmax=50000, nmin=50,
                   nmax=300, theta=10):
    """Poisson arrivals of PA jobs: FM or glass with equal odds, L even uniform in
    [Lmin, Lmax], R log-uniform in [Rmin, Rmax], schedule lengths uniform in
    [nmin, nmax], beta_f = 1 (FM) or 3 (glass).  Returns [(arrival_s, RunDesc)]."""
    rng = np.random.default_rng(seed)
    t, out, m = 0.0, [], 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        model = int(rng.integers(0, 2))
        L = int(2 * rng.integers(Lmin // 2, Lmax // 2 + 1))
        R = int(round(math.exp(rng.uniform(math.log(Rmin), math.log(Rmax)))))
        n = int(rng.integers(nmin, nmax + 1))
        b = schedule(1.0 if model == FERRO else 3.0, n)
        out.append((t, RunDesc(L, model, R, theta, b, seed, m, m)))
        m += 1
    return out
