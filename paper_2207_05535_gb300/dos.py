"""Exact energy density of states of a periodic L x L Ising lattice (small L).

The theta -> infinity mode of Sec. V.B draws energies from the exact energy
distribution, which needs g(E).  This module counts states by unsatisfied bonds
u (E = 2u - 2N; a bond with coupling J between spins s, s' is unsatisfied when
J s s' = -1) with a site-by-site transfer matrix:

  - row 0 is fixed to each of its 2^L configurations in turn (periodic
    boundaries in y close on it at the end);
  - the state is one spin per column, the latest one added in that column; adding
    site (x, y) replaces column x, counting its bonds to the site above, to
    the site on its left, and at the row's and the lattice's last sites the
    periodic bonds back to column 0 and to row 0;
  - polynomial coefficients in u are non-negative float64 sums (relative error
    of a few ulp, no cancellation).

Cost is O(2^(2L) N^2): about a second for L = 6, a few seconds for L = 8.
Couplings are +1 for the ferromagnet; the +-J glass takes the caller's Jr, Jd
(site-order arrays of the right and down bonds).
"""
from __future__ import annotations

import math

import numpy as np


def count_unsatisfied(L: int, Jr=None, Jd=None) -> np.ndarray:
    """g over u = 0..2N (float64; exact up to rounding, sum 2^N)."""
    N = L * L
    Jr = np.ones(N, dtype=np.int8) if Jr is None else np.asarray(Jr, dtype=np.int8)
    Jd = np.ones(N, dtype=np.int8) if Jd is None else np.asarray(Jd, dtype=np.int8)
    if L < 2 or L > 10:
        raise ValueError("L must be in 2..10 for the transfer-matrix density of states")
    S = 1 << L
    U = 2 * N
    st = np.arange(S)
    bit = lambda a, x: (a >> x) & 1

    def unsat(a, b, J):  # bits a, b of two spins joined by coupling J
        diff = np.asarray(a) != np.asarray(b)
        return np.where(np.asarray(J) > 0, diff, ~diff).astype(np.int64)

    # row 0: the state is s0 itself; its horizontal bonds
    u0 = np.zeros(S, dtype=np.int64)
    for x in range(L):
        u0 += unsat(bit(st, x), bit(st, (x + 1) % L), Jr[x])
    V = np.zeros((S, S, U + 1))          # [s0, state, u]
    V[st, st, u0] = 1.0
    top = int(u0.max())                   # largest u reached so far
    for y in range(1, L):
        for x in range(L):
            n = y * L + x
            add_max = 2 + (x == L - 1) + (y == L - 1)
            Vn = np.zeros_like(V)
            for b in (0, 1):              # spin above, held in column x of the state
                src = st[bit(st, x) == b]
                for t in (0, 1):          # the new spin
                    dst = (src & ~(1 << x)) | (t << x)
                    k = unsat(b, t, Jd[(y - 1) * L + x]) * np.ones_like(src)
                    if x > 0:             # left neighbour (column x - 1, this row)
                        k = k + unsat(bit(src, x - 1), t, Jr[n - 1])
                    if x == L - 1:        # periodic bond to column 0 of this row
                        k = k + unsat(t, bit(src, 0), Jr[n])
                    if y < L - 1:
                        groups = [(V[None], Vn[None], 0)]
                    else:                 # periodic bond to row 0: split row-0 configurations by column x
                        shp = (S >> (x + 1), 2, 1 << x, S, U + 1)
                        groups = [(V.reshape(shp)[:, h], Vn.reshape(shp)[:, h], int(unsat(t, h, Jd[n])))
                                  for h in (0, 1)]
                    for Vg, Vng, extra in groups:  # views [s0 high bits, s0 low bits, state, u]
                        kt = k + extra
                        for kk in np.unique(kt):
                            kk = int(kk)
                            sel = kt == kk
                            w = min(top, U - kk) + 1
                            Vng[:, :, dst[sel], kk:kk + w] += Vg[:, :, src[sel], :w]
            V = Vn
            top = min(U, top + add_max)
    return V.sum(axis=(0, 1))


def log_dos(L: int, Jr=None, Jd=None) -> np.ndarray:
    """ln g(E) at E = 2u - 2N, u = 0..2N (-inf where g = 0): the layout the
    engine's theta = PA_THETA_INF descriptors take."""
    g = count_unsatisfied(L, Jr, Jd)
    out = np.full(len(g), -math.inf)
    nz = g > 0.5
    out[nz] = np.log(g[nz])
    return out
