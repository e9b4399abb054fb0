"""ctypes binding of the plain C oracle (``pa_oracle.c``).

Test infrastructure only: the CUDA engine never imports this module.  Every
function here marshals arguments; all arithmetic lives in ``pa_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pa_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
ORACLE_LIB = os.path.join(_BUILD, "libpa_oracle.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, IEEE FP64)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(ORACLE_LIB)
            and os.path.getmtime(ORACLE_LIB) >= os.path.getmtime(_SRC)):
        return ORACLE_LIB
    tmp = ORACLE_LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, ORACLE_LIB)
    return ORACLE_LIB


class Desc(C.Structure):
    _fields_ = [("L", C.c_uint32), ("model", C.c_uint32), ("R", C.c_uint32), ("R_cap", C.c_uint32),
                ("theta", C.c_uint32), ("n_beta", C.c_uint32), ("beta", C.POINTER(C.c_double)),
                ("seed", C.c_uint32), ("run_id", C.c_uint32), ("disorder_id", C.c_uint32),
                ("resample", C.c_uint32), ("overlap", C.c_uint32), ("log_g", C.POINTER(C.c_double))]


THETA_INF = 0xFFFFFFFF  # theta = infinity: energies drawn from the exact distribution (needs log_g)


RECORD_DTYPE = np.dtype([
    ("beta", "f8"), ("lnQ", "f8"), ("minus_betaF", "f8"),
    ("sumE", "i8"), ("sumE2", "i8"), ("sumAbsM", "i8"), ("sumM2", "i8"),
    ("sum_c2", "i8"), ("sum_absq", "i8"), ("sum_absq_pair", "i8"),
    ("R", "u4"), ("R_target", "u4"), ("n_fam", "u4"), ("max_fam", "u4"),
    ("n_q", "u4"), ("n_q_pair", "u4"), ("N", "u4"), ("status", "u4"),
    ("sumE3", "u8", (2,)), ("sumE4", "u8", (2,)), ("sumAbsM3", "u8", (2,)), ("sumM4", "u8", (2,)),
    ("sum_absq_wang", "i8"), ("n_q_wang", "u4"), ("wang_swaps", "u4"),
])

WAVG_DTYPE = np.dtype([
    ("beta", "f8"), ("W_e", "f8"), ("W_e2", "f8"), ("W_m", "f8"), ("W_m2", "f8"),
    ("Wvar_c", "f8"), ("Wvar_chi", "f8"), ("W_c", "f8"), ("W_chi", "f8"),
    ("W_minus_betaF", "f8"), ("W_absq", "f8"), ("W_absq_pair", "f8"),
    ("w_max", "f8"), ("sum_w", "f8"),
    ("W_e3", "f8"), ("W_e4", "f8"), ("W_m3", "f8"), ("W_m4", "f8"),
    ("Wk3_e", "f8"), ("Wk4_e", "f8"), ("Wk3_m", "f8"), ("Wk4_m", "f8"),
    ("W_U4", "f8"), ("W_U4_conf", "f8"), ("W_absq_wang", "f8"),
])


def i128(w):
    """A record's 128-bit sum (two uint64 words, low first, two's complement) as a Python int."""
    v = int(w[0]) | int(w[1]) << 64
    return v - (1 << 128) if v >> 127 else v


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = C.CDLL(ORACLE_LIB)
        u32, i32, f64 = C.c_uint32, C.c_int32, C.c_double
        P = C.POINTER
        lib.or_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
        lib.or_philox4x32_10.restype = None
        lib.or_energy.argtypes = [u32, P(C.c_int8), P(C.c_int8), P(C.c_int8)]
        lib.or_energy.restype = C.c_int64
        lib.or_couplings.argtypes = [u32, u32, u32, u32, P(C.c_int8), P(C.c_int8)]
        lib.or_couplings.restype = None
        lib.or_metropolis_threshold.argtypes = [f64, C.c_int]
        lib.or_metropolis_threshold.restype = C.c_uint64
        lib.or_sweep_lattice.argtypes = [u32, P(C.c_int8), P(C.c_int8), P(C.c_int8), f64, u32, u32, u32, u32,
                                         u32, P(i32), P(i32)]
        lib.or_sweep_lattice.restype = None
        lib.or_create.argtypes = [P(Desc), P(C.c_int)]
        lib.or_create.restype = C.c_void_p
        lib.or_destroy.argtypes = [C.c_void_p]
        lib.or_destroy.restype = None
        lib.or_step.argtypes = [C.c_void_p]
        lib.or_step.restype = C.c_int
        lib.or_measure_pair.argtypes = [C.c_void_p, C.c_void_p]
        lib.or_measure_pair.restype = C.c_int
        lib.or_current_step.argtypes = [C.c_void_p]
        lib.or_current_step.restype = u32
        lib.or_current_R.argtypes = [C.c_void_p]
        lib.or_current_R.restype = u32
        lib.or_get_record.argtypes = [C.c_void_p, u32, C.c_void_p]
        lib.or_get_record.restype = None
        lib.or_get_qhist.argtypes = [C.c_void_p, u32, P(u32), P(u32), P(u32)]
        lib.or_get_qhist.restype = None
        lib.or_get_counts.argtypes = [C.c_void_p, P(u32), u32]
        lib.or_get_counts.restype = None
        lib.or_get_population.argtypes = [C.c_void_p, P(C.c_int8), P(i32), P(i32), P(u32)]
        lib.or_get_population.restype = None
        lib.or_get_couplings.argtypes = [C.c_void_p, P(C.c_int8), P(C.c_int8)]
        lib.or_get_couplings.restype = None
        lib.or_weighted_average.argtypes = [C.c_void_p, P(u32), P(u32), P(u32), u32, u32, u32, u32, C.c_void_p,
                                            P(f64), P(f64), P(f64), P(f64)]
        lib.or_weighted_average.restype = C.c_int
        lib.or_log_weight.argtypes = [C.c_void_p, u32, u32, u32, u32]
        lib.or_log_weight.restype = f64
        lib.or_bruteforce.argtypes = [u32, P(C.c_int8), P(C.c_int8), f64, P(f64), P(f64), P(f64), P(f64),
                                      P(f64), P(f64)]
        lib.or_bruteforce.restype = C.c_int
        lib.or_bruteforce_moments.argtypes = [u32, P(C.c_int8), P(C.c_int8), f64, P(f64)]
        lib.or_bruteforce_moments.restype = C.c_int
        lib.or_wang_pairing.argtypes = [u32, u32, u32, u32, P(u32), P(u32), P(u32)]
        lib.or_wang_pairing.restype = C.c_int
        lib.or_kaufman_lnZ.argtypes = [u32, f64]
        lib.or_kaufman_lnZ.restype = f64
        lib.or_dos_transfer.argtypes = [u32, P(C.c_int8), P(C.c_int8), P(C.c_uint64), P(C.c_uint64)]
        lib.or_dos_transfer.restype = C.c_int
        for name in ("or_sizeof_record", "or_sizeof_wavg", "or_sizeof_desc"):
            getattr(lib, name).argtypes = []
            getattr(lib, name).restype = u32
        assert lib.or_sizeof_record() == RECORD_DTYPE.itemsize, "record layout mismatch"
        assert lib.or_sizeof_wavg() == WAVG_DTYPE.itemsize, "wavg layout mismatch"
        assert lib.or_sizeof_desc() == C.sizeof(Desc), "desc layout mismatch"
        _lib = lib
        return lib


# --------------------------------------------------------------------------- #
def philox4x32_10(ctr, key):
    lib = load()
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    o = np.zeros(4, dtype=np.uint32)
    lib.or_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(o, C.c_uint32))
    return o


def couplings(L, model, seed, disorder_id):
    lib = load()
    Jr = np.zeros(L * L, dtype=np.int8)
    Jd = np.zeros(L * L, dtype=np.int8)
    lib.or_couplings(L, model, seed, disorder_id, _p(Jr, C.c_int8), _p(Jd, C.c_int8))
    return Jr, Jd


def energy(L, s, Jr, Jd):
    lib = load()
    s = np.ascontiguousarray(s, dtype=np.int8)
    return int(lib.or_energy(L, _p(s, C.c_int8), _p(np.ascontiguousarray(Jr, np.int8), C.c_int8),
                             _p(np.ascontiguousarray(Jd, np.int8), C.c_int8)))


def metropolis_threshold(beta, m):
    return int(load().or_metropolis_threshold(float(beta), int(m)))


def sweep_lattice(L, s, Jr, Jd, beta, theta, seed, run_id, j, step):
    """Sweep one lattice in place; returns (E, M) after the sweeps."""
    lib = load()
    s = np.ascontiguousarray(s, dtype=np.int8)
    E = np.array([energy(L, s, Jr, Jd)], dtype=np.int32)
    M = np.array([int(s.astype(np.int64).sum())], dtype=np.int32)
    Jr = np.ascontiguousarray(Jr, np.int8)
    Jd = np.ascontiguousarray(Jd, np.int8)
    lib.or_sweep_lattice(L, _p(s, C.c_int8), _p(Jr, C.c_int8), _p(Jd, C.c_int8), float(beta), theta, seed,
                         run_id, j, step, _p(E, C.c_int32), _p(M, C.c_int32))
    return s, int(E[0]), int(M[0])


def bruteforce(L, Jr, Jd, beta):
    lib = load()
    N = L * L
    out = [C.c_double() for _ in range(5)]
    pE = np.zeros(N + 1, dtype=np.float64)
    rc = lib.or_bruteforce(L, _p(np.ascontiguousarray(Jr, np.int8), C.c_int8),
                           _p(np.ascontiguousarray(Jd, np.int8), C.c_int8), float(beta),
                           *[C.byref(o) for o in out], _p(pE, C.c_double))
    if rc != 0:
        raise ValueError("bruteforce: lattice too large")
    lnZ, e, c, m, chi = (o.value for o in out)
    return dict(lnZ=lnZ, e=e, c=c, absm=m, chi=chi, pE=pE)


def wang_pairing(seed, run_id, step, fam):
    """Wang pairing of replicas with families fam (Sec. III.D): (pi* or None, swaps)."""
    lib = load()
    f = np.ascontiguousarray(fam, dtype=np.uint32)
    pi = np.zeros(max(1, len(f)), dtype=np.uint32)
    sw = C.c_uint32(0)
    ok = lib.or_wang_pairing(seed, run_id, step, len(f), _p(f, C.c_uint32), _p(pi, C.c_uint32), C.byref(sw))
    return (pi[:len(f)] if ok else None), int(sw.value)


def bruteforce_moments(L, Jr, Jd, beta):
    """Exact <e^k> and <|m|^k>, k = 1..4, by enumeration (N <= 24): two arrays of 4."""
    lib = load()
    out = np.zeros(8, dtype=np.float64)
    rc = lib.or_bruteforce_moments(L, _p(np.ascontiguousarray(Jr, np.int8), C.c_int8),
                                   _p(np.ascontiguousarray(Jd, np.int8), C.c_int8), float(beta),
                                   _p(out, C.c_double))
    if rc != 0:
        raise ValueError("bruteforce_moments: lattice too large")
    return out[:4], out[4:]


def kaufman_lnZ(L, K):
    return float(load().or_kaufman_lnZ(L, float(K)))


def dos_transfer(L, Jr, Jd):
    """Exact g over (E + 2N)/2 = 0..2N as Python ints."""
    lib = load()
    N = L * L
    lo = np.zeros(2 * N + 1, dtype=np.uint64)
    hi = np.zeros(2 * N + 1, dtype=np.uint64)
    rc = lib.or_dos_transfer(L, _p(np.ascontiguousarray(Jr, np.int8), C.c_int8),
                             _p(np.ascontiguousarray(Jd, np.int8), C.c_int8), _p(lo, C.c_uint64),
                             _p(hi, C.c_uint64))
    if rc != 0:
        raise ValueError(f"dos_transfer failed ({rc})")
    return [int(h) << 64 | int(l) for l, h in zip(lo, hi)]


class OracleRun:
    """One PA run of the oracle (steps (i)-(vi) of Sec. II.B)."""

    def __init__(self, L, model, R, R_cap, theta, betas, seed, run_id, disorder_id, resample=0, overlap=0,
                 log_g=None):
        self.lib = load()
        self.betas = np.ascontiguousarray(betas, dtype=np.float64)
        self.L, self.N = L, L * L
        self.n_beta = len(self.betas)
        self.log_g = None if log_g is None else np.ascontiguousarray(log_g, dtype=np.float64)
        d = Desc(L, model, R, R_cap, theta, self.n_beta, _p(self.betas, C.c_double), seed, run_id, disorder_id,
                 resample, overlap, _p(self.log_g, C.c_double))
        st = C.c_int(0)
        self.h = self.lib.or_create(C.byref(d), C.byref(st))
        if not self.h:
            raise ValueError(f"or_create failed (status {st.value})")

    @classmethod
    def from_desc(cls, desc):
        return cls(desc.L, desc.model, desc.R, desc.R_cap, desc.theta, desc.betas, desc.seed, desc.run_id,
                   desc.disorder_id, desc.resample, desc.overlap, getattr(desc, "log_g", None))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.or_destroy(h)
            self.h = None

    def step(self):
        return int(self.lib.or_step(self.h))

    def measure_pair(self, other):
        rc = self.lib.or_measure_pair(self.h, other.h)
        if rc:
            raise RuntimeError(f"or_measure_pair failed ({rc})")

    @property
    def cur_step(self):
        return int(self.lib.or_current_step(self.h))

    @property
    def R(self):
        return int(self.lib.or_current_R(self.h))

    def record(self, step):
        r = np.zeros(1, dtype=RECORD_DTYPE)
        self.lib.or_get_record(self.h, step, r.ctypes.data)
        return r[0]

    def records(self):
        return np.concatenate([np.atleast_1d(self.record(i)) for i in range(self.cur_step + 1)])

    def qhist(self, step):
        a = np.zeros(self.N + 1, dtype=np.uint32)
        b = np.zeros(self.N + 1, dtype=np.uint32)
        self.lib.or_get_qhist(self.h, step, _p(a, C.c_uint32), _p(b, C.c_uint32), None)
        return a, b

    def qhist_wang(self, step):
        """Histogram over d of the Wang pairs at this step (zeros if none were measured)."""
        w = np.zeros(self.N + 1, dtype=np.uint32)
        self.lib.or_get_qhist(self.h, step, None, None, _p(w, C.c_uint32))
        return w

    def counts(self, n):
        r = np.zeros(n, dtype=np.uint32)
        self.lib.or_get_counts(self.h, _p(r, C.c_uint32), n)
        return r

    def population(self):
        R = self.R
        s = np.zeros((R, self.N), dtype=np.int8)
        E = np.zeros(R, dtype=np.int32)
        M = np.zeros(R, dtype=np.int32)
        fam = np.zeros(R, dtype=np.uint32)
        self.lib.or_get_population(self.h, _p(s, C.c_int8), _p(E, C.c_int32), _p(M, C.c_int32),
                                   _p(fam, C.c_uint32))
        return s, E, M, fam

    def couplings(self):
        Jr = np.zeros(self.N, dtype=np.int8)
        Jd = np.zeros(self.N, dtype=np.int8)
        self.lib.or_get_couplings(self.h, _p(Jr, C.c_int8), _p(Jd, C.c_int8))
        return Jr, Jd

    def run_to_end(self):
        while self.cur_step + 1 < self.n_beta:
            rc = self.step()
            if rc:
                raise RuntimeError(f"or_step failed ({rc})")


def weighted_average(recs, N, kind=0, qh=None, qh_pair=None, return_weights=False, qh_wang=None):
    """recs: array [M, n_steps] of RECORD_DTYPE; qh, qh_pair, qh_wang: uint32 [M, n_steps, N+1].
    Returns (out, Pq, Pq_pair), then Pq_wang if qh_wang is given, then the weights if asked."""
    lib = load()
    recs = np.ascontiguousarray(recs, dtype=RECORD_DTYPE)
    M, n = recs.shape
    out = np.zeros(n, dtype=WAVG_DTYPE)
    Pq = np.zeros((n, N + 1)) if qh is not None else None
    Pp = np.zeros((n, N + 1)) if qh_pair is not None else None
    Pw = np.zeros((n, N + 1)) if qh_wang is not None else None
    qh = np.ascontiguousarray(qh, dtype=np.uint32) if qh is not None else None
    qh_pair = np.ascontiguousarray(qh_pair, dtype=np.uint32) if qh_pair is not None else None
    qh_wang = np.ascontiguousarray(qh_wang, dtype=np.uint32) if qh_wang is not None else None
    w = np.zeros((n, M)) if return_weights else None
    rc = lib.or_weighted_average(recs.ctypes.data, _p(qh, C.c_uint32), _p(qh_pair, C.c_uint32),
                                 _p(qh_wang, C.c_uint32), M, n, N, kind, out.ctypes.data, _p(Pq, C.c_double),
                                 _p(Pp, C.c_double), _p(Pw, C.c_double), _p(w, C.c_double))
    if rc:
        raise ValueError(f"or_weighted_average failed ({rc})")
    res = (out, Pq, Pp) + ((Pw,) if qh_wang is not None else ()) + ((w,) if return_weights else ())
    return res


def log_weights(recs, kind=0):
    """The exponents lambda[i, m] that weighted_average normalises into its weights
    (Eq. appropriateWeight for kind 0, Eq. simpleWeight for kind 1)."""
    lib = load()
    recs = np.ascontiguousarray(recs, dtype=RECORD_DTYPE)
    M, n = recs.shape
    return np.array([[lib.or_log_weight(recs.ctypes.data, n, m, i, kind) for m in range(M)] for i in range(n)])
