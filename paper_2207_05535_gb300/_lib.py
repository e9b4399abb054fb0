"""ctypes binding of libpa.so (include/pa.h): the same names, argument
marshalling only.  Every computation runs in the CUDA engine; there is no
CPU fallback: if the library is missing this module raises."""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpa.so")

PA_OK = 0
STATUS = {0: "PA_OK", 1: "PA_ERR_INVALID_ARG", 2: "PA_ERR_OOM", 3: "PA_ERR_CAPACITY", 4: "PA_ERR_EXTINCT",
          5: "PA_ERR_CUDA", 6: "PA_ERR_TIMEOUT", 7: "PA_ERR_STATE", 8: "PA_ERR_BUSY"}


class PAError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)}")


class pa_server_config(C.Structure):
    _fields_ = [("max_runs", C.c_uint32), ("reserved", C.c_uint32), ("replica_capacity", C.c_uint64),
                ("spin_words", C.c_uint64), ("record_capacity", C.c_uint64), ("qhist_words", C.c_uint64),
                ("scratch_words", C.c_uint64), ("coupling_words", C.c_uint64), ("table_doubles", C.c_uint64)]


class pa_run_desc(C.Structure):
    _fields_ = [("L", C.c_uint32), ("model", C.c_uint32), ("R", C.c_uint32), ("R_cap", C.c_uint32),
                ("theta", C.c_uint32), ("n_beta", C.c_uint32), ("beta", C.POINTER(C.c_double)),
                ("seed", C.c_uint32), ("run_id", C.c_uint32), ("disorder_id", C.c_uint32),
                ("resample", C.c_uint32), ("overlap", C.c_uint32), ("paired", C.c_int32),
                ("reserved", C.c_uint32), ("log_g", C.POINTER(C.c_double))]


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

EXPORTS = ["pa_create", "pa_create_ex", "pa_pool_sizes", "pa_server_create", "pa_admit", "pa_retire", "pa_finished", "pa_run_state",
           "pa_reset", "pa_anneal_step", "pa_sync", "pa_records", "pa_measure", "pa_population", "pa_population_slice",
           "pa_checkpoint", "pa_restore",
           "pa_weighted_average_runs", "pa_weighted_average", "pa_weighted_average_noalloc", "pa_launch_count", "pa_set_profiling",
           "pa_step_records", "pa_set_allocator", "pa_tuning_pending",
           "pa_kernel_times", "pa_transfer_bytes", "pa_calibrate_philox", "pa_sweep_shape", "pa_destroy", "pa_status_string"]
KERNEL_KINDS = ["resample", "sweep", "overlap", "measure", "init", "wavg", "small"]

# pa_alloc_fn / pa_free_fn (include/pa.h)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_int, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_int, C.c_void_p, C.c_void_p)

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libpa.so; raises if it has not been built (no fallback path)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libpa.so not found at {path}: build it with "
                               "`python -m paper_2207_05535_gb300.build` (the CUDA engine is required)")
        lib = C.CDLL(path)
        P, u32, vp = C.POINTER, C.c_uint32, C.c_void_p
        lib.pa_create.argtypes = [P(pa_run_desc), u32, vp, P(vp)]
        lib.pa_create_ex.argtypes = [P(pa_run_desc), u32, vp, u32, P(vp)]
        lib.pa_pool_sizes.argtypes = [P(pa_run_desc), u32, P(pa_server_config)]
        lib.pa_server_create.argtypes = [P(pa_server_config), vp, u32, P(vp)]
        lib.pa_admit.argtypes = [vp, P(pa_run_desc), u32, P(u32)]
        lib.pa_retire.argtypes = [vp, u32]
        lib.pa_finished.argtypes = [vp, P(u32), u32, P(u32)]
        lib.pa_run_state.argtypes = [vp, u32, P(u32), P(u32), P(u32)]
        lib.pa_reset.argtypes = [vp]
        lib.pa_anneal_step.argtypes = [vp, u32, C.c_int]
        lib.pa_sync.argtypes = [vp]
        lib.pa_records.argtypes = [vp, u32, vp, P(u32), P(u32), P(u32)]
        lib.pa_measure.argtypes = [vp, u32, u32, vp, P(u32), P(u32), P(u32)]
        lib.pa_step_records.argtypes = [vp, P(u32), u32, vp]
        lib.pa_tuning_pending.argtypes = [vp, P(u32)]
        lib.pa_set_allocator.argtypes = [ALLOC_FN, FREE_FN, vp]
        lib.pa_population.argtypes = [vp, u32, P(C.c_int8), P(C.c_int32), P(C.c_int32), P(u32), P(u32), P(u32)]
        lib.pa_population_slice.argtypes = [vp, u32, u32, u32, P(C.c_int8), P(C.c_int32), P(C.c_int32), P(u32),
                                            P(u32), P(u32)]
        lib.pa_checkpoint.argtypes = [vp, u32, vp, P(C.c_size_t)]
        lib.pa_restore.argtypes = [vp, u32, vp, C.c_size_t]
        lib.pa_weighted_average_runs.argtypes = [vp, P(u32), u32, u32, u32, vp, P(C.c_double), P(C.c_double),
                                                 P(C.c_double)]
        lib.pa_weighted_average.argtypes = [vp, P(u32), P(u32), P(u32), u32, u32, u32, u32, vp, P(C.c_double),
                                            P(C.c_double), P(C.c_double), vp]
        lib.pa_weighted_average_noalloc.argtypes = [vp, u32, u32, u32, u32, vp, vp]
        lib.pa_launch_count.argtypes = [vp]
        lib.pa_launch_count.restype = C.c_uint64
        lib.pa_sweep_shape.argtypes = [vp, u32, P(u32), P(u32), P(u32), P(u32)]
        lib.pa_set_profiling.argtypes = [vp, C.c_int]
        lib.pa_kernel_times.argtypes = [vp, P(C.c_double), P(C.c_uint64)]
        lib.pa_transfer_bytes.argtypes = [vp, P(C.c_uint64), P(C.c_uint64)]
        lib.pa_calibrate_philox.argtypes = [u32, u32, vp, P(C.c_double)]
        lib.pa_destroy.argtypes = [vp]
        lib.pa_status_string.argtypes = [C.c_int]
        lib.pa_status_string.restype = C.c_char_p
        for n in EXPORTS:
            if n not in ("pa_launch_count", "pa_status_string"):
                getattr(lib, n).restype = C.c_int
        _lib = lib
        return lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def _check(rc, what):
    if rc != PA_OK:
        raise PAError(rc, what)


def make_descs(runs):
    """RunDesc list -> ctypes array (keeps the beta arrays alive on the result)."""
    arr = (pa_run_desc * len(runs))()
    keep = []
    for k, r in enumerate(runs):
        b = np.ascontiguousarray(r.betas, dtype=np.float64)
        g = None if r.log_g is None else np.ascontiguousarray(r.log_g, dtype=np.float64)
        keep += [b, g]
        arr[k] = pa_run_desc(r.L, r.model, r.R, r.R_cap, r.theta, len(b), _p(b, C.c_double), r.seed, r.run_id,
                             r.disorder_id, r.resample, r.overlap, r.paired if r.overlap & W.Q_PAIR else -1, 0,
                             _p(g, C.c_double))
    arr._keep = keep
    return arr


# ------------------------------------------------------------ C-ABI mirrors
def pa_create(runs, stream=None):
    lib = load()
    d = make_descs(runs)
    h = C.c_void_p()
    s = C.c_void_p(stream) if stream else None
    _check(lib.pa_create(d, len(runs), s, C.byref(h)), "pa_create")
    return h


PA_CREATE_GENERIC_SWEEP = 1
PA_CREATE_NO_AUTOTUNE = 2


def pa_create_ex(runs, stream=None, flags=0):
    lib = load()
    d = make_descs(runs)
    h = C.c_void_p()
    s = C.c_void_p(stream) if stream else None
    _check(lib.pa_create_ex(d, len(runs), s, flags, C.byref(h)), "pa_create_ex")
    return h


def pa_pool_sizes(runs):
    """Pool sizes (a pa_server_config) that hold these runs at once; host only."""
    cfg = pa_server_config()
    _check(load().pa_pool_sizes(make_descs(runs), len(runs), C.byref(cfg)), "pa_pool_sizes")
    return cfg


def pa_server_create(cfg, stream=None, flags=0):
    h = C.c_void_p()
    s = C.c_void_p(stream) if stream else None
    _check(load().pa_server_create(C.byref(cfg), s, flags, C.byref(h)), "pa_server_create")
    return h


def pa_admit(h, runs):
    """Admit runs (pair indices relative to the list); returns their slots.
    Raises PAError with code PA_ERR_BUSY (8) when there is no room."""
    d = make_descs(runs)
    slots = (C.c_uint32 * len(runs))()
    _check(load().pa_admit(h, d, len(runs), slots), "pa_admit")
    return [int(x) for x in slots]


def pa_retire(h, slot):
    _check(load().pa_retire(h, slot), "pa_retire")


def pa_finished(h, cap=4096):
    buf = (C.c_uint32 * cap)()
    n = C.c_uint32()
    _check(load().pa_finished(h, buf, cap, C.byref(n)), "pa_finished")
    return [int(buf[k]) for k in range(min(n.value, cap))]


def pa_run_state(h, slot):
    a, b, c = C.c_uint32(), C.c_uint32(), C.c_uint32()
    _check(load().pa_run_state(h, slot, C.byref(a), C.byref(b), C.byref(c)), "pa_run_state")
    return int(a.value), int(b.value), int(c.value)


def pa_reset(h):
    _check(load().pa_reset(h), "pa_reset")


def pa_anneal_step(h, n_steps=1, use_graph=True):
    _check(load().pa_anneal_step(h, n_steps, int(bool(use_graph))), "pa_anneal_step")


def pa_sync(h):
    rc = load().pa_sync(h)
    _check(rc, "pa_sync")


def pa_records(h, run, n_beta, N=None, qhist=False, wang=False):
    """Records [n_beta]; with qhist also the index-shift and pair histograms
    (rec, qa, qb); with wang the Wang-pair histograms are appended."""
    lib = load()
    rec = np.zeros(n_beta, dtype=RECORD_DTYPE)
    qa = np.zeros((n_beta, N + 1), dtype=np.uint32) if qhist else None
    qb = np.zeros((n_beta, N + 1), dtype=np.uint32) if qhist else None
    qw = np.zeros((n_beta, N + 1), dtype=np.uint32) if wang else None
    _check(lib.pa_records(h, run, rec.ctypes.data, _p(qa, C.c_uint32), _p(qb, C.c_uint32), _p(qw, C.c_uint32)),
           "pa_records")
    out = (rec,) + ((qa, qb) if qhist else ()) + ((qw,) if wang else ())
    return out if len(out) > 1 else rec


def pa_measure(h, run, step):
    rec = np.zeros(1, dtype=RECORD_DTYPE)
    _check(load().pa_measure(h, run, step, rec.ctypes.data, None, None, None), "pa_measure")
    return rec[0]


def pa_population(h, run, R_cap, N):
    s = np.zeros((R_cap, N), dtype=np.int8)
    E = np.zeros(R_cap, dtype=np.int32)
    M = np.zeros(R_cap, dtype=np.int32)
    fam = np.zeros(R_cap, dtype=np.uint32)
    R = C.c_uint32()
    step = C.c_uint32()
    _check(load().pa_population(h, run, _p(s, C.c_int8), _p(E, C.c_int32), _p(M, C.c_int32), _p(fam, C.c_uint32),
                                C.byref(R), C.byref(step)), "pa_population")
    n = R.value
    return s[:n], E[:n], M[:n], fam[:n], step.value


def pa_population_slice(h, run, first, count, N, spins=True):
    """Replicas first..first+count-1 of the current population: (spins or None, E, M, fam, R_i, step)."""
    s = np.zeros((count, N), dtype=np.int8) if spins else None
    E = np.zeros(count, dtype=np.int32)
    M = np.zeros(count, dtype=np.int32)
    fam = np.zeros(count, dtype=np.uint32)
    R = C.c_uint32()
    step = C.c_uint32()
    _check(load().pa_population_slice(h, run, first, count, _p(s, C.c_int8), _p(E, C.c_int32), _p(M, C.c_int32),
                                      _p(fam, C.c_uint32), C.byref(R), C.byref(step)), "pa_population_slice")
    n = max(0, min(count, R.value - min(first, R.value)))
    return (s[:n] if spins else None), E[:n], M[:n], fam[:n], R.value, step.value


def pa_checkpoint(h, run):
    """Run `run`'s state between anneal steps, as bytes (see pa.h)."""
    n = C.c_size_t(0)
    _check(load().pa_checkpoint(h, run, None, C.byref(n)), "pa_checkpoint")
    buf = (C.c_char * n.value)()
    _check(load().pa_checkpoint(h, run, buf, C.byref(n)), "pa_checkpoint")
    return bytes(buf[:n.value])


def pa_restore(h, run, data):
    """Overwrite run `run` with a checkpoint taken by pa_checkpoint (see pa.h)."""
    buf = C.create_string_buffer(bytes(data), len(data))
    _check(load().pa_restore(h, run, buf, len(data)), "pa_restore")


def pa_calibrate_philox(wide=False, reps=5, stream=None):
    """Philox4x32-10 calls per second on the current device (see pa.h)."""
    v = C.c_double(0.0)
    _check(load().pa_calibrate_philox(int(bool(wide)), reps, C.c_void_p(stream) if stream else None, C.byref(v)),
           "pa_calibrate_philox")
    return v.value


def pa_weighted_average_runs(h, run_idx, M, n_steps, N, kind=0, q=False, wang=False):
    """out [G][n_steps]; with q also (Pq, Pq_pair); with wang Pq_wang is appended."""
    idx = np.ascontiguousarray(run_idx, dtype=np.uint32).reshape(-1)
    G = len(idx) // M
    out = np.zeros((G, n_steps), dtype=WAVG_DTYPE)
    Pq = np.zeros((G, n_steps, N + 1)) if q else None
    Pp = np.zeros((G, n_steps, N + 1)) if q else None
    Pw = np.zeros((G, n_steps, N + 1)) if wang else None
    _check(load().pa_weighted_average_runs(h, _p(idx, C.c_uint32), G, M, kind, out.ctypes.data,
                                           _p(Pq, C.c_double), _p(Pp, C.c_double), _p(Pw, C.c_double)),
           "pa_weighted_average_runs")
    res = (out,) + ((Pq, Pp) if q else ()) + ((Pw,) if wang else ())
    return res if len(res) > 1 else out


def pa_weighted_average(recs, N, kind=0, qh=None, qh_pair=None, stream=None, qh_wang=None):
    """(out, Pq, Pq_pair), with Pq_wang appended when qh_wang is given."""
    recs = np.ascontiguousarray(recs, dtype=RECORD_DTYPE)
    M, n = recs.shape
    out = np.zeros(n, dtype=WAVG_DTYPE)
    qh = np.ascontiguousarray(qh, dtype=np.uint32) if qh is not None else None
    qh_pair = np.ascontiguousarray(qh_pair, dtype=np.uint32) if qh_pair is not None else None
    qh_wang = np.ascontiguousarray(qh_wang, dtype=np.uint32) if qh_wang is not None else None
    Pq = np.zeros((n, N + 1)) if qh is not None else None
    Pp = np.zeros((n, N + 1)) if qh_pair is not None else None
    Pw = np.zeros((n, N + 1)) if qh_wang is not None else None
    s = C.c_void_p(stream) if stream else None
    _check(load().pa_weighted_average(recs.ctypes.data, _p(qh, C.c_uint32), _p(qh_pair, C.c_uint32),
                                      _p(qh_wang, C.c_uint32), M, n, N, kind, out.ctypes.data, _p(Pq, C.c_double),
                                      _p(Pp, C.c_double), _p(Pw, C.c_double), s),
           "pa_weighted_average")
    return (out, Pq, Pp) + ((Pw,) if qh_wang is not None else ())


def pa_step_records(h, runs, out=None):
    """Records of runs[k] at the temperature each has reached (RECORD_DTYPE[n]);
    `out`: optional preallocated host array (for example in pinned memory)."""
    runs = np.ascontiguousarray(runs, dtype=np.uint32)
    if out is None:
        out = np.zeros(len(runs), dtype=RECORD_DTYPE)
    _check(load().pa_step_records(h, _p(runs, C.c_uint32), len(runs), out.ctypes.data), "pa_step_records")
    return out


_allocator_keep = []  # every installed pair: engines created with it call it until destroyed


def pa_set_allocator(alloc=None, free=None, ctx=None):
    """Install device allocator callbacks (Python callables with the pa_alloc_fn /
    pa_free_fn signatures) for engines created afterwards; no arguments restores
    cudaMalloc.  The callbacks are kept alive here while installed."""
    if alloc is None:
        _check(load().pa_set_allocator(ALLOC_FN(), FREE_FN(), None), "pa_set_allocator")
        return
    a, f = ALLOC_FN(alloc), FREE_FN(free)
    _check(load().pa_set_allocator(a, f, ctx), "pa_set_allocator")
    _allocator_keep.append((a, f))


def pa_tuning_pending(h):
    n = C.c_uint32()
    _check(load().pa_tuning_pending(h, C.byref(n)), "pa_tuning_pending")
    return int(n.value)


def pa_launch_count(h):
    return int(load().pa_launch_count(h))


def pa_sweep_shapes(h):
    """[(L, words_per_thread, block, tuned)] for every lattice-size group."""
    out, g = [], 0
    lib = load()
    while True:
        v = [C.c_uint32() for _ in range(4)]
        if lib.pa_sweep_shape(h, g, *[C.byref(x) for x in v]) != PA_OK:
            return out
        out.append(tuple(int(x.value) for x in v))
        g += 1


def pa_set_profiling(h, on=True):
    _check(load().pa_set_profiling(h, int(bool(on))), "pa_set_profiling")


def pa_kernel_times(h):
    ms = np.zeros(len(KERNEL_KINDS))
    n = np.zeros(len(KERNEL_KINDS), dtype=np.uint64)
    _check(load().pa_kernel_times(h, _p(ms, C.c_double), _p(n, C.c_uint64)), "pa_kernel_times")
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_KINDS)}


def pa_transfer_bytes(h):
    a, b = C.c_uint64(), C.c_uint64()
    _check(load().pa_transfer_bytes(h, C.byref(a), C.byref(b)), "pa_transfer_bytes")
    return int(a.value), int(b.value)


def pa_destroy(h):
    if h:
        _check(load().pa_destroy(h), "pa_destroy")


def pa_status_string(code):
    return load().pa_status_string(code).decode()


class Engine:
    """Owner of one pa_engine handle (context manager)."""

    def __init__(self, runs, stream=None, flags=0):
        self.runs = list(runs)
        self.h = pa_create_ex(self.runs, stream, flags) if flags else pa_create(self.runs, stream)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def close(self):
        if getattr(self, "h", None):
            pa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        pa_reset(self.h)

    def step(self, n=1, use_graph=True):
        pa_anneal_step(self.h, n, use_graph)

    def run_to_end(self, use_graph=True):
        n = max(r.n_beta for r in self.runs) - 1
        if n > 0:
            pa_anneal_step(self.h, n, use_graph)
        pa_sync(self.h)

    def sync(self):
        pa_sync(self.h)

    def step_records(self, runs, out=None):
        return pa_step_records(self.h, runs, out)

    def records(self, run, qhist=False, wang=False):
        r = self.runs[run]
        return pa_records(self.h, run, r.n_beta, r.N, qhist, wang)

    def checkpoint(self, run):
        return pa_checkpoint(self.h, run)

    def restore(self, run, data):
        pa_restore(self.h, run, data)

    def population(self, run):
        r = self.runs[run]
        return pa_population(self.h, run, r.R_cap, r.N)

    def weighted_average(self, run_idx, M, kind=0, q=False, wang=False):
        r = self.runs[int(np.asarray(run_idx).reshape(-1)[0])]
        return pa_weighted_average_runs(self.h, run_idx, M, r.n_beta, r.N, kind, q, wang)

    @property
    def launches(self):
        return pa_launch_count(self.h)
