"""Thin ctypes binding of ``libmcfmm.so`` (the C ABI of ``include/mcfmm.h``).

Argument marshalling only: every step of the Monte Carlo path runs in the
library's CUDA kernels.  Loading fails loudly when the library is missing;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmcfmm.so")

MC_OK = 0
BC_PBC, BC_FREE = 0, 1
TINFOIL, VACUUM = 0, 1
FP64, FP32_EVAL = 0, 1
SCHEDULE_PHASED, SCHEDULE_PIPELINED, SCHEDULE_PLAIN, SCHEDULE_ASYNC = 0, 1, 2, 3
SETUP_P2L, SETUP_FMM, SETUP_MULTIPOLE = 0, 1, 2
PROF_COUNTERS = 56

EXPORTED = ["mc_init", "mc_setup", "mc_propose", "mc_accept", "mc_run", "mc_energy",
            "mc_energy_fresh", "mc_get_positions", "mc_get_local", "mc_get_far",
            "mc_lattice_sums", "mc_status", "mc_set_wait_limit", "mc_profile", "mc_profile_read",
            "mc_destroy", "mc_strerror", "mc_p2l_level_noalloc", "mc_batch_create",
            "mc_batch_tune", "mc_batch_run", "mc_batch_info", "mc_batch_destroy",
            "mc_set_schedule", "mc_set_ctas", "mc_batch_set_schedule", "mc_inject_wait_fault",
            "mc_get_multipole", "mc_set_lj", "mc_step_counter", "mc_probe_fma_rate",
            "mc_set_near_parts"]


class McStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("accepted", ctypes.c_int64),
                ("borderline", ctypes.c_int64), ("resetups", ctypes.c_int64),
                ("energy", ctypes.c_double), ("max_drift", ctypes.c_double),
                ("sum_drift", ctypes.c_double), ("sum_abs_drift", ctypes.c_double)]


class McError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {_lib_strerror(code)} ({code})")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libmcfmm.so not built at {path}; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    P, I, D, I64, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64
    L.mc_init.argtypes = [ctypes.POINTER(P), I64, P, P, D, I, I, I, I, I, P]
    L.mc_setup.argtypes = [P, I]
    L.mc_propose.argtypes = [P, I64, P, P]
    L.mc_accept.argtypes = [P, I64, P, P]
    L.mc_run.argtypes = [P, I64, U64, D, D, I64, P, P, P, P]
    L.mc_energy.argtypes = [P, P]
    L.mc_step_counter.argtypes = [P, P]
    L.mc_probe_fma_rate.argtypes = [I, D, P]
    L.mc_energy_fresh.argtypes = [P, P]
    L.mc_get_positions.argtypes = [P, P]
    L.mc_get_local.argtypes = [P, I, P]
    L.mc_get_multipole.argtypes = [P, I, P]
    L.mc_set_lj.argtypes = [P, D, D, D]
    L.mc_set_near_parts.argtypes = [P, I, P]
    L.mc_get_far.argtypes = [P, P, P]
    L.mc_lattice_sums.argtypes = [I, P]
    L.mc_status.argtypes = [P]
    L.mc_set_wait_limit.argtypes = [P, I64]
    L.mc_inject_wait_fault.argtypes = [P, ctypes.c_int]
    L.mc_profile.argtypes = [P, I]
    L.mc_profile_read.argtypes = [P, P]
    L.mc_p2l_level_noalloc.argtypes = [P, P, I64, D, I, I, I, I, P, P]
    L.mc_destroy.argtypes = [P]
    L.mc_destroy.restype = None
    L.mc_batch_create.argtypes = [ctypes.POINTER(P), I, P]
    L.mc_batch_tune.argtypes = [P, I64, D, D]
    L.mc_batch_run.argtypes = [P, I64, P, D, D, P, P, P, P]
    L.mc_batch_info.argtypes = [P, P, P]
    L.mc_set_schedule.argtypes = [P, I]
    L.mc_set_ctas.argtypes = [P, I]
    L.mc_batch_set_schedule.argtypes = [P, I]
    L.mc_batch_destroy.argtypes = [P]
    L.mc_batch_destroy.restype = None
    L.mc_strerror.argtypes = [I]
    L.mc_strerror.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("mc_destroy", "mc_strerror", "mc_batch_destroy"):
            getattr(L, name).restype = I
    _lib = L
    return L


def _lib_strerror(code):
    try:
        return load().mc_strerror(int(code)).decode()
    except OSError:
        return "library not loaded"


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _check(code, what):
    if code != MC_OK:
        raise McError(code, what)


def p2l_level_noalloc(d_part, d_cell_start, n, box, levels, level, p, bc, d_out, stream=None):
    """Allocation-free level expansions from caller-owned device buffers
    (raw device addresses as ints); see mc_p2l_level_noalloc in mcfmm.h."""
    return load().mc_p2l_level_noalloc(ctypes.c_void_p(d_part), ctypes.c_void_p(d_cell_start),
                                       int(n), float(box), int(levels), int(level), int(p),
                                       int(bc), ctypes.c_void_p(d_out),
                                       ctypes.c_void_p(stream) if stream else None)


def probe_fma_rate(fp64: bool, target_seconds: float = 0.2) -> float:
    """Measured FMA-pipe peak of the current device in flop/s (FP64 or FP32)."""
    out = np.zeros(1)
    _check(load().mc_probe_fma_rate(1 if fp64 else 0, float(target_seconds), _ptr(out)),
           "mc_probe_fma_rate")
    return float(out[0])


def lattice_sums(lmax: int):
    out = np.zeros(2 * (lmax + 1) ** 2)
    _check(load().mc_lattice_sums(lmax, _ptr(out)), "mc_lattice_sums")
    return out[0::2] + 1j * out[1::2]


class Context:
    """One system on the GPU (the library owns all its device memory)."""

    def __init__(self, pos, q, box, levels, p, bc=BC_PBC, dipole_bc=TINFOIL,
                 precision=FP64, stream=None):
        L = load()
        pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
        q = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
        self.n, self.box, self.levels, self.p = len(q), float(box), int(levels), int(p)
        self.C = (self.p + 1) ** 2
        h = ctypes.c_void_p()
        _check(L.mc_init(ctypes.byref(h), self.n, _ptr(pos), _ptr(q), self.box, self.levels,
                         self.p, bc, dipole_bc, precision,
                         ctypes.c_void_p(stream) if stream else None), "mc_init")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().mc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def setup(self, mode=SETUP_P2L):
        _check(load().mc_setup(self._h, mode), "mc_setup")

    def propose(self, j, r_new):
        r = np.ascontiguousarray(np.asarray(r_new, dtype=np.float64))
        out = np.zeros(1)
        _check(load().mc_propose(self._h, int(j), _ptr(r), _ptr(out)), "mc_propose")
        return float(out[0])

    def accept(self, j, r_new, dE=None):
        r = np.ascontiguousarray(np.asarray(r_new, dtype=np.float64))
        d = np.array([dE], dtype=np.float64) if dE is not None else None
        _check(load().mc_accept(self._h, int(j), _ptr(r), _ptr(d)), "mc_accept")

    def run(self, n_steps, seed, beta=1.0, half_width=0.5, resetup_every=0, log=False,
            stats=True):
        n_steps = int(n_steps)
        st = McStats()
        lj = np.zeros(n_steps, dtype=np.int64) if log else None
        ld = np.zeros(n_steps) if log else None
        la = np.zeros(n_steps, dtype=np.uint8) if log else None
        _check(load().mc_run(self._h, n_steps, int(seed), float(beta), float(half_width),
                             int(resetup_every), ctypes.byref(st) if stats else None,
                             _ptr(lj), _ptr(ld), _ptr(la)), "mc_run")
        res = {k: getattr(st, k) for k, _ in McStats._fields_} if stats else {}
        if log:
            res.update(j=lj, dE=ld, acc=la)
        return res

    def energy(self):
        out = np.zeros(1)
        _check(load().mc_energy(self._h, _ptr(out)), "mc_energy")
        return float(out[0])

    def step_counter(self):
        out = np.zeros(1, dtype=np.int64)
        _check(load().mc_step_counter(self._h, _ptr(out)), "mc_step_counter")
        return int(out[0])

    def energy_fresh(self):
        out = np.zeros(1)
        _check(load().mc_energy_fresh(self._h, _ptr(out)), "mc_energy_fresh")
        return float(out[0])

    def positions(self):
        out = np.zeros((self.n, 3))
        _check(load().mc_get_positions(self._h, _ptr(out)), "mc_get_positions")
        return out

    def local(self, level):
        nl = 1 << (level - 1)
        out = np.zeros((nl ** 3, self.C))
        _check(load().mc_get_local(self._h, int(level), _ptr(out)), "mc_get_local")
        return out

    def set_lj(self, eps, sigma, cutoff):
        _check(load().mc_set_lj(self._h, float(eps), float(sigma), float(cutoff)), "mc_set_lj")

    def set_near_parts(self, parts=0):
        """Near-field (Alg. 1) items per cell and side; 0 = automatic.
        Returns the split in force."""
        out = np.zeros(1, dtype=np.int32)
        _check(load().mc_set_near_parts(self._h, int(parts), _ptr(out)), "mc_set_near_parts")
        return int(out[0])

    def multipole(self, level):
        nl = 1 << (level - 1)
        out = np.zeros((nl ** 3, self.C))
        _check(load().mc_get_multipole(self._h, int(level), _ptr(out)), "mc_get_multipole")
        return out

    def far(self):
        K, H = np.zeros(self.C), np.zeros(self.C)
        _check(load().mc_get_far(self._h, _ptr(K), _ptr(H)), "mc_get_far")
        return K, H

    def status(self):
        return load().mc_status(self._h)

    def profile(self, on=True):
        _check(load().mc_profile(self._h, 1 if on else 0), "mc_profile")

    def profile_read(self):
        out = np.zeros(PROF_COUNTERS, dtype=np.uint64)
        _check(load().mc_profile_read(self._h, _ptr(out)), "mc_profile_read")
        return out

    def set_schedule(self, schedule):
        _check(load().mc_set_schedule(self._h, int(schedule)), "mc_set_schedule")

    def set_ctas(self, n_cta):
        _check(load().mc_set_ctas(self._h, int(n_cta)), "mc_set_ctas")

    def set_wait_limit(self, ns):
        _check(load().mc_set_wait_limit(self._h, int(ns)), "mc_set_wait_limit")

    def inject_wait_fault(self, missing_arrivals):
        _check(load().mc_inject_wait_fault(self._h, int(missing_arrivals)),
               "mc_inject_wait_fault")


class Batch:
    """Many independent chains in one persistent launch (the contexts keep
    their systems; close the batch before the contexts)."""

    def __init__(self, contexts):
        L = load()
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c._h.value for c in self.contexts])
        h = ctypes.c_void_p()
        _check(L.mc_batch_create(ctypes.byref(h), len(self.contexts),
                                 ctypes.cast(arr, ctypes.c_void_p)), "mc_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().mc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tune(self, trial_steps=500, beta=1.0, half_width=0.3):
        _check(load().mc_batch_tune(self._h, int(trial_steps), float(beta), float(half_width)),
               "mc_batch_tune")

    def set_schedule(self, schedule):
        _check(load().mc_batch_set_schedule(self._h, int(schedule)), "mc_batch_set_schedule")

    def info(self):
        ctas = np.zeros(len(self.contexts), dtype=np.int32)
        nf = np.zeros(1, dtype=np.int32)
        _check(load().mc_batch_info(self._h, _ptr(ctas), _ptr(nf)), "mc_batch_info")
        return ctas, int(nf[0])

    def run(self, n_steps, seeds, beta=1.0, half_width=0.3, stats=True, log=False):
        n = len(self.contexts)
        seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
        st = (McStats * n)() if stats else None
        lj = np.zeros((n, n_steps), dtype=np.int64) if log else None
        ld = np.zeros((n, n_steps)) if log else None
        la = np.zeros((n, n_steps), dtype=np.uint8) if log else None
        _check(load().mc_batch_run(self._h, int(n_steps), _ptr(seeds), float(beta),
                                   float(half_width), ctypes.cast(st, ctypes.c_void_p) if stats
                                   else None, _ptr(lj), _ptr(ld), _ptr(la)), "mc_batch_run")
        out = {}
        if stats:
            out["stats"] = [{k: getattr(st[i], k) for k, _ in McStats._fields_} for i in range(n)]
        if log:
            out.update(j=lj, dE=ld, acc=la)
        return out
