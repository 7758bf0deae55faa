"""CPU oracle for the multilevel local-expansion Metropolis-Hastings method
(Saunders, Grant & Mueller, arXiv 2006.16622).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, single-threaded FP64
implementation of Algorithms L.1-L.3, Algorithm 1 and the periodic extensions
of Sec. 3.4, written from the paper.  Only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline legs of ``bench.py`` may import it; the product path
(the CUDA library and its binding) never does.

Parity status per function (pins live in ``tests/test_oracle_*.py``):
  harmonics, M2L, lattice sums, Ewald, setup, propose, accept, energy: pinned
  Philox stream: pinned only by its definition (statistics + independence of
  counter words); the paper fixes no generator.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mc_oracle.c")
_HDR = os.path.join(_HERE, "mc_oracle.h")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

BC_PBC, BC_FREE = 0, 1
TINFOIL, VACUUM = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(f) > os.path.getmtime(_LIB) for f in (_SRC, _HDR))
    if stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_D = ctypes.c_double
_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_create.restype = _P
            L.orc_create.argtypes = [_I64, _P, _P, _D, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int]
            L.orc_destroy.argtypes = [_P]
            L.orc_setup.argtypes = [_P]
            L.orc_setup_fmm.argtypes = [_P]
            L.orc_fmm_local_cell.argtypes = [_P, ctypes.c_int, _P, _P]
            L.orc_local_cell_direct.argtypes = [_P, ctypes.c_int, _P, _P]
            L.orc_setup_multipole.argtypes = [_P]
            L.orc_set_lj.argtypes = [_P, _D, _D, _D]
            L.orc_get_multipole.argtypes = [_P, ctypes.c_int, _P]
            L.orc_propose.restype = _D
            L.orc_propose.argtypes = [_P, _I64, _P]
            L.orc_last_parts.argtypes = [_P, _P]
            L.orc_far_delta_factored.restype = _D
            L.orc_far_delta_factored.argtypes = [_P, _I64, _P]
            L.orc_accept.argtypes = [_P, _I64, _P, _D]
            L.orc_energy.restype = _D
            L.orc_energy.argtypes = [_P]
            L.orc_energy_fresh.restype = _D
            L.orc_energy_fresh.argtypes = [_P]
            L.orc_get_positions.argtypes = [_P, _P]
            L.orc_get_local.restype = ctypes.c_int
            L.orc_get_local.argtypes = [_P, ctypes.c_int, _P]
            L.orc_get_KH.argtypes = [_P, _P, _P]
            L.orc_ylm.argtypes = [ctypes.c_int, _D, _D, _P]
            L.orc_regular.argtypes = [ctypes.c_int, _P, _P]
            L.orc_irregular.argtypes = [ctypes.c_int, _P, _P]
            L.orc_multipole.argtypes = [ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]
            L.orc_m2l.argtypes = [ctypes.c_int, _P, _P, _P]
            L.orc_eval_local.restype = _D
            L.orc_eval_local.argtypes = [ctypes.c_int, _P, _P]
            L.orc_lattice_sums.argtypes = [ctypes.c_int, _P]
            L.orc_philox4x32_10.argtypes = [_P, _P, _P]
            L.orc_proposal.argtypes = [_I64, _D, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_uint32, _P, _P, _P]
            L.orc_run.restype = _I64
            L.orc_run.argtypes = [_P, _I64, ctypes.c_uint64, ctypes.c_uint64,
                                  ctypes.c_uint32, _D, _D, _P, _P, _P, _P]
            L.orc_run_follow.restype = _I64
            L.orc_run_follow.argtypes = [_P, _I64, ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.c_uint32, _D, _D, _P, _P, _P, _P, _P]
            L.orc_interaction_list.restype = ctypes.c_int
            L.orc_interaction_list.argtypes = [_P, ctypes.c_int, _P, _P]
            L.orc_ewald_energy.restype = _D
            L.orc_ewald_energy.argtypes = [_I64, _P, _P, _D, _D, ctypes.c_int, ctypes.c_int]
            L.orc_direct_energy.restype = _D
            L.orc_direct_energy.argtypes = [_I64, _P, _P]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def idx(n: int, m: int) -> int:
    """index of (n, m) in the full complex coefficient arrays"""
    return n * n + n + m


def ylm(p, theta, phi):
    out = np.zeros(2 * (p + 1) ** 2)
    lib().orc_ylm(p, theta, phi, _ptr(out))
    return out[0::2] + 1j * out[1::2]


def regular(p, x):
    x = _f64(x)
    out = np.zeros(2 * (p + 1) ** 2)
    lib().orc_regular(p, _ptr(x), _ptr(out))
    return out[0::2] + 1j * out[1::2]


def irregular(p, x):
    x = _f64(x)
    out = np.zeros(2 * (p + 1) ** 2)
    lib().orc_irregular(p, _ptr(x), _ptr(out))
    return out[0::2] + 1j * out[1::2]


def multipole(p, pos, q, c):
    pos, q, c = _f64(pos), _f64(q), _f64(c)
    out = np.zeros(2 * (p + 1) ** 2)
    lib().orc_multipole(p, len(q), _ptr(pos), _ptr(q), _ptr(c), _ptr(out))
    return out[0::2] + 1j * out[1::2]


def m2l(p, M, c):
    Mi = np.zeros(2 * (p + 1) ** 2)
    Mi[0::2], Mi[1::2] = M.real, M.imag
    c = _f64(c)
    out = np.zeros(2 * (p + 1) ** 2)
    lib().orc_m2l(p, _ptr(Mi), _ptr(c), _ptr(out))
    return out[0::2] + 1j * out[1::2]


def eval_local(p, Lc, x):
    Li = np.zeros(2 * (p + 1) ** 2)
    Li[0::2], Li[1::2] = Lc.real, Lc.imag
    x = _f64(x)
    return lib().orc_eval_local(p, _ptr(Li), _ptr(x))


def lattice_sums(lmax):
    out = np.zeros(2 * (lmax + 1) ** 2)
    lib().orc_lattice_sums(lmax, _ptr(out))
    return out[0::2] + 1j * out[1::2]


def philox(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def proposal(n, half_width, seed, step, chain=0):
    j = np.zeros(1, dtype=np.int64)
    d = np.zeros(3)
    u = np.zeros(1)
    lib().orc_proposal(n, half_width, seed, step, chain, _ptr(j), _ptr(d), _ptr(u))
    return int(j[0]), d, float(u[0])


def ewald_energy(pos, q, a, kappa=None, nreal=2, nrecip=12):
    pos, q = _f64(pos), _f64(q)
    if kappa is None:
        kappa = 6.0 / a
    return lib().orc_ewald_energy(len(q), _ptr(pos), _ptr(q), a, kappa, nreal, nrecip)


def direct_energy(pos, q):
    pos, q = _f64(pos), _f64(q)
    return lib().orc_direct_energy(len(q), _ptr(pos), _ptr(q))


class System:
    """One oracle system: positions (n, 3) in [0, a)^3, charges (n,)."""

    def __init__(self, pos, q, a, levels, p, bc=BC_PBC, dipole_bc=TINFOIL):
        self._pos = _f64(pos).reshape(-1, 3)
        self._q = _f64(q)
        self.n, self.a, self.L, self.p = len(self._q), float(a), int(levels), int(p)
        self.C = (self.p + 1) ** 2
        self.bc = bc
        self._h = lib().orc_create(self.n, _ptr(self._pos), _ptr(self._q), self.a,
                                   self.L, self.p, bc, dipole_bc)
        if not self._h:
            raise ValueError("orc_create rejected the arguments")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def setup(self):
        lib().orc_setup(self._h)

    def setup_fmm(self):
        lib().orc_setup_fmm(self._h)

    def set_lj(self, eps, sig, rc):
        if lib().orc_set_lj(self._h, float(eps), float(sig), float(rc)) != 0:
            raise ValueError("bad Lennard-Jones parameters (rc must not exceed the finest cell width)")

    def setup_multipole(self):
        lib().orc_setup_multipole(self._h)

    def multipole(self, level):
        nl = 1 << (level - 1)
        out = np.zeros((nl ** 3, self.C))
        if lib().orc_get_multipole(self._h, level, _ptr(out)) != 0:
            raise ValueError("bad level or no multipoles")
        return out

    def fmm_local_cell(self, level, c):
        cc = np.ascontiguousarray(np.asarray(c, dtype=np.int32))
        out = np.zeros(self.C)
        if lib().orc_fmm_local_cell(self._h, level, _ptr(cc), _ptr(out)) != 0:
            raise ValueError("bad level")
        return out

    def local_cell_direct(self, level, c):
        """Alg. L.3 expansion of one cell by its definition (no setup
        needed), real layout, paper normalisation."""
        cc = np.ascontiguousarray(np.asarray(c, dtype=np.int32))
        out = np.zeros(self.C)
        if lib().orc_local_cell_direct(self._h, level, _ptr(cc), _ptr(out)) != 0:
            raise ValueError("bad level or cell")
        return out

    def propose(self, j, rnew):
        r = _f64(rnew)
        return lib().orc_propose(self._h, int(j), _ptr(r))

    def last_parts(self):
        out = np.zeros(4)
        lib().orc_last_parts(self._h, _ptr(out))
        return out

    def far_delta_factored(self, j, rnew):
        r = _f64(rnew)
        return lib().orc_far_delta_factored(self._h, int(j), _ptr(r))

    def accept(self, j, rnew, dE):
        r = _f64(rnew)
        lib().orc_accept(self._h, int(j), _ptr(r), float(dE))

    def energy(self):
        return lib().orc_energy(self._h)

    def energy_fresh(self):
        return lib().orc_energy_fresh(self._h)

    def positions(self):
        out = np.zeros((self.n, 3))
        lib().orc_get_positions(self._h, _ptr(out))
        return out

    def local(self, level):
        nl = 1 << (level - 1)
        out = np.zeros((nl ** 3, self.C))
        if lib().orc_get_local(self._h, level, _ptr(out)) != 0:
            raise ValueError("bad level")
        return out

    def KH(self):
        K, H = np.zeros(self.C), np.zeros(self.C)
        lib().orc_get_KH(self._h, _ptr(K), _ptr(H))
        return K, H

    def interaction_list(self, level, c):
        cc = np.ascontiguousarray(np.asarray(c, dtype=np.int32))
        out = np.zeros((189, 4), dtype=np.int32)
        k = lib().orc_interaction_list(self._h, level, _ptr(cc), _ptr(out))
        return out[:k]

    def run(self, n_steps, seed, step0=0, chain=0, beta=1.0, half_width=0.5, log=True):
        n_steps = int(n_steps)
        lj = np.zeros(n_steps, dtype=np.int64) if log else None
        ld = np.zeros(n_steps) if log else None
        la = np.zeros(n_steps, dtype=np.uint8) if log else None
        nb = np.zeros(1, dtype=np.int64)
        nacc = lib().orc_run(self._h, n_steps, seed, step0, chain, beta, half_width,
                             _ptr(lj) if log else None, _ptr(ld) if log else None,
                             _ptr(la) if log else None, _ptr(nb))
        return dict(n_acc=int(nacc), n_borderline=int(nb[0]), j=lj, dE=ld, acc=la)

    def run_follow(self, follow, seed, step0=0, chain=0, beta=1.0, half_width=0.5):
        """The chain of ``run`` with step t accepted iff follow[t] (the
        decisions of another chain); ``acc`` holds this chain's own rule."""
        f = np.ascontiguousarray(np.asarray(follow, dtype=np.uint8))
        n_steps = len(f)
        lj = np.zeros(n_steps, dtype=np.int64)
        ld = np.zeros(n_steps)
        la = np.zeros(n_steps, dtype=np.uint8)
        nb = np.zeros(1, dtype=np.int64)
        nacc = lib().orc_run_follow(self._h, n_steps, seed, step0, chain, beta, half_width,
                                    _ptr(f), _ptr(lj), _ptr(ld), _ptr(la), _ptr(nb))
        return dict(n_acc=int(nacc), n_borderline=int(nb[0]), j=lj, dE=ld, acc=la)
