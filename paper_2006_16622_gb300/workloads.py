"""Seeded synthetic inputs for the multilevel Monte Carlo electrostatics path.

This module only draws inputs (positions, charges, system sizes); it holds
none of the method's arithmetic, so both the CUDA path and the CPU oracle may
be fed from it.  Recipes (all systems neutral, +/-1 charges, periodic cube):

* ``uniform_system``: N/2 charges +1 and N/2 charges -1, signs assigned by a
  random permutation, positions uniform in [0, a)^3 with a = (N / rho)^(1/3).
* ``rocksalt``: the NaCl arrangement of m^3 ions at spacing d, offset by d/2
  so that no ion lies on a cell face.
* ``batched_systems``: chain sizes N_i = round(exp(U(ln N_lo, ln N_hi))) made
  even, a_i = (N_i / rho)^(1/3), levels 1 + round(log8(N_i / 20)), >= 3.

The named workloads mirror the paper's timing setting (uniform random charges
in a periodic cube, Sec. 5.2) at the sizes the benchmarks use.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    # a "setup" stream distinct from the Monte Carlo proposal stream
    return np.random.Generator(np.random.Philox(key=[0x5E7C0DE, seed]))


def uniform_system(n: int, a: float, seed: int = 0):
    """Neutral +/-1 system, uniform positions in [0, a)^3 (float64)."""
    if n % 2:
        raise ValueError("n must be even for a neutral +/-1 system")
    g = _rng(seed)
    q = np.concatenate([np.ones(n // 2), -np.ones(n // 2)])
    q = q[g.permutation(n)]
    pos = g.uniform(0.0, a, size=(n, 3))
    pos = np.minimum(pos, np.nextafter(a, 0.0))
    return np.ascontiguousarray(pos), np.ascontiguousarray(q)


def rocksalt(m: int, d: float = 1.0):
    g = np.arange(m)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1).astype(np.float64) * d + 0.5 * d
    q = np.where((X + Y + Z).ravel() % 2 == 0, 1.0, -1.0)
    return np.ascontiguousarray(pos), np.ascontiguousarray(q), m * d


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    a: float
    levels: int
    p: int
    moves: int
    half_width: float
    beta: float = 1.0
    seed: int = 0

    def system(self):
        return uniform_system(self.n, self.a, self.seed)


# N = 1000 charges in a cube of side 10, 3 levels, p = 8, h = 0.5
SMALL = Workload("uniform N=1000 a=10 L=3 p=8 h=0.5", 1000, 10.0, 3, 8, 10_000, 0.5)
# N = 1e5 at density 0.1 (a = 100), 5 levels (~24 charges per finest cell), p = 12, h = 0.3
LARGE = Workload("uniform N=100000 rho=0.1 a=100 L=5 p=12 h=0.3", 100_000, 100.0, 5, 12,
                 1_000_000, 0.3)
# N = 1e6 at density 0.1, 6 levels, p = 12
HUGE = Workload("uniform N=1000000 rho=0.1 a=215.44 L=6 p=12 h=0.3", 1_000_000,
                (1_000_000 / 0.1) ** (1.0 / 3.0), 6, 12, 1_000_000, 0.3)


def batched_systems(n_chains: int = 64, n_lo: int = 1000, n_hi: int = 50000, rho: float = 0.1,
                    per_cell: float = 20.0, seed: int = 0):
    """Sizes, box sides and level counts of independent chains of uneven N."""
    g = _rng(10_000 + seed)
    out = []
    for i in range(n_chains):
        n = int(round(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        n += n % 2
        a = (n / rho) ** (1.0 / 3.0)
        levels = max(3, 1 + int(round(math.log(n / per_cell, 8))))
        out.append((n, a, levels, i))
    return out


def size_sweep(sizes=(1_000, 10_000, 100_000, 1_000_000), rho: float = 0.1,
               per_cell: float = 20.0, p: int = 12, half_width: float = 0.3):
    """Workloads of the per-operation timing against N at fixed density and
    about `per_cell` charges per finest cell (levels = 1 + round(log8(N /
    per_cell)), at least 3)."""
    out = []
    for n in sizes:
        a = (n / rho) ** (1.0 / 3.0)
        levels = max(3, 1 + int(round(np.log(n / per_cell) / np.log(8.0))))
        out.append(Workload(f"uniform N={n} rho={rho} a={a:.2f} L={levels} p={p} h={half_width}",
                            n, a, levels, p, 0, half_width))
    return out


# The acceptance-probability study (Sec. 5.1): a simple cubic NaCl crystal
# (lattice constant 3.3 Angstrom, charges +-1 e) with every ion shifted by a
# uniform random vector of at most 1 % of the lattice constant per axis, at
# T = 273 K; energies in e^2/Angstrom, so beta = (e^2 / (4 pi eps0 A)) / kT.
NACL_SPACING = 3.3
NACL_BETA = 14.399645 / (8.617333262e-5 * 273.0)


def perturbed_nacl(m: int, seed: int, spacing: float = NACL_SPACING):
    """m^3 ions of rock salt, each shifted by U(-0.01, 0.01) x spacing per axis."""
    pos, q, a = rocksalt(m, spacing)
    g = _rng(seed)
    pos = (pos + g.uniform(-0.01 * spacing, 0.01 * spacing, pos.shape)) % a
    pos = np.minimum(pos, np.nextafter(a, 0.0))
    return np.ascontiguousarray(pos), q, a


def study_moves(n: int, a: float, pos, count: int, seed: int, half_width: float = 0.25):
    """Seeded proposals (j, r') for the acceptance study: j uniform, r' = r +
    U(-h, h)^3 wrapped into the box (h = 0.25 Angstrom)."""
    g = _rng(seed + 7919)
    js = g.integers(0, n, size=count)
    rn = (pos[js] + g.uniform(-half_width, half_width, (count, 3))) % a
    rn = np.minimum(rn, np.nextafter(a, 0.0))
    return js, rn


# Full Monte Carlo NaCl runs (Sec. 5.3): the paper adds a repulsive
# Lennard-Jones term with a 12 Angstrom cutoff and gives no parameters;
# reading: epsilon = 0.1 eV (in e^2/Angstrom) and sigma with the well
# minimum at the lattice spacing.  Largest crystal: 46^3 ions in a 153.2
# Angstrom box, 12 expansion terms (p = 11), moves of +-0.25 Angstrom.
NACL_LJ_EPS = 0.1 / 14.399645
NACL_LJ_SIGMA = NACL_SPACING / 2.0 ** (1.0 / 6.0)
NACL_LJ_CUTOFF = 12.0
NACL_FULL_MC = dict(m=46, box=153.2, levels=4, p=11, half_width=0.25)


def nacl_full_mc_system(m: int = 46, box: float = 153.2, seed: int = 0):
    """m^3 rock salt in a cube of side `box` (spacing box/m), perturbed by
    1 % of the spacing (the starting state of the paper's full MC runs)."""
    return perturbed_nacl(m, seed=seed, spacing=box / m)
