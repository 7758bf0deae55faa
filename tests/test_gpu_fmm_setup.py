"""Parity of the fast (FMM-variant) setup with the oracle's FMM-variant setup.

The fast setup (Sec. 3.2, last paragraph) forms every cell's multipole
(Eq. 4) and translates it into the local expansion of each cell of whose
interaction list it is part.  Small systems: every level's expansions within
1e-12 of the oracle's FMM pass, K within 1e-12, energy within 1e-10, and a
replayed chain started from the fast setup has the oracle's decisions.  At
the N=1e5 benchmark size: sampled cells of every level against the oracle's
single-cell evaluation (source multipoles taken from the charges), and the
gap to the exact setup (Alg. L.3) at truncation level.
"""
import numpy as np
import pytest

import oracle as O
from paper_2006_16622_gb300 import mcfmm
from paper_2006_16622_gb300.workloads import LARGE, uniform_system

pytestmark = pytest.mark.gpu

ARR_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    mcfmm.load()


# (n, a, L, p, bc): L=2 has a single level whose 189 offsets all wrap onto
# 8 cells; p = 3, 8, 12, 15 take each output-slot count of the kernel
CASES = [(64, 4.0, 2, 6, mcfmm.BC_PBC), (200, 6.0, 3, 3, mcfmm.BC_PBC),
         (300, 8.0, 3, 8, mcfmm.BC_PBC), (600, 9.0, 4, 10, mcfmm.BC_PBC),
         (1000, 10.0, 3, 12, mcfmm.BC_PBC), (500, 8.0, 3, 15, mcfmm.BC_PBC),
         (400, 8.0, 4, 8, mcfmm.BC_FREE)]


@pytest.mark.parametrize("n,a,L,p,bc", CASES)
def test_fast_setup_matches_oracle(n, a, L, p, bc):
    pos, q = uniform_system(n, a, seed=n + p)
    g = mcfmm.Context(pos, q, a, L, p, bc=bc)
    g.setup(mcfmm.SETUP_FMM)
    o = O.System(pos, q, a, L, p, bc=bc)
    o.setup_fmm()
    for lev in range(2, L + 1):
        A, B = g.local(lev), o.local(lev)
        scale = np.max(np.abs(B))
        if scale == 0.0:  # free space: no interaction list on level 2
            assert np.max(np.abs(A)) == 0.0
            continue
        assert np.max(np.abs(A - B)) <= ARR_TOL * scale, lev
    if bc == mcfmm.BC_PBC:
        Kg, _ = g.far()
        Ko, _ = o.KH()
        assert np.max(np.abs(Kg - Ko)) <= ARR_TOL * np.max(np.abs(Ko))
    assert abs(g.energy() - o.energy()) <= 1e-10 * max(1.0, abs(o.energy()))
    g.close()


def test_fast_setup_with_empty_cells_and_repeated_calls():
    # charges crowded into one corner leave most cells empty; a second call
    # reuses the multipole tables and must give the same arrays
    rng = np.random.default_rng(5)
    a, L, p = 8.0, 4, 8
    pos = rng.uniform(0.0, 2.5, size=(150, 3))
    q = np.where(np.arange(150) % 2 == 0, 1.0, -1.0)
    g = mcfmm.Context(pos, q, a, L, p)
    g.setup(mcfmm.SETUP_FMM)
    first = [g.local(lev).copy() for lev in range(2, L + 1)]
    g.setup(mcfmm.SETUP_FMM)
    for lev in range(2, L + 1):
        assert np.array_equal(g.local(lev), first[lev - 2])
    o = O.System(pos, q, a, L, p)
    o.setup_fmm()
    for lev in range(2, L + 1):
        B = o.local(lev)
        assert np.max(np.abs(first[lev - 2] - B)) <= ARR_TOL * np.max(np.abs(B)), lev
    g.close()


def test_chain_after_fast_setup_replays_oracle():
    n, a, L, p = 800, 9.0, 3, 10
    pos, q = uniform_system(n, a, seed=77)
    g = mcfmm.Context(pos, q, a, L, p)
    g.setup(mcfmm.SETUP_FMM)
    o = O.System(pos, q, a, L, p)
    o.setup_fmm()
    rg = g.run(400, seed=3, beta=1.0, half_width=0.5, log=True)
    ro = o.run(400, seed=3, step0=0, beta=1.0, half_width=0.5)
    assert ro["n_borderline"] == 0 and rg["borderline"] == 0
    assert np.array_equal(rg["j"], ro["j"])
    err = np.abs(rg["dE"] - ro["dE"]) / np.maximum(1.0, np.abs(ro["dE"]))
    assert np.max(err) <= 1e-10, np.max(err)
    assert np.array_equal(rg["acc"], ro["acc"])
    assert np.array_equal(g.positions(), o.positions())
    g.close()


def test_fast_setup_full_size_sampled_cells_and_truncation_gap():
    W = LARGE
    pos, q = W.system()
    g = mcfmm.Context(pos, q, W.a, W.levels, W.p)
    g.setup(mcfmm.SETUP_FMM)
    fast = {lev: g.local(lev).copy() for lev in range(2, W.levels + 1)}
    e_fast = g.energy()
    o = O.System(pos, q, W.a, W.levels, W.p)
    rng = np.random.default_rng(11)
    for lev in range(2, W.levels + 1):
        nl = 1 << (lev - 1)
        scale = np.max(np.abs(fast[lev]))
        for _ in range(1 if lev == 2 else 2):
            c = rng.integers(0, nl, size=3)
            ref = o.fmm_local_cell(lev, c)
            got = fast[lev][(c[0] * nl + c[1]) * nl + c[2]]
            assert np.max(np.abs(got - ref)) <= ARR_TOL * scale, (lev, c)
    # the exact setup differs from the fast one by the multipole truncation
    g.setup(mcfmm.SETUP_P2L)
    for lev in range(2, W.levels + 1):
        A = g.local(lev)
        assert np.max(np.abs(A - fast[lev])) <= 1e-6 * np.max(np.abs(A)), lev
    assert abs(g.energy() - e_fast) <= 1e-5 * abs(g.energy())
    g.close()
