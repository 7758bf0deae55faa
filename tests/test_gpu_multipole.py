"""Parity of the multipole method (Alg. M.1-M.3) on the GPU with the oracle.

Setup (Alg. M.3): every level's multipoles within 1e-12 of the largest of
their level, K within 1e-12, energy within 1e-10.  Chains (Alg. M.1 with
Alg. 1 and the periodic terms, Alg. M.2 on accept): every dE within
1e-10 max(1, |dE|) and every decision identical.  Properties: multipoles
after a chain equal a fresh Alg. M.3 on the final positions; the FP32-eval
form stays within the FP32 tolerance of the FP64 form.
"""
import numpy as np
import pytest

import oracle as O
from paper_2006_16622_gb300 import mcfmm
from paper_2006_16622_gb300.workloads import uniform_system

pytestmark = pytest.mark.gpu

ARR_TOL = 1e-12
DE_TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    mcfmm.load()


def _pair(n, a, L, p, seed, bc=mcfmm.BC_PBC, precision=mcfmm.FP64):
    pos, q = uniform_system(n, a, seed=seed)
    g = mcfmm.Context(pos, q, a, L, p, bc=bc, precision=precision)
    g.setup(mcfmm.SETUP_MULTIPOLE)
    o = O.System(pos, q, a, L, p, bc=bc)
    o.setup_multipole()
    return g, o, pos, q


@pytest.mark.parametrize("n,a,L,p,bc", [(64, 4.0, 2, 6, mcfmm.BC_PBC), (300, 8.0, 3, 8, mcfmm.BC_PBC),
                                        (600, 9.0, 4, 10, mcfmm.BC_PBC),
                                        (1000, 10.0, 3, 12, mcfmm.BC_PBC),
                                        (500, 8.0, 3, 15, mcfmm.BC_PBC),
                                        (400, 8.0, 4, 8, mcfmm.BC_FREE)])
def test_multipole_setup_matches_oracle(n, a, L, p, bc):
    g, o, _, _ = _pair(n, a, L, p, seed=n + 3, bc=bc)
    lmin = 2 if bc == mcfmm.BC_PBC else 3
    for lev in range(lmin, L + 1):
        A, B = g.multipole(lev), o.multipole(lev)
        assert np.max(np.abs(A - B)) <= ARR_TOL * np.max(np.abs(B)), lev
    if bc == mcfmm.BC_PBC:
        Kg, _ = g.far()
        Ko, _ = o.KH()
        assert np.max(np.abs(Kg - Ko)) <= ARR_TOL * np.max(np.abs(Ko))
    assert abs(g.energy() - o.energy()) <= DE_TOL * max(1.0, abs(o.energy()))
    with pytest.raises(mcfmm.McError):
        g.local(L)  # the multipole method keeps no local expansions
    g.close()


@pytest.mark.parametrize("n,a,L,p,bc,h", [(1000, 10.0, 3, 8, mcfmm.BC_PBC, 0.5),
                                          (16, 3.0, 2, 3, mcfmm.BC_PBC, 0.9),
                                          (900, 9.0, 4, 7, mcfmm.BC_PBC, 0.9),
                                          (500, 10.0, 4, 8, mcfmm.BC_FREE, 0.6)])
def test_multipole_chain_replays_oracle(n, a, L, p, bc, h):
    g, o, _, _ = _pair(n, a, L, p, seed=n, bc=bc)
    steps = 2000 if n >= 500 else 800
    rg = g.run(steps, seed=4, beta=1.0, half_width=h, log=True)
    ro = o.run(steps, seed=4, step0=0, beta=1.0, half_width=h)
    assert ro["n_borderline"] == 0 and rg["borderline"] == 0
    assert np.array_equal(rg["j"], ro["j"])
    fin = np.isfinite(ro["dE"])
    assert np.array_equal(np.isfinite(rg["dE"]), fin)
    err = np.abs(rg["dE"][fin] - ro["dE"][fin]) / np.maximum(1.0, np.abs(ro["dE"][fin]))
    assert np.max(err) <= DE_TOL, np.max(err)
    assert np.array_equal(rg["acc"], ro["acc"])
    assert np.array_equal(g.positions(), o.positions())
    assert abs(g.energy() - o.energy()) <= 1e-9 * max(1.0, abs(o.energy()))
    lmin = 2 if bc == mcfmm.BC_PBC else 3
    for lev in range(lmin, L + 1):
        A, B = g.multipole(lev), o.multipole(lev)
        assert np.max(np.abs(A - B)) <= 1e-11 * np.max(np.abs(B)), lev
    g.close()


def test_multipole_single_propose_accept():
    g, o, pos, q = _pair(500, 8.0, 3, 10, seed=21)
    rng = np.random.default_rng(22)
    for _ in range(8):
        j = int(rng.integers(len(q)))
        rn = (o.positions()[j] + rng.uniform(-0.7, 0.7, 3)) % 8.0
        dg, do = g.propose(j, rn), o.propose(j, rn)
        assert abs(dg - do) <= DE_TOL * max(1.0, abs(do))
        g.accept(j, rn)
        o.accept(j, rn, do)
    assert abs(g.energy() - o.energy()) <= 1e-9 * max(1.0, abs(o.energy()))
    g.close()


def test_multipole_chain_equals_fresh_setup_and_fp32_tolerance():
    n, a, L, p = 10_000, (10_000 / 0.1) ** (1 / 3), 4, 12
    pos, q = uniform_system(n, a, seed=31)
    g = mcfmm.Context(pos, q, a, L, p)
    g.setup(mcfmm.SETUP_MULTIPOLE)
    g.run(20_000, seed=5, beta=1.0, half_width=0.3)
    f = mcfmm.Context(g.positions(), q, a, L, p)
    f.setup(mcfmm.SETUP_MULTIPOLE)
    for lev in range(2, L + 1):
        A, B = g.multipole(lev), f.multipole(lev)
        assert np.max(np.abs(A - B)) <= 1e-11 * np.max(np.abs(B)), lev
    # FP32-eval form against FP64 on the same states: the first proposals
    s32 = mcfmm.Context(pos, q, a, L, p, precision=mcfmm.FP32_EVAL)
    s32.setup(mcfmm.SETUP_MULTIPOLE)
    s64 = mcfmm.Context(pos, q, a, L, p)
    s64.setup(mcfmm.SETUP_MULTIPOLE)
    rng = np.random.default_rng(32)
    errs = []
    for _ in range(40):
        j = int(rng.integers(n))
        rn = (pos[j] + rng.uniform(-0.3, 0.3, 3)) % a
        d64, d32 = s64.propose(j, rn), s32.propose(j, rn)
        errs.append(abs(d32 - d64) / max(1.0, abs(d64)))
    assert np.percentile(errs, 95) <= 1e-4 and max(errs) <= 1e-3
    for c in (g, f, s32, s64):
        c.close()


def test_multipole_batch_replays_each_chain():
    ctxs, ors = [], []
    for i, (n, a, L) in enumerate([(300, 8.0, 3), (500, 9.0, 3), (200, 7.0, 2)]):
        pos, q = uniform_system(n, a, seed=40 + i)
        c = mcfmm.Context(pos, q, a, L, 6)
        c.setup(mcfmm.SETUP_MULTIPOLE)
        ctxs.append(c)
        o = O.System(pos, q, a, L, 6)
        o.setup_multipole()
        ors.append(o)
    b = mcfmm.Batch(ctxs)
    seeds = np.array([7, 8, 9], dtype=np.uint64)
    res = b.run(300, seeds, beta=1.0, half_width=0.5, log=True)
    for i, o in enumerate(ors):
        ro = o.run(300, seed=int(seeds[i]), step0=0, beta=1.0, half_width=0.5, chain=i)
        assert np.array_equal(res["acc"][i], ro["acc"])
        err = np.abs(res["dE"][i] - ro["dE"]) / np.maximum(1.0, np.abs(ro["dE"]))
        assert np.max(err) <= DE_TOL
    b.close()
    for c in ctxs:
        c.close()
