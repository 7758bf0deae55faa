"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64 form: per-proposal dE within 1e-10 max(1, |dE|) of the oracle, every
Metropolis decision identical, setup arrays within 1e-12 of the largest
coefficient of their level.  Inputs come from the seeded generators of
paper_2006_16622_gb300.workloads; the oracle never sees a CUDA output.
"""
import numpy as np
import pytest

import oracle as O
from paper_2006_16622_gb300 import mcfmm
from paper_2006_16622_gb300.workloads import rocksalt, uniform_system

pytestmark = pytest.mark.gpu

DE_TOL = 1e-10
ARR_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    mcfmm.load()


def _pair(n, a, L, p, seed=0, bc=mcfmm.BC_PBC, precision=mcfmm.FP64, pos=None, q=None):
    if pos is None:
        pos, q = uniform_system(n, a, seed=seed)
    g = mcfmm.Context(pos, q, a, L, p, bc=bc, precision=precision)
    g.setup()
    o = O.System(pos, q, a, L, p, bc=bc)
    o.setup()
    return g, o, pos, q


def _rel(x, ref):
    return abs(x - ref) / max(1.0, abs(ref))


def test_lattice_sums_match_oracle():
    for lmax in (16, 24, 30):
        S_g = mcfmm.lattice_sums(lmax)
        S_o = O.lattice_sums(lmax)
        scale = np.max(np.abs(S_o))
        assert np.max(np.abs(S_g - S_o)) <= 1e-12 * scale, lmax


@pytest.mark.parametrize("n,a,L,p", [(64, 4.0, 2, 6), (300, 8.0, 3, 8), (600, 9.0, 4, 10),
                                     (1000, 10.0, 3, 12), (700, 10.0, 4, 15)])
def test_setup_arrays_and_energy(n, a, L, p):
    g, o, pos, q = _pair(n, a, L, p, seed=n)
    for lev in range(2, L + 1):
        A, B = g.local(lev), o.local(lev)
        assert np.max(np.abs(A - B)) <= ARR_TOL * np.max(np.abs(B)), lev
    Kg, Hg = g.far()
    Ko, Ho = o.KH()
    assert np.max(np.abs(Kg - Ko)) <= ARR_TOL * np.max(np.abs(Ko))
    assert np.max(np.abs(Hg - Ho)) <= 1e-11 * max(1e-300, np.max(np.abs(Ho)))
    assert _rel(g.energy(), o.energy()) <= DE_TOL


@pytest.mark.parametrize("bc", [mcfmm.BC_PBC, mcfmm.BC_FREE])
def test_propose_accept_sequence(bc):
    n, a, L, p = 800, 10.0, 4, 10
    g, o, pos, q = _pair(n, a, L, p, seed=7, bc=bc)
    rng = np.random.default_rng(3)
    for t in range(40):
        j = int(rng.integers(n))
        r = o.positions()[j]
        step = rng.uniform(-1.0, 1.0, 3) * (4.0 if t % 7 == 0 else 0.6)  # some far moves
        rn = (r + step) % a if bc == mcfmm.BC_PBC else np.clip(r + step, 0.0, a - 1e-9)
        dg, do = g.propose(j, rn), o.propose(j, rn)
        assert _rel(dg, do) <= DE_TOL, (t, dg, do)
        if t % 3 != 2:
            g.accept(j, rn, dg)
            o.accept(j, rn, do)
    assert np.array_equal(g.positions(), o.positions())
    for lev in range(2, L + 1):
        A, B = g.local(lev), o.local(lev)
        assert np.max(np.abs(A - B)) <= ARR_TOL * np.max(np.abs(B))
    assert _rel(g.energy(), o.energy()) <= DE_TOL
    # accept without a given dE recomputes it (the paper's accept())
    j = 11
    rn = (o.positions()[j] + 0.25) % a
    do = o.propose(j, rn)
    g.accept(j, rn)
    o.accept(j, rn, do)
    assert _rel(g.energy(), o.energy()) <= DE_TOL


@pytest.mark.parametrize("schedule", [mcfmm.SCHEDULE_PHASED, mcfmm.SCHEDULE_PLAIN,
                                      mcfmm.SCHEDULE_ASYNC])
def test_replay_small_workload_full_chain(schedule):
    """N=1000, a=10, L=3, p=8, h=0.5, beta=1, seed 0: the full 10^4-move chain"""
    n, a, L, p = 1000, 10.0, 3, 8
    g, o, pos, q = _pair(n, a, L, p, seed=0)
    g.set_schedule(schedule)
    steps = 10_000
    rg = g.run(steps, seed=0, beta=1.0, half_width=0.5, log=True)
    ro = o.run(steps, seed=0, step0=0, beta=1.0, half_width=0.5)
    assert ro["n_borderline"] == 0 and rg["borderline"] == 0
    assert np.array_equal(rg["j"], ro["j"])
    err = np.abs(rg["dE"] - ro["dE"]) / np.maximum(1.0, np.abs(ro["dE"]))
    assert np.max(err) <= DE_TOL, np.max(err)
    assert np.array_equal(rg["acc"], ro["acc"])
    assert rg["accepted"] == ro["n_acc"]
    assert _rel(g.energy(), o.energy()) <= 1e-9
    assert np.array_equal(g.positions(), o.positions())


@pytest.mark.parametrize("schedule", [mcfmm.SCHEDULE_PHASED, mcfmm.SCHEDULE_PLAIN,
                                      mcfmm.SCHEDULE_ASYNC])
def test_replay_ragged_and_edge_cases(schedule):
    # tiny box with 2 cells per axis (27 image copies of every cell), p = 0
    for (n, a, L, p) in [(16, 3.0, 2, 0), (40, 5.0, 2, 3), (126, 7.0, 3, 5), (900, 9.0, 4, 7)]:
        g, o, pos, q = _pair(n, a, L, p, seed=n)
        g.set_schedule(schedule)
        rg = g.run(500, seed=9, beta=0.7, half_width=0.9, log=True)
        ro = o.run(500, seed=9, step0=0, beta=0.7, half_width=0.9)
        assert np.array_equal(rg["acc"], ro["acc"])
        err = np.abs(rg["dE"] - ro["dE"]) / np.maximum(1.0, np.abs(ro["dE"]))
        assert np.max(err) <= DE_TOL
    # rock salt: exact lattice, moves from lattice sites
    pos, q, a = rocksalt(6)
    g, o, _, _ = _pair(len(q), a, 3, 8, pos=pos, q=q)
    assert _rel(g.energy(), o.energy()) <= DE_TOL
    rn = pos[3] + np.array([0.2, 0.1, -0.05])
    assert _rel(g.propose(3, rn), o.propose(3, rn)) <= DE_TOL
    # a proposal onto another charge is rejected (+inf on both sides)
    assert g.propose(3, pos[4]) == np.inf and o.propose(3, pos[4]) == np.inf
    # no move
    assert g.propose(3, pos[3]) == 0.0


def test_fp32_eval_error_against_fp64_oracle():
    n, a, L, p = 1000, 10.0, 3, 12
    g, o, pos, q = _pair(n, a, L, p, seed=5, precision=mcfmm.FP32_EVAL)
    rng = np.random.default_rng(8)
    errs = []
    for t in range(200):
        j = int(rng.integers(n))
        rn = (o.positions()[j] + rng.uniform(-0.3, 0.3, 3)) % a
        dg, do = g.propose(j, rn), o.propose(j, rn)
        errs.append(abs(dg - do))
        if t % 2 == 0:
            g.accept(j, rn, do)
            o.accept(j, rn, do)
    errs = np.array(errs)
    assert np.percentile(errs, 95) <= 1e-4 and errs.max() <= 1e-3, (np.percentile(errs, 95), errs.max())
    # the FP64 accumulators stay within FP32 rounding of the oracle's
    for lev in range(2, L + 1):
        A, B = g.local(lev), o.local(lev)
        assert np.max(np.abs(A - B)) <= 1e-5 * np.max(np.abs(B))
