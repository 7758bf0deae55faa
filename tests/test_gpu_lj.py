"""The short-range Lennard-Jones term (Sec. 5.3) on the GPU against the oracle.

A perturbed 8^3 NaCl crystal (spacing 3.3 A, 2 levels: finest cells of
13.2 A hold every pair within the 12 A cutoff) at T = 273 K with moves of
+-0.25 A: setup energy within 1e-10, replayed chains of both methods with
every dE within 1e-10 max(1, |dE|) and every decision identical.
"""
import numpy as np
import pytest

import oracle as O
from paper_2006_16622_gb300 import mcfmm
from paper_2006_16622_gb300.workloads import (NACL_BETA, NACL_LJ_CUTOFF, NACL_LJ_EPS,
                                              NACL_LJ_SIGMA, perturbed_nacl)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    mcfmm.load()


@pytest.mark.parametrize("method", ["local", "local-phased", "multipole"])
def test_lj_chain_replays_oracle(method):
    pos, q, a = perturbed_nacl(8, seed=3)
    L, p = 2, 8
    g = mcfmm.Context(pos, q, a, L, p)
    if method == "local-phased":
        g.set_schedule(mcfmm.SCHEDULE_PHASED)
    g.set_lj(NACL_LJ_EPS, NACL_LJ_SIGMA, NACL_LJ_CUTOFF)
    o = O.System(pos, q, a, L, p)
    o.set_lj(NACL_LJ_EPS, NACL_LJ_SIGMA, NACL_LJ_CUTOFF)
    if method != "multipole":
        g.setup()
        o.setup()
    else:
        g.setup(mcfmm.SETUP_MULTIPOLE)
        o.setup_multipole()
    assert abs(g.energy() - o.energy()) <= 1e-10 * abs(o.energy())
    steps = 1500
    rg = g.run(steps, seed=11, beta=NACL_BETA, half_width=0.25, log=True)
    ro = o.run(steps, seed=11, step0=0, beta=NACL_BETA, half_width=0.25)
    assert ro["n_borderline"] == 0 and rg["borderline"] == 0
    err = np.abs(rg["dE"] - ro["dE"]) / np.maximum(1.0, np.abs(ro["dE"]))
    assert np.max(err) <= 1e-10, np.max(err)
    assert np.array_equal(rg["acc"], ro["acc"])
    assert 0.05 < rg["accepted"] / steps < 0.95
    assert np.array_equal(g.positions(), o.positions())
    assert abs(g.energy() - o.energy()) <= 1e-9 * abs(o.energy())
    g.close()


def test_lj_arguments_and_switch_off():
    pos, q, a = perturbed_nacl(8, seed=4)
    g = mcfmm.Context(pos, q, a, 2, 6)
    with pytest.raises(mcfmm.McError):
        g.set_lj(NACL_LJ_EPS, NACL_LJ_SIGMA, 13.5)  # beyond the finest cell width (13.2)
    g.setup()
    e0 = g.energy()
    g.set_lj(NACL_LJ_EPS, NACL_LJ_SIGMA, NACL_LJ_CUTOFF)
    with pytest.raises(mcfmm.McError):
        g.run(10, seed=1)  # set up again first
    g.setup()
    assert g.energy() != e0
    g.set_lj(0.0, NACL_LJ_SIGMA, NACL_LJ_CUTOFF)
    g.setup()
    assert g.energy() == e0
    g.close()
