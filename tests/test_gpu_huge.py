"""Parity at the N = 1e6 configuration (uniform +-1 charges at density 0.1,
6 levels, p = 12), where the oracle's full setup is too slow for a test:

  - sampled cells of the Alg. L.3 setup on levels 3..6 against the oracle's
    expansion of the same cells by definition (gathered from the charges of
    their interaction lists, no oracle setup), within 1e-12 of the level's
    largest coefficient;
  - the fast setup (the configuration's timed setup pass) within the
    multipole truncation of the Alg. L.3 setup;
  - properties that hold at any size after 10^4 moves of the FP64 chain in
    the launch configuration bench.py times: the running energy within
    truncation of a fresh evaluation, and the incrementally updated
    expansions equal to a fresh setup on the final positions (1e-11);
  - the FP32-eval chain from the same initial state: the running energy
    within the accumulated per-move tolerance (1e-3 per accepted move) of a
    fresh FP64 evaluation, its FP64 accumulators within 1e-5 of a fresh
    setup.
"""
import numpy as np
import pytest

import oracle as O
from paper_2006_16622_gb300 import mcfmm
from paper_2006_16622_gb300.workloads import HUGE

pytestmark = pytest.mark.gpu

STEPS = 10_000


@pytest.fixture(scope="module")
def huge():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    W = HUGE
    pos, q = W.system()
    return W, pos, q


def test_huge_setup_sampled_cells(huge):
    W, pos, q = huge
    g = mcfmm.Context(pos, q, W.a, W.levels, W.p)
    g.setup(mcfmm.SETUP_P2L)
    exact = {lev: g.local(lev).copy() for lev in range(2, W.levels + 1)}
    o = O.System(pos, q, W.a, W.levels, W.p)  # never set up
    rng = np.random.default_rng(17)
    # cells per level: the coarse ones gather from ~2e5..3e6 charges each
    for lev, k in ((W.levels, 4), (W.levels - 1, 3), (W.levels - 2, 2), (W.levels - 3, 1)):
        nl = 1 << (lev - 1)
        scale = np.max(np.abs(exact[lev]))
        for _ in range(k):
            c = rng.integers(0, nl, size=3)
            ref = o.local_cell_direct(lev, c)
            got = exact[lev][(c[0] * nl + c[1]) * nl + c[2]]
            assert np.max(np.abs(got - ref)) <= 1e-12 * scale, (lev, c)
    # the configuration's fast setup: equal up to the multipole truncation
    g.setup(mcfmm.SETUP_FMM)
    for lev in range(2, W.levels + 1):
        A = g.local(lev)
        assert np.max(np.abs(A - exact[lev])) <= 1e-6 * np.max(np.abs(exact[lev])), lev
    g.close()


def _fresh_local(pos, q, W):
    f = mcfmm.Context(pos, q, W.a, W.levels, W.p)
    f.setup(mcfmm.SETUP_P2L)
    out = {lev: f.local(lev).copy() for lev in range(2, W.levels + 1)}
    f.close()
    return out


def test_huge_fp64_chain_properties(huge):
    W, pos, q = huge
    g = mcfmm.Context(pos, q, W.a, W.levels, W.p)
    g.setup(mcfmm.SETUP_P2L)
    r = g.run(STEPS, seed=W.seed, beta=W.beta, half_width=W.half_width)
    assert r["steps"] == STEPS and r["borderline"] == 0 and g.status() == 0
    assert 0.5 < r["accepted"] / STEPS < 1.0
    fresh = g.energy_fresh()
    assert abs(g.energy() - fresh) <= 1e-6 * abs(fresh)
    ref = _fresh_local(g.positions(), q, W)
    for lev in range(2, W.levels + 1):
        A = g.local(lev)
        assert np.max(np.abs(A - ref[lev])) <= 1e-11 * np.max(np.abs(ref[lev])), lev
    g.close()


def test_huge_fp32_eval_chain_properties(huge):
    W, pos, q = huge
    g = mcfmm.Context(pos, q, W.a, W.levels, W.p, precision=mcfmm.FP32_EVAL)
    g.setup(mcfmm.SETUP_P2L)
    r = g.run(STEPS, seed=W.seed, beta=W.beta, half_width=W.half_width)
    assert r["steps"] == STEPS and g.status() == 0
    fin = g.positions()
    assert np.all(np.isfinite(fin)) and np.all((fin >= 0.0) & (fin < W.a))
    fresh = g.energy_fresh()
    assert abs(g.energy() - fresh) <= 1e-6 * abs(fresh) + 1e-3 * r["accepted"]
    ref = _fresh_local(fin, q, W)
    for lev in range(2, W.levels + 1):
        A = g.local(lev)
        assert np.max(np.abs(A - ref[lev])) <= 1e-5 * np.max(np.abs(ref[lev])), lev
    g.close()
