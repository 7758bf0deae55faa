"""Failure detection on the GPU without a GPU fault.

Every device-side wait of the persistent chain kernel is bounded by wall
time.  The test makes the grid barrier wait for one CTA that never arrives
(mc_inject_wait_fault): the wait runs out, mc_run returns MC_ERR_TIMEOUT
within the limit, nothing of the chain is applied, and the same context then
runs a normal chain that replays the oracle.
"""
import time

import numpy as np
import pytest

import oracle as O
from paper_2006_16622_gb300 import mcfmm
from paper_2006_16622_gb300.workloads import uniform_system

pytestmark = pytest.mark.gpu

MC_ERR_TIMEOUT = -7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    mcfmm.load()


def test_barrier_wait_runs_out_and_context_stays_usable():
    n, a, L, p = 300, 8.0, 3, 8
    pos, q = uniform_system(n, a, seed=4)
    g = mcfmm.Context(pos, q, a, L, p)
    g.setup()
    e0, x0 = g.energy(), g.positions().copy()
    g.set_wait_limit(200_000_000)  # 0.2 s
    g.inject_wait_fault(1)
    t0 = time.perf_counter()
    with pytest.raises(mcfmm.McError) as err:
        g.run(1000, seed=1, beta=1.0, half_width=0.5)
    elapsed = time.perf_counter() - t0
    assert err.value.code == MC_ERR_TIMEOUT
    assert elapsed < 5.0
    assert np.array_equal(g.positions(), x0)
    assert g.energy() == e0
    # back to normal: the same context replays the oracle's chain
    g.inject_wait_fault(0)
    g.set_wait_limit(2_000_000_000)
    rg = g.run(200, seed=1, beta=1.0, half_width=0.5, log=True)
    o = O.System(pos, q, a, L, p)
    o.setup()
    ro = o.run(200, seed=1, step0=0, beta=1.0, half_width=0.5)
    assert ro["n_borderline"] == 0 and rg["borderline"] == 0
    assert np.array_equal(rg["acc"], ro["acc"])
    assert np.array_equal(g.positions(), o.positions())
    g.close()


def test_fault_injection_argument_checks():
    pos, q = uniform_system(50, 4.0, seed=2)
    g = mcfmm.Context(pos, q, 4.0, 2, 4)
    with pytest.raises(mcfmm.McError):
        g.inject_wait_fault(-1)
    with pytest.raises(mcfmm.McError):
        g.inject_wait_fault(5000)
    g.close()
