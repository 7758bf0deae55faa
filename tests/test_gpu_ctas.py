"""Chains on fewer CTAs than SMs (mc_set_ctas) against the oracle.

The items of a step are dealt over the warps of the grid and their partial
results combined in one fixed order, so the chain must replay the oracle on
any grid: every decision identical and every dE within 1e-10 max(1, |dE|)
(FP64) for each schedule, also on grids so small that a warp takes many
items of a kind and the far-field items read the far operator's columns
from memory instead of registers.
"""
import numpy as np
import pytest

import oracle as O
from paper_2006_16622_gb300 import mcfmm
from paper_2006_16622_gb300.workloads import uniform_system

pytestmark = pytest.mark.gpu

DE_TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    mcfmm.load()


@pytest.fixture(scope="module")
def system():
    n, a, L, p = 1200, 10.0, 4, 8
    pos, q = uniform_system(n, a, seed=41)
    o = O.System(pos, q, a, L, p)
    o.setup()
    ro = o.run(600, seed=9, step0=0, beta=1.0, half_width=0.6)
    assert ro["n_borderline"] == 0
    return pos, q, a, L, p, ro


@pytest.mark.parametrize("schedule", [mcfmm.SCHEDULE_ASYNC, mcfmm.SCHEDULE_PHASED,
                                      mcfmm.SCHEDULE_PLAIN])
@pytest.mark.parametrize("n_cta", [3, 37, 100])
def test_small_grid_replays_oracle(system, schedule, n_cta):
    pos, q, a, L, p, ro = system
    g = mcfmm.Context(pos, q, a, L, p)
    g.setup()
    g.set_schedule(schedule)
    g.set_ctas(n_cta)
    rg = g.run(600, seed=9, beta=1.0, half_width=0.6, log=True)
    assert g.status() == 0
    assert np.array_equal(rg["j"], ro["j"])
    err = np.abs(rg["dE"] - ro["dE"]) / np.maximum(1.0, np.abs(ro["dE"]))
    assert np.max(err) <= DE_TOL, np.max(err)
    assert np.array_equal(rg["acc"], ro["acc"])
    g.close()


def test_set_ctas_range(system):
    import torch
    pos, q, a, L, p, _ = system
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    g = mcfmm.Context(pos, q, a, L, p)
    for bad in (-1, sms + 1):
        with pytest.raises(mcfmm.McError):
            g.set_ctas(bad)
    g.set_ctas(sms)
    g.set_ctas(0)  # back to the default grid
    g.close()
