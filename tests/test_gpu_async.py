"""The barrier-free chain schedule (MC_SCHEDULE_ASYNC) against the oracle.

The same Alg. L.1 / L.2 chain as the phased schedule, with the steps'
geometry published ahead of the previous decision and every wait on data
(partial slots, counters) instead of barriers: the replayed chains must
give every decision of the oracle and every dE within 1e-10 max(1, |dE|)
(FP64), also in free space, over several launches (the chain continued
across mc_run calls), with the periodic re-setup (which stops a launch
after a number of accepts, leaving a step published early undone), and
with a proposal that draws the particle of the step before (whose geometry
waits for that step's decision).  FP32-eval: within the FP32 tolerance of
the oracle, same decisions on these seeds.
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


def _ctx(pos, q, a, L, p, bc=mcfmm.BC_PBC, precision=mcfmm.FP64):
    g = mcfmm.Context(pos, q, a, L, p, bc=bc, precision=precision)
    g.setup()
    g.set_schedule(mcfmm.SCHEDULE_ASYNC)
    return g


def _check(dE, acc, ro, tol=DE_TOL):
    err = np.abs(dE - ro["dE"]) / np.maximum(1.0, np.abs(ro["dE"]))
    assert np.max(err) <= tol, np.max(err)
    assert np.array_equal(acc, ro["acc"])


def test_default_schedule_by_precision():
    # FP64 contexts run the barrier-free chain by default, FP32-eval ones the
    # phased chain: told apart by the profile counters (the phased chain
    # times its decisions in counter 2, the barrier-free one leaves it 0)
    pos, q = uniform_system(300, 8.0, seed=1)
    for prec, async_default in ((mcfmm.FP64, True), (mcfmm.FP32_EVAL, False)):
        g = mcfmm.Context(pos, q, 8.0, 3, 6, precision=prec)
        g.setup()
        g.profile(True)
        g.profile_read()
        g.run(200, seed=1, beta=1.0, half_width=0.5, stats=False)
        pr = g.profile_read()
        g.profile(False)
        assert pr[5] == 200
        assert (pr[2] == 0) == async_default, pr[:8]
        with pytest.raises(mcfmm.McError):
            g.set_schedule(7)
        with pytest.raises(mcfmm.McError):  # the withdrawn pipelined schedule
            g.set_schedule(mcfmm.SCHEDULE_PIPELINED)
        g.close()


@pytest.mark.parametrize("n,a,L,p,bc", [(500, 10.0, 4, 8, mcfmm.BC_FREE), (300, 8.0, 3, 6, mcfmm.BC_FREE),
                                        (2000, 12.0, 4, 10, mcfmm.BC_PBC)])
def test_async_replays_oracle(n, a, L, p, bc):
    pos, q = uniform_system(n, a, seed=n + L)
    g = _ctx(pos, q, a, L, p, bc=bc)
    o = O.System(pos, q, a, L, p, bc=bc)
    o.setup()
    steps = 1500
    rg = g.run(steps, seed=5, beta=1.0, half_width=0.6, log=True)
    ro = o.run(steps, seed=5, step0=0, beta=1.0, half_width=0.6)
    assert ro["n_borderline"] == 0 and rg["borderline"] == 0
    assert np.array_equal(rg["j"], ro["j"])
    fin = np.isfinite(ro["dE"])
    assert np.array_equal(np.isfinite(rg["dE"]), fin)
    _check(np.where(fin, rg["dE"], 0.0), rg["acc"], {"dE": np.where(fin, ro["dE"], 0.0), "acc": ro["acc"]})
    assert np.array_equal(g.positions(), o.positions())
    assert abs(g.energy() - o.energy()) <= 1e-9 * max(1.0, abs(o.energy()))
    g.close()


def test_async_continued_launches_and_resetup():
    n, a, L, p = 1000, 10.0, 3, 8
    pos, q = uniform_system(n, a, seed=0)
    o = O.System(pos, q, a, L, p)
    o.setup()
    ro = o.run(900, seed=0, step0=0, beta=1.0, half_width=0.5)
    g = _ctx(pos, q, a, L, p)
    parts = [g.run(k, seed=0, beta=1.0, half_width=0.5, log=True) for k in (1, 299, 600)]
    _check(np.concatenate([r["dE"] for r in parts]), np.concatenate([r["acc"] for r in parts]), ro)
    assert np.array_equal(g.positions(), o.positions())
    g.close()
    # re-setup every 37 accepts: each launch stops after 37 accepts
    g = _ctx(pos, q, a, L, p)
    rg = g.run(900, seed=0, beta=1.0, half_width=0.5, resetup_every=37, log=True)
    _check(rg["dE"], rg["acc"], ro)
    assert np.array_equal(g.positions(), o.positions())
    g.close()


def test_async_proposal_of_the_same_particle_twice():
    # 8 charges: consecutive proposals often draw the same particle, whose
    # geometry must wait for the previous step's decision
    rng = np.random.default_rng(3)
    a, L, p = 4.0, 2, 6
    pos = rng.uniform(0.0, a, size=(8, 3))
    q = np.array([1.0, -1.0] * 4)
    o = O.System(pos, q, a, L, p)
    o.setup()
    ro = o.run(400, seed=2, step0=0, beta=1.0, half_width=0.4)
    assert np.any(ro["j"][1:] == ro["j"][:-1])
    g = _ctx(pos, q, a, L, p)
    rg = g.run(400, seed=2, beta=1.0, half_width=0.4, log=True)
    assert np.array_equal(rg["j"], ro["j"])
    _check(rg["dE"], rg["acc"], ro)
    assert np.array_equal(g.positions(), o.positions())
    g.close()


def test_async_fp32_eval_within_tolerance():
    n, a, L, p = 1000, 10.0, 3, 10
    pos, q = uniform_system(n, a, seed=9)
    o = O.System(pos, q, a, L, p)
    o.setup()
    ro = o.run(600, seed=4, step0=0, beta=1.0, half_width=0.5)
    g = _ctx(pos, q, a, L, p, precision=mcfmm.FP32_EVAL)
    rg = g.run(600, seed=4, beta=1.0, half_width=0.5, log=True)
    err = np.abs(rg["dE"] - ro["dE"])
    assert np.percentile(err, 95) <= 1e-4 and err.max() <= 1e-3
    assert np.array_equal(rg["acc"], ro["acc"])
    g.close()
