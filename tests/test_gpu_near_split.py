"""The split near-field sum (Alg. 1 over each near cell by several items)
against the oracle.

Dense cells (about 94 charges per finest cell: N = 6000 at density 0.1 on
three levels) with the split forced to 1..4 items per cell and side (2..8 per
cell when r and r' share their finest cell, each item taking every k-th
block of 32 slots, so some parts get one block, some two, some none), on
both chain schedules: every dE within 1e-10 max(1, |dE|) of the oracle's
chain and every decision identical.  The same with the Lennard-Jones term on
a perturbed NaCl crystal (64 ions per finest cell), in FP32-eval (the
oracle follows the GPU's decisions; beta |d dE| with p95 <= 1e-4 and max <=
1e-3), in the batched form with a forced split per chain, and in the
multipole method's chain.  The split changes the order of the near sum
only.
"""
import numpy as np
import pytest

import oracle as O
from paper_2006_16622_gb300 import mcfmm
from paper_2006_16622_gb300.workloads import (NACL_BETA, NACL_LJ_CUTOFF, NACL_LJ_EPS,
                                              NACL_LJ_SIGMA, perturbed_nacl, uniform_system)

pytestmark = pytest.mark.gpu

DE_TOL = 1e-10
N, L, P_EXP, H, STEPS = 6000, 3, 8, 0.5, 1500
A = (N / 0.1) ** (1.0 / 3.0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    mcfmm.load()


@pytest.fixture(scope="module")
def dense():
    pos, q = uniform_system(N, A, seed=21)
    o = O.System(pos, q, A, L, P_EXP)
    o.setup()
    ro = o.run(STEPS, seed=5, step0=0, beta=1.0, half_width=H)
    return pos, q, ro, o.positions(), o.energy()


def _check_replay(rg, ro):
    assert ro["n_borderline"] == 0 and rg["borderline"] == 0
    assert np.array_equal(rg["j"], ro["j"])
    # +inf (overlap, or a move out of a free-space box) on both sides alike
    fin = np.isfinite(ro["dE"])
    assert np.array_equal(np.isfinite(rg["dE"]), fin)
    assert np.array_equal(rg["dE"][~fin], ro["dE"][~fin])
    err = np.abs(rg["dE"][fin] - ro["dE"][fin]) / np.maximum(1.0, np.abs(ro["dE"][fin]))
    assert np.max(err) <= DE_TOL, np.max(err)
    assert np.array_equal(rg["acc"], ro["acc"])


def test_automatic_split_and_arguments():
    pos, q = uniform_system(N, A, seed=21)
    g = mcfmm.Context(pos, q, A, L, P_EXP)
    # ~94 charges per finest cell: two items per cell and side
    assert g.set_near_parts(0) == 2
    assert g.set_near_parts(4) == 4
    for bad in (-1, 5):
        with pytest.raises(RuntimeError):
            g.set_near_parts(bad)
    assert g.set_near_parts(0) == 2
    g.close()
    # sparse cells (N = 1000 on 3 levels, ~16 per cell): one item
    pos, q = uniform_system(1000, 10.0, seed=0)
    g = mcfmm.Context(pos, q, 10.0, 3, 8)
    assert g.set_near_parts(0) == 1
    g.close()


@pytest.mark.parametrize("schedule", [mcfmm.SCHEDULE_ASYNC, mcfmm.SCHEDULE_PHASED])
@pytest.mark.parametrize("parts", [1, 2, 3, 4])
def test_dense_cells_replay_oracle(dense, schedule, parts):
    pos, q, ro, pos_o, e_o = dense
    g = mcfmm.Context(pos, q, A, L, P_EXP)
    assert g.set_near_parts(parts) == parts
    g.setup()
    g.set_schedule(schedule)
    rg = g.run(STEPS, seed=5, beta=1.0, half_width=H, log=True)
    _check_replay(rg, ro)
    assert np.array_equal(g.positions(), pos_o)
    assert abs(g.energy() - e_o) <= 1e-9 * max(1.0, abs(e_o))
    g.close()


@pytest.mark.parametrize("schedule", [mcfmm.SCHEDULE_ASYNC, mcfmm.SCHEDULE_PHASED])
def test_lj_split_replays_oracle(schedule):
    pos, q, a = perturbed_nacl(8, seed=3)
    Lj, p = 2, 8
    o = O.System(pos, q, a, Lj, p)
    o.set_lj(NACL_LJ_EPS, NACL_LJ_SIGMA, NACL_LJ_CUTOFF)
    o.setup()
    ro = o.run(STEPS, seed=11, step0=0, beta=NACL_BETA, half_width=0.25)
    for parts in (2, 4):
        g = mcfmm.Context(pos, q, a, Lj, p)
        g.set_lj(NACL_LJ_EPS, NACL_LJ_SIGMA, NACL_LJ_CUTOFF)
        g.set_near_parts(parts)
        g.setup()
        g.set_schedule(schedule)
        rg = g.run(STEPS, seed=11, beta=NACL_BETA, half_width=0.25, log=True)
        _check_replay(rg, ro)
        assert np.array_equal(g.positions(), o.positions())
        g.close()


@pytest.mark.parametrize("schedule", [mcfmm.SCHEDULE_ASYNC, mcfmm.SCHEDULE_PHASED])
def test_fp32_eval_split_within_tolerance(dense, schedule):
    pos, q, _, _, _ = dense
    g = mcfmm.Context(pos, q, A, L, P_EXP, precision=mcfmm.FP32_EVAL)
    g.set_near_parts(3)
    g.setup()
    g.set_schedule(schedule)
    rg = g.run(STEPS, seed=6, beta=1.0, half_width=H, log=True)
    fin = g.positions()
    g.close()
    o = O.System(pos, q, A, L, P_EXP)
    o.setup()
    r = o.run_follow(rg["acc"], seed=6, step0=0, chain=0, beta=1.0, half_width=H)
    assert np.array_equal(rg["j"], r["j"])
    both = np.isfinite(rg["dE"]) & np.isfinite(r["dE"])
    assert np.array_equal(np.isfinite(rg["dE"]), np.isfinite(r["dE"]))
    e = np.abs(rg["dE"][both] - r["dE"][both])
    assert np.percentile(e, 95) <= 1e-4, np.percentile(e, 95)
    assert e.max() <= 1e-3, e.max()
    assert np.array_equal(fin, o.positions())


def test_batch_with_forced_split_replays_oracle():
    sizes = [(3000, 3), (4500, 3), (1500, 2)]
    ctxs, sys_ = [], []
    for i, (n, Lb) in enumerate(sizes):
        a = (n / 0.1) ** (1.0 / 3.0)
        pos, q = uniform_system(n, a, seed=100 + i)
        c = mcfmm.Context(pos, q, a, Lb, 6)
        assert c.set_near_parts(i + 2) == i + 2
        c.setup()
        ctxs.append(c)
        sys_.append((pos, q, a, Lb))
    b = mcfmm.Batch(ctxs)
    steps = 400
    seeds = np.arange(len(ctxs), dtype=np.uint64)
    rl = b.run(steps, seeds, beta=1.0, half_width=0.4, log=True)
    for i, (pos, q, a, Lb) in enumerate(sys_):
        o = O.System(pos, q, a, Lb, 6)
        o.setup()
        ro = o.run(steps, seed=i, step0=0, chain=i, beta=1.0, half_width=0.4)
        assert np.array_equal(rl["j"][i], ro["j"]), i
        err = np.abs(rl["dE"][i] - ro["dE"]) / np.maximum(1.0, np.abs(ro["dE"]))
        assert np.max(err) <= DE_TOL, (i, np.max(err))
        assert np.array_equal(rl["acc"][i], ro["acc"]), i
        assert np.array_equal(ctxs[i].positions(), o.positions()), i
    b.close()
    for c in ctxs:
        c.close()


def test_multipole_method_split_replays_oracle(dense):
    """The multipole method's chain (Alg. M.1-M.3) shares the near-field
    items: forced splits replay the oracle's multipole chain."""
    pos, q, _, _, _ = dense
    o = O.System(pos, q, A, L, P_EXP)
    o.setup_multipole()
    steps = 600
    ro = o.run(steps, seed=8, step0=0, beta=1.0, half_width=H)
    for parts in (2, 4):
        g = mcfmm.Context(pos, q, A, L, P_EXP)
        g.set_near_parts(parts)
        g.setup(mcfmm.SETUP_MULTIPOLE)
        rg = g.run(steps, seed=8, beta=1.0, half_width=H, log=True)
        _check_replay(rg, ro)
        assert np.array_equal(g.positions(), o.positions())
        g.close()


@pytest.mark.parametrize("schedule", [mcfmm.SCHEDULE_ASYNC, mcfmm.SCHEDULE_PHASED])
def test_free_space_split_replays_oracle(schedule):
    """Free space: near cells outside the box are skipped by every part; a
    move leaving the box is rejected (+inf) on both sides."""
    pos, q = uniform_system(N, A, seed=22)
    o = O.System(pos, q, A, L, P_EXP, bc=mcfmm.BC_FREE)
    o.setup()
    steps = 800
    ro = o.run(steps, seed=12, step0=0, beta=1.0, half_width=H)
    g = mcfmm.Context(pos, q, A, L, P_EXP, bc=mcfmm.BC_FREE)
    g.set_near_parts(3)
    g.setup()
    g.set_schedule(schedule)
    rg = g.run(steps, seed=12, beta=1.0, half_width=H, log=True)
    _check_replay(rg, ro)
    assert np.array_equal(g.positions(), o.positions())
    g.close()
