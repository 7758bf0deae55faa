"""Batched form: independent chains of uneven size in one persistent launch.

Each chain of the batch must replay its own oracle chain exactly (same seed,
Philox counter word 2 = chain index): every dE within 1e-10 max(1, |dE|) and
every decision identical, although the chains share the GPU and run on CTA
groups of different sizes.  The autotuned, graph-replayed runs keep every
chain consistent (running energy within truncation of a fresh evaluation).
"""
import numpy as np
import pytest

import oracle as O
from paper_2006_16622_gb300 import mcfmm
from paper_2006_16622_gb300.workloads import uniform_system

pytestmark = pytest.mark.gpu

SIZES = [(120, 3), (400, 3), (1000, 4), (1800, 4), (256, 3)]  # (N, levels), density 0.3
P = 6


def _systems():
    out = []
    for i, (n, L) in enumerate(SIZES):
        a = (n / 0.3) ** (1.0 / 3.0)
        pos, q = uniform_system(n, a, seed=100 + i)
        out.append((pos, q, a, L))
    return out


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    mcfmm.load()


@pytest.mark.parametrize("precision,schedule", [(mcfmm.FP64, mcfmm.SCHEDULE_PHASED),
                                                (mcfmm.FP64, mcfmm.SCHEDULE_PLAIN)])
def test_batch_replays_every_chain(precision, schedule):
    syst = _systems()
    ctxs = []
    for pos, q, a, L in syst:
        c = mcfmm.Context(pos, q, a, L, P, precision=precision)
        c.setup()
        ctxs.append(c)
    b = mcfmm.Batch(ctxs)
    b.set_schedule(schedule)
    seeds = np.arange(len(ctxs), dtype=np.uint64) + 7
    steps = 400
    r = b.run(steps, seeds, beta=1.0, half_width=0.4, log=True)
    for i, (pos, q, a, L) in enumerate(syst):
        o = O.System(pos, q, a, L, P)
        o.setup()
        ro = o.run(steps, seed=int(seeds[i]), step0=0, chain=i, beta=1.0, half_width=0.4)
        assert np.array_equal(r["j"][i], ro["j"]), i
        err = np.abs(r["dE"][i] - ro["dE"]) / np.maximum(1.0, np.abs(ro["dE"]))
        assert np.max(err) <= 1e-10, (i, np.max(err))
        assert np.array_equal(r["acc"][i], ro["acc"]), i
        assert r["stats"][i]["steps"] == steps
        assert np.array_equal(ctxs[i].positions(), o.positions())
    b.close()
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("precision", [mcfmm.FP64, mcfmm.FP32_EVAL])
def test_batch_tuned_graph_runs(precision):
    syst = _systems()
    ctxs = []
    for pos, q, a, L in syst:
        c = mcfmm.Context(pos, q, a, L, P, precision=precision)
        c.setup()
        ctxs.append(c)
    b = mcfmm.Batch(ctxs)
    b.tune(trial_steps=200, half_width=0.4)
    ctas, nf = b.info()
    assert ctas.min() >= 1 and 1 <= nf <= 16
    seeds = np.arange(len(ctxs), dtype=np.uint64) + 11
    for _ in range(3):  # first run captures the graph, then replays
        r = b.run(300, seeds, half_width=0.4)
        for st in r["stats"]:
            assert st["steps"] == 300 and 0 < st["accepted"] <= 300
    for c in ctxs:
        e, f = c.energy(), c.energy_fresh()
        assert abs(e - f) <= 1e-4 * max(1.0, abs(f))
    b.close()
    for c in ctxs:
        c.close()
