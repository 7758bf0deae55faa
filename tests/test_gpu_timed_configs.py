"""The configurations bench.py times, replayed against the oracle.

* Batched FP64: the benchmark's 64 chains (N log-uniform in [1000, 50000],
  density 0.1, ~20 charges per finest cell, levels 3..5, p = 10, h = 0.3,
  beta = 1, seed i for chain i) in the default batch schedule (speculative
  Alg. L.2 contributions in pair-of-floats arithmetic, FP64 accumulators),
  with the CTA split and far-field tiles picked by mc_batch_tune and the
  chains run by graph-replayed mc_batch_run.  Every chain must end where its
  oracle chain ends: the same positions bit for bit and the running energy
  within 1e-9 max(1, |E|); a logged run on the same tuned split then gives every
  dE within 1e-10 max(1, |dE|) and every decision identical.
* Batched FP32-eval: the same 64 chains, tuned and graph-replayed; then a
  logged run whose states the oracle follows (it takes the GPU's decisions):
  beta |dE_gpu - dE_oracle| has p95 <= 1e-4 and max <= 1e-3, the stated
  tolerance of the FP32-eval form (below the paper's acceptance-probability
  error of about 1e-3 at p = 11, Sec. 5.1, since dP ~ beta |d dE|).
* FP32-eval mc_run with a full FP64 re-setup every R accepts: the same
  tolerance across the re-setups, positions equal to the oracle's, and the
  recorded drift finite and below R x 1e-4 (every accepted move within the
  p95 tolerance, added up in the worst case).

The oracle chains run in spawned processes, one per host core (each chain's
setup takes up to ~40 s of one core at N = 5e4).
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle as O
from paper_2006_16622_gb300 import mcfmm
from paper_2006_16622_gb300.workloads import batched_systems, uniform_system

pytestmark = pytest.mark.gpu

P_BATCH = 10
H = 0.3
BETA = 1.0
TUNE_STEPS = 60      # trial proposals per tuning launch
GRAPH_STEPS = 200    # proposals per graph-replayed launch
GRAPH_RUNS = 3       # the first captures the graph, the others replay it
LOG_STEPS = 150
TUNE_SEED0 = 0x5EED  # the autotuner's seeds: 0x5EED + chain index
FP32_P95, FP32_MAX = 1e-4, 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    mcfmm.load()


def _pool():
    k = max(1, min(os.cpu_count() or 1, 32))
    return mp.get_context("spawn").Pool(processes=k)


def _bench_batch():
    """the benchmark's 64 chains: (N, box, levels, chain index)"""
    return batched_systems(64, 1000, 50000, 0.1, 20.0)


def _oracle_replay_fp64(task):
    """The oracle chain of one batched FP64 chain: the tuner's trial runs,
    the graph-replayed runs, then a logged run (spawned process)."""
    n, a, L, i, tuned, graphed, log_steps = task
    import oracle
    from paper_2006_16622_gb300.workloads import uniform_system as us
    pos, q = us(n, a, seed=1000 + i)
    o = oracle.System(pos, q, a, L, P_BATCH)
    o.setup()
    o.run(tuned, seed=TUNE_SEED0 + i, step0=0, chain=i, beta=BETA, half_width=H, log=False)
    o.run(graphed, seed=i, step0=tuned, chain=i, beta=BETA, half_width=H, log=False)
    mid = (o.positions(), o.energy())
    r = o.run(log_steps, seed=i, step0=tuned + graphed, chain=i, beta=BETA, half_width=H)
    return i, mid, (r["j"], r["dE"], r["acc"], r["n_borderline"]), o.positions()


def _oracle_follow(task):
    """The oracle on a GPU chain's current positions, following its decisions
    (spawned process): the FP64 energy changes of the same states."""
    pos, q, a, L, p, seed, step0, chain, beta, h, follow = task
    import oracle
    o = oracle.System(pos, q, a, L, p)
    o.setup()
    r = o.run_follow(follow, seed=seed, step0=step0, chain=chain, beta=beta, half_width=h)
    return r["j"], r["dE"], r["acc"], o.positions()


def _batch_contexts(precision):
    ctxs = []
    for n, a, L, i in _bench_batch():
        pos, q = uniform_system(n, a, seed=1000 + i)
        c = mcfmm.Context(pos, q, a, L, P_BATCH, precision=precision)
        c.setup()
        ctxs.append(c)
    return ctxs


def _tuned_graphed(ctxs):
    """tune, then GRAPH_RUNS graph launches; returns the batch and the step
    counters after the tuner"""
    b = mcfmm.Batch(ctxs)
    b.tune(trial_steps=TUNE_STEPS, beta=BETA, half_width=H)
    ctas, nf = b.info()
    assert ctas.min() >= 1 and 1 <= nf <= 16
    tuned = [c.step_counter() for c in ctxs]
    seeds = np.arange(len(ctxs), dtype=np.uint64)
    for k in range(GRAPH_RUNS):
        r = b.run(GRAPH_STEPS, seeds, beta=BETA, half_width=H, stats=(k == GRAPH_RUNS - 1))
    for st in r["stats"]:
        assert st["steps"] == GRAPH_STEPS
    for c, t in zip(ctxs, tuned):
        assert c.step_counter() == t + GRAPH_RUNS * GRAPH_STEPS
        assert c.status() == 0
    return b, tuned, seeds


def test_batched_fp64_bench_workload_replays_oracle():
    ctxs = _batch_contexts(mcfmm.FP64)
    b, tuned, seeds = _tuned_graphed(ctxs)
    mids = [(c.positions(), c.energy()) for c in ctxs]
    rl = b.run(LOG_STEPS, seeds, beta=BETA, half_width=H, log=True)
    finals = [c.positions() for c in ctxs]
    b.close()
    for c in ctxs:
        c.close()
    tasks = [(n, a, L, i, tuned[i], GRAPH_RUNS * GRAPH_STEPS, LOG_STEPS)
             for n, a, L, i in _bench_batch()]
    # largest chains first: the pool's slowest tasks start at once
    tasks.sort(key=lambda t: -t[0] * (t[2] - 1))
    with _pool() as pool:
        res = pool.map(_oracle_replay_fp64, tasks, chunksize=1)
    assert len(res) == 64
    for i, (pos_o, e_o), (j_o, dE_o, acc_o, nb), fin_o in res:
        pos_g, e_g = mids[i]
        assert np.array_equal(pos_g, pos_o), i
        # the running energy is the setup energy plus the accepted dE, each
        # within 1e-10 max(1, |dE|): its error is absolute (a neutral +-1
        # system's total can be near 0), hence the floor of 1
        assert abs(e_g - e_o) <= 1e-9 * max(1.0, abs(e_o)), (i, e_g, e_o)
        assert nb == 0
        assert np.array_equal(rl["j"][i], j_o), i
        err = np.abs(rl["dE"][i] - dE_o) / np.maximum(1.0, np.abs(dE_o))
        assert np.max(err) <= 1e-10, (i, np.max(err))
        assert np.array_equal(rl["acc"][i], acc_o), i
        assert np.array_equal(finals[i], fin_o), i


def _fp32_errors(dE_g, dE_o, beta):
    both = np.isfinite(dE_g) & np.isfinite(dE_o)
    # an exact overlap is +inf on both sides
    assert np.array_equal(np.isfinite(dE_g), np.isfinite(dE_o))
    return beta * np.abs(dE_g[both] - dE_o[both])


def _check_flips(acc_g, acc_o, dE_g, dE_o, n, seed, step0, chain, beta, h):
    """A decision may differ from the oracle's only where the FP32 error of
    dE could move it across the threshold: |log u + beta dE_oracle| no larger
    than beta |dE_gpu - dE_oracle| (u re-drawn from the oracle's stream)."""
    for t in np.nonzero(acc_g != acc_o)[0]:
        _, _, u = O.proposal(n, h, seed, step0 + int(t), chain)
        gap = abs(np.log(u) + beta * dE_o[t])
        assert gap <= beta * abs(dE_g[t] - dE_o[t]) + 1e-12, (chain, t, gap)


def test_batched_fp32_eval_bench_workload_within_tolerance():
    ctxs = _batch_contexts(mcfmm.FP32_EVAL)
    b, tuned, seeds = _tuned_graphed(ctxs)
    systems = _bench_batch()
    tasks = []
    for c, (n, a, L, i) in zip(ctxs, systems):
        _, q = uniform_system(n, a, seed=1000 + i)
        tasks.append([c.positions(), q, a, L, P_BATCH, i, c.step_counter(), i, BETA, H, None])
    rl = b.run(LOG_STEPS, seeds, beta=BETA, half_width=H, log=True)
    finals = [c.positions() for c in ctxs]
    b.close()
    for c in ctxs:
        c.close()
    for t, (_, _, _, i) in zip(tasks, systems):
        t[-1] = rl["acc"][i]
    with _pool() as pool:
        res = pool.map(_oracle_follow, [tuple(t) for t in tasks], chunksize=1)
    errs, dEs = [], []
    for (n, a, L, i), (j_o, dE_o, acc_o, fin_o) in zip(systems, res):
        assert np.array_equal(rl["j"][i], j_o), i
        errs.append(_fp32_errors(rl["dE"][i], dE_o, BETA))
        dEs.append(dE_o[np.isfinite(dE_o) & np.isfinite(rl["dE"][i])])
        _check_flips(rl["acc"][i], acc_o, rl["dE"][i], dE_o, n, i, tasks[i][6], i, BETA, H)
        assert np.array_equal(finals[i], fin_o), i
    e = np.concatenate(errs)
    worst = np.argsort(e)[-5:]
    assert np.percentile(e, 95) <= FP32_P95, np.percentile(e, 95)
    assert e.max() <= FP32_MAX, (e[worst], np.concatenate(dEs)[worst])


def test_fp32_eval_chain_with_resetup_within_tolerance():
    n, L, p, h, R = 10_000, 4, 12, 0.3, 400
    a = (n / 0.1) ** (1.0 / 3.0)
    pos, q = uniform_system(n, a, seed=4)
    g = mcfmm.Context(pos, q, a, L, p, precision=mcfmm.FP32_EVAL)
    g.setup()
    steps = 2500
    rg = g.run(steps, seed=9, beta=BETA, half_width=h, resetup_every=R, log=True)
    assert rg["steps"] == steps
    assert rg["resetups"] >= 4, rg["resetups"]
    assert np.isfinite(rg["max_drift"]) and rg["max_drift"] <= R * FP32_P95, rg["max_drift"]
    fin = g.positions()
    g.close()
    with _pool() as pool:
        j_o, dE_o, acc_o, fin_o = pool.apply(
            _oracle_follow, ((pos, q, a, L, p, 9, 0, 0, BETA, h, rg["acc"]),))
    assert np.array_equal(rg["j"], j_o)
    e = _fp32_errors(rg["dE"], dE_o, BETA)
    assert np.percentile(e, 95) <= FP32_P95, np.percentile(e, 95)
    assert e.max() <= FP32_MAX, e.max()
    _check_flips(rg["acc"], acc_o, rg["dE"], dE_o, n, 9, 0, 0, BETA, h)
    assert np.array_equal(fin, fin_o)
