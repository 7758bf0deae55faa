"""The benchmark's algorithmic work model (no GPU): the flop and byte counts
per MH step and per setup pass, and the speed-of-light step times that turn
a measured rate into a roofline fraction, checked against hand counts and
their ordering (an FP32-eval step is never slower at the roofline than the
same step in FP64; the HBM term binds the FP32-eval form at N = 1e5)."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_model", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_step_flops_hand_count(bench):
    p, levels, nbar, nu = 12, 5, 24.4, 0.9
    C, hset, L_eff = 169, 3 * 13 * 14, 4
    F, fp, fa = bench.algorithmic_flops_per_step(p, levels, nbar, nu)
    assert fp == pytest.approx(2 * L_eff * (hset + 2 * C) + 2 * 27 * nbar * 11 + 2 * hset + 2 * C * C + 4 * C + 27 * 11)
    assert fa == 2 * 189 * L_eff * (hset + 2 * C) + 189 * L_eff * C + 4 * C
    assert F == pytest.approx(fp + nu * fa)


def test_setup_flops_hand_count(bench):
    n, p, levels = 1000, 4, 3
    C, hset, L_eff = 25, 3 * 5 * 6, 2
    nbar = n / 64
    energy = n * (L_eff * (hset + 2 * C) + 27 * nbar * 11)
    assert bench.setup_flops(n, p, levels, "p2l") == pytest.approx(n * L_eff * 189 * (hset + 2 * C) + energy)
    cells = [8, 64]
    fmm = n * (hset + 2 * C) + 64 * 2 * C * C + sum(cells) * 189 * 2 * C * C + energy
    assert bench.setup_flops(n, p, levels, "fmm") == pytest.approx(fmm)


def test_roofline_step_times(bench):
    nbar = 1e5 / 8 ** 4
    t64 = bench.roofline_step_time(12, 5, nbar, 0.9, False)
    t32 = bench.roofline_step_time(12, 5, nbar, 0.9, True)
    F, _, _ = bench.algorithmic_flops_per_step(12, 5, nbar, 0.9)
    assert t64 == pytest.approx(F / bench.FP64_PEAK_FLOPS)  # FP64: compute-bound
    assert t32 < t64
    bw, _ = bench.hbm_peak_bytes()
    assert t32 == pytest.approx(bench.bytes_per_step(12, 5, nbar, 0.9) / bw)  # FP32-eval: the HBM term
