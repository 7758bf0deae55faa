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


def test_result_line_fits_the_stored_tail(bench):
    """The result line keeps every form and its roofline fraction within the
    last 1500 characters of the output (the bulky legs go on the line before)."""
    import json

    class A:
        steps, warmup, mh_steps = 20, 5, 50_000
    r64 = {"clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 599}}
    e2e = {"value": 61870.47288800432, "unit": "MH steps/s", "h2d_bytes_per_step": 3200000,
           "d2h_bytes_per_step": 3200008,
           "what": "mc_init from host arrays, mc_setup, mc_run, positions+energy back, mc_destroy"}
    roof = {"bound": "alu", "achieved": 0.11386945026033803, "peak": 1.25856, "unit": "TFLOP/s",
            "frac": 0.09047598069248826, "traffic": 82680000.0,
            "traffic_source": "ncu summary of one full launch (profiles/), null if taken on other sources",
            "kernel": "mc_async_kernel<double>",
            "peak_source": "derived",
            "peak_measured": 1.2012345678, "frac_of_measured": 0.0951234567,
            "flops_per_mh_step": 1325465.733925, "acceptance": 0.8496}
    cpu = bench.cpu_baseline_from({"value": 1171.5416817472792, "sample": 3000, "setup_s": 41.2})
    forms = {"fp64": 85909.0109580918, "fp32_eval": 88831.123456, "multipole_fp64": 56468.123456,
             "batched_fp64": 558506.123456, "batched_fp32_eval": 911236.123456,
             "n1e6_fp64": 73544.123456, "n1e6_fp32_eval": 84665.123456}
    fr = {"fp64": 0.0951234567, "fp32_eval": 0.0281234567, "batched_fp32_eval": 0.151234567,
          "batched_fp64": 0.321234567}
    prec = {"moves": 10_000_000, "dE_err_p95": 5.7e-06, "dE_err_max": 0.00014,
            "fp32_eval": {"mh_steps_per_s": 80123.456, "resetups": 89,
                          "drift_mean_abs_per_1e6_acc": 0.19812345},
            "fp64_floor": {"drift_mean_abs_per_1e6_acc": 0.0028123}}
    line = bench.compact_line(85909.0109580918, 582.0111236572266, A, 1, r64, e2e, roof, cpu,
                              forms, fr, prec, "uniform N=100000 rho=0.1 a=100 L=5 p=12 h=0.3")
    text = json.dumps(line)
    assert len(text) < 1450, len(text)
    back = json.loads(text)
    for k in ("fp64", "fp32_eval", "batched_fp64", "batched_fp32_eval"):
        assert k in back["forms"] and k in back["roofline_frac"]
    for k in ("metric", "value", "unit", "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"):
        assert k in back


def test_performance_model_fit_recovers_table_1():
    """The Sec. 5.4 fit, fed times generated from the paper's Table 1
    coefficients (local propose and multipole propose) over the paper's
    N = 1e3..1e6 with its level rule, returns those coefficients, and the
    asymptotic speed-up of Table 1's gammas at nu = 0.438 is the paper's
    S_inf = 2.02."""
    import bench
    table = {"loc_prop": (304.01, 9.92, 0.61, 4.12e-5), "loc_acc": (225.80, 239.99, 0.19, 4.37e-5),
             "mp_prop": (89.15, 228.40, 0.50, 1.49e-4), "mp_acc": (436.71, 8.12, 0.27, 7.11e-6)}
    sizes = [int(round(10 ** (3 + 0.25 * k))) for k in range(13)]
    for key, (tau, gamma, kappa, sigma) in table.items():
        alpha = 0.327 if key.startswith("loc") else 0.138
        f = {"tau": tau, "gamma": gamma, "kappa": kappa, "sigma": sigma}
        rows = [{"n": n, "levels": bench.model_levels(n, alpha),
                 "t": bench.performance_model(f, n, bench.model_levels(n, alpha))} for n in sizes]
        got = bench.fit_performance_model(rows, "t")
        for name in ("tau", "gamma", "kappa", "sigma"):
            assert abs(got[name] - f[name]) <= 1e-6 * max(1.0, abs(f[name])), (key, name, got[name])
        assert got["rms_residual_us"] < 1e-6
    nu = 0.438
    s_inf = (table["mp_prop"][1] + nu * table["mp_acc"][1]) / (table["loc_prop"][1] + nu * table["loc_acc"][1])
    assert abs(s_inf - 2.02) < 0.005


def test_model_levels_follow_the_paper_rule():
    import bench
    # Sec. 5.1: L = floor(log8(alpha N)); the NaCl 46^3 system with the local
    # alpha gives the paper's L = 4
    assert bench.model_levels(97_336, 0.327) == 4
    assert bench.model_levels(1000, 0.327) == 2 and bench.model_levels(10 ** 6, 0.327) == 6
