"""Benchmark: Metropolis-Hastings steps per second of the multilevel
local-expansion electrostatics method on the uniform N=1e5 workload
(density 0.1, a=100, 5 levels, p=12, h=0.3, beta=1).

One bench step = one persistent launch (mc_run) of --mh-steps proposals on
the resident system.  `value` is the FP64 form, timed with CUDA events on the
library's stream, L2 flushed between timed steps.  The last stdout line (the
result) also carries the FP32-eval and batched forms with their roofline
fractions, the precision form's dE error and drift, the end-to-end number
through the C ABI with host buffers, the roofline of the chain kernel and the
CPU oracle baseline; the line before it ("detail") holds the bulky legs
(per-chain batch split, N = 1e6 setup-heavy case, per-operation timing
against N, the full-MC NaCl setting).  --impl reference times the CPU oracle
instead; --profile FORM brackets one launch for ncu.

Multi-GPU: independent replicas (one chain per GPU, seed = rank), no
collective on the data path; value = all ranks' proposals / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MH steps/sec at N=1e5, p=12: plain FP64 vs FP32-eval/FP64-acc and batched"
UNIT = "MH steps/s"
FP64_PEAK_FLOPS = 152 * 4 * 2.070e9  # 152 SMs x 4 FP64 flop/clk/SM (2 FMA lanes) x max clock
FP32_PEAK_FLOPS = 152 * 256 * 2.070e9  # 152 SMs x 128 FP32 lanes x 2 flop (FMA) x max clock


def fp_peaks_measured():
    """FMA-pipe peaks of this GPU in flop/s (FP64, FP32), measured by the
    library's probe (independent FMA chains on every SM, CUDA events)."""
    from paper_2006_16622_gb300 import mcfmm
    return mcfmm.probe_fma_rate(True, 0.2), mcfmm.probe_fma_rate(False, 0.2)


def csrc_sha16():
    """Hash of the sources of the timed chain kernel and its launch: its
    translation unit (mc_async.cu and every header) and the C ABI that sets
    its launch parameters.  An ncu summary taken on other sources no longer
    describes the kernel that runs."""
    import hashlib
    d = os.path.join(ROOT, "paper_2006_16622_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if f.endswith(".cuh") or f in ("mc_async.cu", "mc_capi.cu"):
            h.update(f.encode())
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def hbm_peak_bytes():
    """Measured copy bandwidth of this GPU model (MEASURED_PEAKS.json), else
    6.8 TB/s (an earlier GB300 measurement)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]) * 1e9, "measured"
    except (OSError, ValueError, KeyError):
        return 6.8e12, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mh-steps", type=int, default=50_000, help="proposals per bench step")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=3000, help="oracle proposals timed")
    ap.add_argument("--batch-steps", type=int, default=5000, help="proposals per chain per batched step")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-huge", action="store_true", help="skip the N=1e6 setup/step leg")
    ap.add_argument("--no-sweep", action="store_true", help="skip the per-operation timing vs N")
    ap.add_argument("--no-nacl", action="store_true", help="skip the full-MC NaCl leg")
    ap.add_argument("--accuracy", action="store_true",
                    help="run only the acceptance-probability study (relative error of P vs p)")
    ap.add_argument("--accuracy-configs", type=int, default=16)
    ap.add_argument("--model-fit", action="store_true",
                    help="run only the performance-model fit of Sec. 5.4 (propose and accept times vs N)")
    ap.add_argument("--accuracy-moves", type=int, default=1000)
    ap.add_argument("--huge-steps", type=int, default=1_000_000,
                    help="proposals timed per form on the N=1e6 workload")
    ap.add_argument("--c3-moves", type=int, default=10_000_000,
                    help="FP32-eval proposals of the precision-form run (re-setups included)")
    ap.add_argument("--c3-resetup", type=int, default=100_000,
                    help="accepted moves between full FP64 re-setups in the precision-form run")
    ap.add_argument("--c3-floor-moves", type=int, default=2_000_000,
                    help="FP64 proposals of the drift-floor run")
    ap.add_argument("--schedules", action="store_true",
                    help="also time the phased FP64 and plain FP32-eval schedules")
    ap.add_argument("--profile", default=None,
                    choices=["fp64", "fp64_phased", "fp32_eval", "fp32_eval_async", "batched_fp64",
                             "batched_fp32_eval", "setup_p2l", "setup_fmm"],
                    help="build the workload, warm up, and bracket one launch with "
                         "cudaProfilerStart/Stop (for ncu --profile-from-start off); no timing")
    ap.add_argument("--profile-n", type=int, default=0,
                    help="system size of --profile (0: the form's bench workload)")
    return ap.parse_args()


# ------------------------------------------------------- replicas over GPUs
def replica_seed(base: int, rank: int) -> int:
    """Seed of the independent chain on GPU `rank` (replicas: no data-path
    collective; only the timing is reduced)."""
    return base + 1000 * rank


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """Largest x over all ranks of the process group (x itself without one)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units of all ranks over the slowest rank's time."""
    return world * units_per_rank / seconds_max


# ------------------------------------------------------------- CPU oracle leg
def _oracle_worker(q_out, sample, warm):
    """Runs in a spawned process: oracle setup (untimed), then `sample`
    proposals of the same chain timed on one host core."""
    import numpy as np  # noqa: F401

    import oracle
    from paper_2006_16622_gb300.workloads import LARGE
    pos, q = LARGE.system()
    t0 = time.perf_counter()
    s = oracle.System(pos, q, LARGE.a, LARGE.levels, LARGE.p)
    s.setup()
    t_setup = time.perf_counter() - t0
    s.run(warm, seed=LARGE.seed, step0=0, beta=LARGE.beta, half_width=LARGE.half_width, log=False)
    t0 = time.perf_counter()
    r = s.run(sample, seed=LARGE.seed, step0=warm, beta=LARGE.beta, half_width=LARGE.half_width,
              log=False)
    dt = time.perf_counter() - t0
    q_out.put(dict(value=sample / dt, setup_s=t_setup, n_acc=r["n_acc"], sample=sample, secs=dt))


def start_oracle(sample, warm=100):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_oracle_worker, args=(q, sample, warm), daemon=True)
    p.start()
    return p, q


def _batch_oracle_worker(task):
    """One chain of the batched workload in a spawned process: oracle setup
    (untimed), 50 warm-up and `proposals` timed proposals on one core."""
    n, a, L, i, proposals = task
    import oracle
    from paper_2006_16622_gb300.workloads import uniform_system
    pos, q = uniform_system(n, a, seed=1000 + i)
    s = oracle.System(pos, q, a, L, 10)
    s.setup()
    s.run(50, seed=i, step0=0, chain=i, beta=1.0, half_width=0.3, log=False)
    t0 = time.perf_counter()
    s.run(proposals, seed=i, step0=50, chain=i, beta=1.0, half_width=0.3, log=False)
    return n, proposals / (time.perf_counter() - t0)


def batched_cpu_baseline(proposals=300):
    """The oracle on the batched workload (64 chains, N log-uniform in
    [1000, 50000], p = 10), one process per host core: a sample of k chains
    spread over the batch (k = cores, at most 16), each timed on its own
    core while the others run.  The 64-chain batch with equal proposals per
    chain then runs at k / sum_i(1 / rate_i) proposals/s on one core and k
    times that on k cores (independent chains, balanced over the cores)."""
    import multiprocessing as mp

    from paper_2006_16622_gb300.workloads import batched_systems
    systems = batched_systems(64, 1000, 50000, 0.1, 20.0)
    k = max(1, min(os.cpu_count() or 1, 16))
    pick = [systems[(j * len(systems)) // k] for j in range(k)]
    with mp.get_context("spawn").Pool(processes=k) as pool:
        res = pool.map(_batch_oracle_worker, [(n, a, L, i, proposals) for n, a, L, i in pick])
    single = k / sum(1.0 / r for _, r in res)
    return {"value": k * single, "unit": UNIT, "cores": k, "single_core": single, "kind": "oracle",
            "sample": (f"{k} of the 64 chains (N {min(n for n, _ in res)}..{max(n for n, _ in res)}), "
                       f"one process per core, {proposals} timed proposals each after 50 warm-up; "
                       f"setups not timed; value = k cores x the single-core rate of the batch")}


def cpu_baseline_from(res):
    return {"value": res["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{res['sample']} proposals, setup untimed"}


def reference_arm(args):
    import torch.distributed as dist  # noqa: F401
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2006_16622_gb300.workloads import LARGE
    oracle.build()
    pos, q = LARGE.system()
    t0 = time.perf_counter()
    s = oracle.System(pos, q, LARGE.a, LARGE.levels, LARGE.p)
    s.setup()
    setup_s = time.perf_counter() - t0
    per = 500
    step = 0
    for _ in range(args.warmup):
        s.run(per, seed=LARGE.seed, step0=step, beta=LARGE.beta, half_width=LARGE.half_width,
              log=False)
        step += per
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        s.run(per, seed=LARGE.seed, step0=step, beta=LARGE.beta, half_width=LARGE.half_width,
              log=False)
        times.append(time.perf_counter() - t0)
        step += per
    tot = sum(times)
    v = per * args.steps / tot
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": LARGE.name, "mh_steps_per_step": per, "form": "fp64"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{per} proposals per step of the N=1e5 chain, one host "
                                       f"thread; setup {setup_s:.0f} s not timed"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        # raw samples: $MC_CLOCKS_DIR if set, else the system's temporary folder
        import tempfile
        out_dir = os.environ.get("MC_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_rank{gpu_index}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl)
                          if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def algorithmic_flops_per_step(p, levels, nbar, nu):
    """FP64 flops of one MH step from the algorithm (not the implementation):
    a solid-harmonic set 3(p+1)(p+2) flops; an expansion evaluation adds a
    2C dot product; a near-field pair 11 flops; the far lattice term two
    harmonic sets and the dense operator (2C^2); an accept 2*189 P2L sets and
    one C-length update per interaction-list cell and level."""
    C = (p + 1) ** 2
    hset = 3 * (p + 1) * (p + 2)
    L_eff = levels - 1
    f_prop = 2 * L_eff * (hset + 2 * C) + 2 * 27 * nbar * 11 + 2 * hset + 2 * C * C + 4 * C + 27 * 11
    f_acc = 2 * 189 * L_eff * (hset + 2 * C) + 189 * L_eff * C + 4 * C
    return f_prop + nu * f_acc, f_prop, f_acc


def setup_flops(n, p, levels, mode):
    """FP64 flops of one setup pass from the algorithm (periodic box, levels
    2..L).  Alg. L.3 ("p2l"): per charge, level and interaction-list cell one
    irregular harmonic set and a C-length multiply-add.  Fast mode ("fmm"):
    charge-to-multipole at the finest level, multipole-to-multipole up the
    tree and multipole-to-local over every cell's 189 interaction-list cells,
    each translation counted as a dense C x C operator (2 C^2).  Both add the
    initial energy: per charge the L - 1 expansion evaluations and the
    27-cell direct sum (11 flops a pair)."""
    C = (p + 1) ** 2
    hset = 3 * (p + 1) * (p + 2)
    L_eff = levels - 1
    nbar = n / (8 ** (levels - 1))
    energy = n * (L_eff * (hset + 2 * C) + 27 * nbar * 11)
    if mode == "p2l":
        return n * L_eff * 189 * (hset + 2 * C) + energy
    cells = [8 ** (l - 1) for l in range(2, levels + 1)]
    m2l = sum(cells) * 189 * 2 * C * C
    m2m = sum(cells[1:]) * 2 * C * C
    return n * (hset + 2 * C) + m2m + m2l + energy


def roofline_step_time(p, levels, nbar, nu, fp32_eval):
    """Speed-of-light time of one MH step: the slowest of the evaluation
    flops at their unit's peak, the FP64 flops at the FP64 peak and the bytes
    at HBM bandwidth.  In the FP32-eval form the FP64 part is what stays
    FP64: the far-lattice change (two harmonic sets about the box centre and
    the dense operator), the image correction, the decision and, per accept,
    the accumulator adds and the K/H update; everything else runs in FP32."""
    C = (p + 1) ** 2
    hset = 3 * (p + 1) * (p + 2)
    F, _, _ = algorithmic_flops_per_step(p, levels, nbar, nu)
    bw, _ = hbm_peak_bytes()
    t_mem = bytes_per_step(p, levels, nbar, nu) / bw
    if not fp32_eval:
        return max(F / FP64_PEAK_FLOPS, t_mem)
    f64 = 2 * hset + 2 * C * C + 4 * C + 27 * 11 + nu * (189 * (levels - 1) * C + 4 * C)
    return max((F - f64) / FP32_PEAK_FLOPS, f64 / FP64_PEAK_FLOPS, t_mem)


def bytes_per_step(p, levels, nbar, nu):
    C = (p + 1) ** 2
    L_eff = levels - 1
    b_prop = 2 * L_eff * C * 8 + 2 * 27 * nbar * 36 + C * C * 8 + 2 * C * 8
    b_acc = 2 * 189 * L_eff * C * 8 + 4 * C * 8
    return b_prop + nu * b_acc


def read_profile_traffic(name="async_fp64_dram_full_launch_N1e5.md"):
    """DRAM bytes per launch of the timed chain kernel (50 000 proposals)
    from the committed ncu summary of one full launch, when that summary was
    taken on the current CUDA sources (its `csrc_sha16:` line), else None."""
    path = os.path.join(ROOT, "profiles", name)
    traffic, sha = None, None
    try:
        for line in open(path):
            if line.startswith("dram_bytes_per_launch:"):
                traffic = float(line.split(":")[1].split()[0])
            elif line.startswith("csrc_sha16:"):
                sha = line.split(":")[1].strip()
    except (OSError, ValueError, IndexError):
        return None
    return traffic if sha == csrc_sha16() else None


def batched_form(args, precision, stream, flush):
    """64 independent chains, N log-uniform in [1000, 50000] at density 0.1,
    ~20 charges per finest cell, p=10, h=0.3, beta=1, seed i for chain i; one
    autotuned persistent launch per step, replayed from a CUDA graph."""
    import numpy as np
    import torch

    from paper_2006_16622_gb300 import mcfmm
    from paper_2006_16622_gb300.workloads import batched_systems, uniform_system

    systems = batched_systems(64, 1000, 50000, 0.1, 20.0)
    ctxs = []
    t0 = time.perf_counter()
    for n, a, L, i in systems:
        pos, q = uniform_system(n, a, seed=1000 + i)
        c = mcfmm.Context(pos, q, a, L, 10, precision=precision, stream=stream.cuda_stream)
        c.setup()
        ctxs.append(c)
    setup_s = time.perf_counter() - t0
    b = mcfmm.Batch(ctxs)
    t0 = time.perf_counter()
    b.tune(trial_steps=300, beta=1.0, half_width=0.3)
    tune_s = time.perf_counter() - t0
    ctas, nf = b.info()
    seeds = np.arange(len(ctxs), dtype=np.uint64)
    Sb = args.batch_steps
    for _ in range(args.warmup):
        b.run(Sb, seeds, beta=1.0, half_width=0.3, stats=False)
    torch.cuda.synchronize()
    durs = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run(Sb, seeds, beta=1.0, half_width=0.3, stats=False)
        e1.record(stream)
        e1.synchronize()
        durs.append(e0.elapsed_time(e1) / 1000.0)
    st = b.run(200, seeds, beta=1.0, half_width=0.3)["stats"]
    acc = sum(x["accepted"] for x in st) / max(1, sum(x["steps"] for x in st))
    b.close()
    for c in ctxs:
        if c.status() != 0:
            raise RuntimeError("batched chain failed")
        c.close()
    return dict(value=len(ctxs) * Sb * args.steps / sum(durs), setup_s=setup_s, tune_s=tune_s,
                ctas=[int(x) for x in ctas], nf_cols=nf, acceptance=acc,
                sizes=[n for n, _, _, _ in systems], levels=[L for _, _, L, _ in systems])


def huge_workload_leg(args, stream, flush):
    """N = 1e6 (density 0.1, 6 levels, p = 12): both setup modes timed with
    CUDA events (each after one untimed call), the truncation-level gap of the
    fast setup, then FP64 and FP32-eval chains of --huge-steps proposals."""
    import torch

    from paper_2006_16622_gb300 import mcfmm
    from paper_2006_16622_gb300.workloads import HUGE as W

    pos, q = W.system()
    out = {"workload": W.name}

    def timed(fn):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1000.0

    ctx = mcfmm.Context(pos, q, W.a, W.levels, W.p, stream=stream.cuda_stream)
    energies = {}
    for mode, name in ((mcfmm.SETUP_FMM, "fmm"), (mcfmm.SETUP_P2L, "p2l")):
        ctx.setup(mode)
        out[f"setup_{name}_s"] = timed(lambda: ctx.setup(mode))
        energies[name] = ctx.energy()
    out["fmm_energy_rel_gap"] = abs(energies["fmm"] - energies["p2l"]) / abs(energies["p2l"])
    out["setup_roofline"] = {}
    for name in ("p2l", "fmm"):
        f = setup_flops(len(q), W.p, W.levels, name)
        ach = f / out[f"setup_{name}_s"]
        out["setup_roofline"][name] = {"bound": "alu", "flops": f, "achieved": ach / 1e12,
                                       "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                                       "frac": ach / FP64_PEAK_FLOPS}
    ctx.close()
    for prec, name in ((mcfmm.FP64, "fp64"), (mcfmm.FP32_EVAL, "fp32_eval")):
        ctx = mcfmm.Context(pos, q, W.a, W.levels, W.p, precision=prec, stream=stream.cuda_stream)
        ctx.setup(mcfmm.SETUP_FMM)
        ctx.run(5000, seed=W.seed, beta=W.beta, half_width=W.half_width, stats=False)
        dt = timed(lambda: ctx.run(args.huge_steps, seed=W.seed + 1, beta=W.beta,
                                   half_width=W.half_width, stats=False))
        status = ctx.status()
        ctx.close()
        if status != 0:
            raise RuntimeError(f"chain status {status}")
        out[f"{name}_mh_steps_per_s"] = args.huge_steps / dt
    out["mh_steps_timed"] = args.huge_steps
    return out


def size_sweep_leg(stream):
    """Per-operation times against N (density 0.1, ~20 charges per finest
    cell, p = 12, h = 0.3): MH steps/s over 20 000 proposals of the local
    method (FP64 and FP32-eval) and of the multipole method (FP64), and from
    the device timers of CTA 0 the propose phase (proposal draw to the
    decision's barrier) and the accept phase per accepted move."""
    import numpy as np
    import torch

    from paper_2006_16622_gb300 import mcfmm
    from paper_2006_16622_gb300.workloads import size_sweep

    rows = []
    for W in size_sweep():
        pos, q = W.system()
        row = {"n": W.n, "levels": W.levels, "p": W.p}
        for prec, name, mode in ((mcfmm.FP64, "fp64", None), (mcfmm.FP32_EVAL, "fp32_eval", None),
                                 (mcfmm.FP64, "multipole_fp64", mcfmm.SETUP_MULTIPOLE)):
            ctx = mcfmm.Context(pos, q, W.a, W.levels, W.p, precision=prec, stream=stream.cuda_stream)
            if mode is None:
                mode = mcfmm.SETUP_FMM if W.n >= 1_000_000 else mcfmm.SETUP_P2L
            ctx.setup(mode)
            ctx.run(2000, seed=1, beta=W.beta, half_width=W.half_width, stats=False)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.run(20_000, seed=2, beta=W.beta, half_width=W.half_width, stats=False)
            e1.record(stream)
            e1.synchronize()
            row[f"{name}_mh_steps_per_s"] = 20_000 / (e0.elapsed_time(e1) / 1000.0)
            ctx.profile(True)
            ctx.profile_read()
            ctx.run(5000, seed=3, beta=W.beta, half_width=W.half_width, stats=False)
            pr = ctx.profile_read().astype(np.float64)
            ctx.profile(False)
            steps, acc = max(pr[5], 1.0), max(pr[6], 1.0)
            if name == "fp64":
                # barrier-free schedule: from the publication of a step's
                # geometry (ahead of the previous decision) to its decision
                row[f"{name}_publish_to_decision_us"] = pr[0] / steps / 1e3
            else:
                row[f"{name}_propose_us"] = (pr[0] + pr[1]) / steps / 1e3
                row[f"{name}_accept_us"] = (pr[3] + pr[4]) / acc / 1e3
            row[f"{name}_acceptance"] = pr[6] / steps
            ctx.close()
        # time per MH step of the multipole method over the local method
        row["multipole_over_local_time"] = row["fp64_mh_steps_per_s"] / row["multipole_fp64_mh_steps_per_s"]
        rows.append(row)
    return rows


def nacl_full_mc_leg(stream):
    """The paper's full Monte Carlo setting (Sec. 5.3): 46^3 NaCl ions in a
    153.2 A box, 12 expansion terms (p = 11), L = 4, T = 273 K, moves of
    +-0.25 A, with the short-range Lennard-Jones term (12 A cutoff); MH
    steps/s of both methods (FP64) over 20 000 proposals."""
    import torch

    from paper_2006_16622_gb300 import mcfmm
    from paper_2006_16622_gb300.workloads import (NACL_BETA, NACL_FULL_MC, NACL_LJ_CUTOFF,
                                                  NACL_LJ_EPS, NACL_LJ_SIGMA, nacl_full_mc_system)

    cfg = NACL_FULL_MC
    pos, q, a = nacl_full_mc_system(cfg["m"], cfg["box"])
    out = {"workload": f"NaCl {cfg['m']}^3 ions, box {cfg['box']} A, L = {cfg['levels']}, "
                       f"p = {cfg['p']}, T = 273 K, h = {cfg['half_width']} A, LJ cutoff 12 A"}
    for name, mode in (("local_fp64", mcfmm.SETUP_P2L), ("multipole_fp64", mcfmm.SETUP_MULTIPOLE)):
        ctx = mcfmm.Context(pos, q, a, cfg["levels"], cfg["p"], stream=stream.cuda_stream)
        ctx.set_lj(NACL_LJ_EPS, NACL_LJ_SIGMA, NACL_LJ_CUTOFF)
        ctx.setup(mode)
        ctx.run(2000, seed=1, beta=NACL_BETA, half_width=cfg["half_width"], stats=False)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.run(20_000, seed=2, beta=NACL_BETA, half_width=cfg["half_width"], stats=False)
        e1.record(stream)
        e1.synchronize()
        out[f"{name}_mh_steps_per_s"] = 20_000 / (e0.elapsed_time(e1) / 1000.0)
        st = ctx.run(5000, seed=3, beta=NACL_BETA, half_width=cfg["half_width"])
        out[f"{name}_acceptance"] = st["accepted"] / max(1, st["steps"])
        if ctx.status() != 0:
            raise RuntimeError("NaCl chain failed")
        ctx.close()
    return out


def _dE_error_vs_fp64(pos, q, W, stream, seed, steps=4000):
    """FP32-eval against the (oracle-parity-tested) FP64 chain from the same
    state and seed: |dE_fp32 - dE_fp64| over the common prefix (until the
    first differing decision) of `steps` logged proposals."""
    import numpy as np

    from paper_2006_16622_gb300 import mcfmm
    logs = {}
    for prec in (mcfmm.FP64, mcfmm.FP32_EVAL):
        c = mcfmm.Context(pos, q, W.a, W.levels, W.p, precision=prec, stream=stream.cuda_stream)
        c.setup()
        logs[prec] = c.run(steps, seed=seed, beta=W.beta, half_width=W.half_width, log=True)
        c.close()
    a64, a32 = logs[mcfmm.FP64], logs[mcfmm.FP32_EVAL]
    diff = np.nonzero(a64["acc"] != a32["acc"])[0]
    k = int(diff[0]) if len(diff) else steps
    e = W.beta * np.abs(a32["dE"][:k] - a64["dE"][:k])
    return e[np.isfinite(e)]


def precision_form_leg(args, W, stream):
    """The precision form as configured: --c3-moves FP32-eval proposals on
    the N = 1e5 workload with a full FP64 re-setup every --c3-resetup
    accepted moves (one mc_run call; wall time includes the re-setups), the
    running-minus-fresh energy drift at every re-setup per 1e6 accepts, next
    to the FP64 form's drift floor (P2L truncation asymmetry) over
    --c3-floor-moves; the dE error against the FP64 chain at the start and
    from the FP32-eval chain's final state (4000 proposals each)."""
    import numpy as np

    from paper_2006_16622_gb300 import mcfmm
    pos, q = W.system()
    R = args.c3_resetup
    out = {"moves": args.c3_moves, "resetup_every_accepts": R}
    final_pos = None
    for name, prec, moves in (("fp32_eval", mcfmm.FP32_EVAL, args.c3_moves),
                              ("fp64_floor", mcfmm.FP64, args.c3_floor_moves)):
        c = mcfmm.Context(pos, q, W.a, W.levels, W.p, precision=prec, stream=stream.cuda_stream)
        c.setup()
        stream.synchronize()
        t0 = time.perf_counter()
        st = c.run(moves, seed=78, beta=W.beta, half_width=W.half_width, resetup_every=R)
        dt = time.perf_counter() - t0
        if name == "fp32_eval":
            final_pos = c.positions()
        status = c.status()
        c.close()
        if status != 0 or st["steps"] != moves:
            raise RuntimeError(f"precision-form chain status {status}")
        k = max(1, st["resetups"])
        out[name] = {"mh_steps_per_s": moves / dt, "accepted": st["accepted"],
                     "resetups": st["resetups"],
                     "drift_max_per_1e6_acc": st["max_drift"] * 1e6 / R,
                     "drift_mean_abs_per_1e6_acc": st["sum_abs_drift"] / k * 1e6 / R,
                     "drift_mean_signed_per_1e6_acc": st["sum_drift"] / k * 1e6 / R}
    e = np.concatenate([_dE_error_vs_fp64(pos, q, W, stream, seed=77),
                        _dE_error_vs_fp64(final_pos, q, W, stream, seed=79)])
    out.update(dE_err_p95=float(np.percentile(e, 95)), dE_err_max=float(e.max()),
               dE_err_samples=int(len(e)))
    return out


def profile_launch(args):
    """One launch of the chosen form bracketed by cudaProfilerStart/Stop, so
    that `ncu --profile-from-start off -k regex:<kernel> -c 1` captures it
    after the untimed warm-up launches.  Chains: --mh-steps proposals on the
    N = 1e5 workload (or --profile-n charges at density 0.1); batches: the
    64-chain batched workload, tuned, --batch-steps proposals per chain;
    setups: one setup pass of --profile-n charges (default 1e5) at density
    0.1, ~20-30 charges per finest cell, p = 12."""
    import numpy as np
    import torch

    from paper_2006_16622_gb300 import mcfmm
    from paper_2006_16622_gb300.workloads import LARGE, batched_systems, size_sweep, uniform_system

    mcfmm.load()
    form = args.profile
    ok = True
    if form.startswith("batched"):
        prec = mcfmm.FP64 if form == "batched_fp64" else mcfmm.FP32_EVAL
        ctxs = []
        for n, a, L, i in batched_systems(64, 1000, 50000, 0.1, 20.0):
            pos, q = uniform_system(n, a, seed=1000 + i)
            c = mcfmm.Context(pos, q, a, L, 10, precision=prec)
            c.setup()
            ctxs.append(c)
        b = mcfmm.Batch(ctxs)
        b.tune(trial_steps=300, beta=1.0, half_width=0.3)
        seeds = np.arange(len(ctxs), dtype=np.uint64)
        for _ in range(3):
            b.run(args.batch_steps, seeds, beta=1.0, half_width=0.3, stats=False)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        b.run(args.batch_steps, seeds, beta=1.0, half_width=0.3, stats=False)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        ok = all(c.status() == 0 for c in ctxs)
        b.close()
        for c in ctxs:
            c.close()
    else:
        W = LARGE if args.profile_n == 0 else size_sweep((args.profile_n,))[0]
        if form.startswith("setup") and args.profile_n == 0:
            W = LARGE
        pos, q = W.system()
        prec = mcfmm.FP32_EVAL if form.startswith("fp32") else mcfmm.FP64
        c = mcfmm.Context(pos, q, W.a, W.levels, W.p, precision=prec)
        if form.startswith("setup"):
            mode = mcfmm.SETUP_P2L if form == "setup_p2l" else mcfmm.SETUP_FMM
            c.setup(mode)
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
            c.setup(mode)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        else:
            c.setup()
            if form == "fp64_phased":
                c.set_schedule(mcfmm.SCHEDULE_PHASED)
            elif form == "fp32_eval_async":
                c.set_schedule(mcfmm.SCHEDULE_ASYNC)
            for _ in range(3):
                c.run(args.mh_steps, seed=W.seed, beta=W.beta, half_width=W.half_width, stats=False)
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
            c.run(args.mh_steps, seed=W.seed, beta=W.beta, half_width=W.half_width, stats=False)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        ok = c.status() == 0
        c.close()
    print(json.dumps({"profile": form, "ok": ok, "mh_steps": args.mh_steps,
                      "batch_steps": args.batch_steps, "n": args.profile_n}), flush=True)
    if not ok:
        sys.exit(1)


def compact_line(value, ms_per_step, args, world, r64, e2e, roof, cpu, forms, fr, prec_stats,
                 workload):
    """The result line: the contract's keys, the three forms with their
    roofline fractions and the precision form's summary; the bulky legs go
    on the line before it."""
    def rnd(x, k=4):
        if isinstance(x, float):
            return float(f"{x:.{k}g}")
        if isinstance(x, dict):
            return {kk: rnd(v, k) for kk, v in x.items()}
        return x
    line = {"metric": METRIC, "value": rnd(value, 7), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rnd(ms_per_step, 6),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload, "l2": "flushed", "parallelism": f"replicas x{world}"},
            "roofline": {k: rnd(v) for k, v in roof.items()
                         if k not in ("traffic_source", "flops_per_mh_step", "acceptance")},
            "cpu_baseline": rnd(cpu) if cpu else None,
            "e2e": {k: rnd(v) for k, v in e2e.items() if k != "what"} if e2e else None,
            "gpu_launches": args.steps,
            "clocks": ({k: rnd(v) for k, v in r64["clocks"].items() if k != "samples"}
                       if r64["clocks"] else None),
            "forms": rnd(forms), "roofline_frac": rnd(fr, 3)}
    if prec_stats:
        line["precision_form"] = {
            "moves": prec_stats["moves"], "resetups": prec_stats["fp32_eval"]["resetups"],
            "rate": rnd(prec_stats["fp32_eval"]["mh_steps_per_s"]),
            "drift_1e6acc": rnd(prec_stats["fp32_eval"]["drift_mean_abs_per_1e6_acc"], 3),
            "floor_1e6acc": rnd(prec_stats["fp64_floor"]["drift_mean_abs_per_1e6_acc"], 3),
            "dE_p95": rnd(prec_stats["dE_err_p95"], 2), "dE_max": rnd(prec_stats["dE_err_max"], 2)}
    return line


def gpu_arm(args):
    import numpy as np
    import torch

    from paper_2006_16622_gb300 import mcfmm
    from paper_2006_16622_gb300.workloads import LARGE

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    oracle_proc = None
    if rank == 0 and world == 1 and not args.no_cpu:
        oracle_proc = start_oracle(args.cpu_sample)

    mcfmm.load()
    stream = torch.cuda.current_stream()
    W = LARGE
    pos, q = W.system()
    S = args.mh_steps
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    fp64_meas, fp32_meas = fp_peaks_measured()

    def time_form(precision, schedule=None):
        # schedule None: the context's default (barrier-free for FP64,
        # phased for FP32-eval)
        ctx = mcfmm.Context(pos, q, W.a, W.levels, W.p, precision=precision,
                            stream=stream.cuda_stream)
        if schedule is not None:
            ctx.set_schedule(schedule)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.setup()
        setup_s = time.perf_counter() - t0
        seed = replica_seed(W.seed, rank)
        for _ in range(args.warmup):
            ctx.run(S, seed=seed, beta=W.beta, half_width=W.half_width, stats=False)
        torch.cuda.synchronize()
        durs = []
        sampler = ClockSampler(local)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        sampler.start()
        for _ in range(args.steps):
            flush.zero_()  # write 256 MiB (> 129 MB L2) between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.run(S, seed=seed, beta=W.beta, half_width=W.half_width, stats=False)
            e1.record(stream)
            e1.synchronize()
            durs.append(e0.elapsed_time(e1) / 1000.0)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        if dist is not None:
            dist.barrier()
        # acceptance rate over a stats-reporting run of the same chain
        st = ctx.run(min(S, 20_000), seed=seed, beta=W.beta, half_width=W.half_width)
        nu = st["accepted"] / max(1, st["steps"])
        status = ctx.status()
        ctx.close()
        if status != 0:
            raise RuntimeError(f"chain status {status}")
        tot = max_over_ranks(sum(durs), dist, "cuda")
        return dict(total=tot, durs=durs, setup_s=setup_s, nu=nu, clocks=clocks)

    r64 = time_form(mcfmm.FP64)
    r32 = r64p = r32p = None
    if not args.no_fp32:
        r32 = time_form(mcfmm.FP32_EVAL)
        if args.schedules:
            r64p = time_form(mcfmm.FP64, mcfmm.SCHEDULE_PHASED)
            r32p = time_form(mcfmm.FP32_EVAL, mcfmm.SCHEDULE_PLAIN)

    rb32 = rb64 = None
    if not args.no_batch:
        rb32 = batched_form(args, mcfmm.FP32_EVAL, stream, flush)
        rb64 = batched_form(args, mcfmm.FP64, stream, flush)
    prec_stats = None if (args.no_precision or rank != 0) else precision_form_leg(args, W, stream)
    huge = None if (args.no_huge or rank != 0) else huge_workload_leg(args, stream, flush)
    sweep = None if (args.no_sweep or rank != 0) else size_sweep_leg(stream)
    nacl = None if (args.no_nacl or rank != 0) else nacl_full_mc_leg(stream)

    # end to end through the C ABI: host arrays in, positions and energy out
    e2e = None
    e2e_fast = None
    if not args.no_e2e:
        torch.cuda.synchronize()

        def e2e_jobs(mode):
            t_e2e = []
            for i in range(2):
                t0 = time.perf_counter()
                ctx = mcfmm.Context(pos, q, W.a, W.levels, W.p, precision=mcfmm.FP64,
                                    stream=stream.cuda_stream)
                ctx.setup(mode)
                ctx.run(S, seed=replica_seed(W.seed + 7, rank), beta=W.beta,
                        half_width=W.half_width, stats=False)
                out_pos = ctx.positions()
                e = ctx.energy()
                ctx.close()
                t_e2e.append(time.perf_counter() - t0)
                assert np.isfinite(e) and out_pos.shape == pos.shape
            return max_over_ranks(max(t_e2e[1:]) if len(t_e2e) > 1 else t_e2e[0], dist, "cuda")

        te = e2e_jobs(mcfmm.SETUP_P2L)
        # the same jobs with the fast (FMM-variant) setup: expansions equal to
        # Alg. L.3's up to the multipole truncation (detail line only)
        e2e_fast = whole_job_rate(S, world, e2e_jobs(mcfmm.SETUP_FMM))
        e2e = {"value": whole_job_rate(S, world, te), "unit": UNIT,
               "h2d_bytes_per_step": int(pos.nbytes + q.nbytes),
               "d2h_bytes_per_step": int(len(q) * 32 + 8),
               "what": "mc_init from host arrays, mc_setup, mc_run, positions+energy back, mc_destroy"}

    if rank != 0:
        return
    value = whole_job_rate(S * args.steps, world, r64["total"])
    nbar = W.n / (8 ** (W.levels - 1))
    F, Fp, Fa = algorithmic_flops_per_step(W.p, W.levels, nbar, r64["nu"])
    per_launch = statistics.mean(r64["durs"])
    achieved = F * S / per_launch
    traffic_launch = read_profile_traffic() if S == 50_000 else None
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": FP64_PEAK_FLOPS / 1e12,
            "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_FLOPS, "traffic": traffic_launch,
            "traffic_source": "ncu summary of one full launch (profiles/), null if taken on other sources",
            "kernel": "mc_async_kernel<double>",
            "peak_source": "derived", "peak_measured": fp64_meas / 1e12, "frac_of_measured": achieved / fp64_meas,
            "flops_per_mh_step": F, "acceptance": r64["nu"]}
    cpu = None
    if oracle_proc is not None:
        proc, qq = oracle_proc
        try:
            res = qq.get(timeout=900)
            cpu = cpu_baseline_from(res)
        except Exception as ex:  # noqa: BLE001
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"oracle leg failed: {ex!r}"}
        proc.join(timeout=10)
    cpu_batched = None
    if world == 1 and not args.no_cpu and not args.no_batch:
        try:
            cpu_batched = batched_cpu_baseline()
        except Exception as ex:  # noqa: BLE001
            cpu_batched = {"value": None, "unit": UNIT, "kind": "oracle",
                           "sample": f"batched oracle leg failed: {ex!r}"}
    forms = {"fp64": value}
    detail = {"mh_steps_per_step": S, "fp64_setup_s": r64["setup_s"],
              "e2e_fast_setup": e2e_fast,
              "roofline_flops_per_mh_step": F, "fp64_acceptance": r64["nu"],
              "peaks_measured_tflops": {"fp64": fp64_meas / 1e12, "fp32": fp32_meas / 1e12}}
    if r32:
        forms["fp32_eval"] = whole_job_rate(S * args.steps, world, r32["total"])
        detail["fp32_eval_acceptance"] = r32["nu"]
        detail["fp32_eval_setup_s"] = r32["setup_s"]
    if r64p:
        detail["fp64_phased_schedule"] = whole_job_rate(S * args.steps, world, r64p["total"])
        detail["fp32_eval_plain_schedule"] = whole_job_rate(S * args.steps, world, r32p["total"])
    if sweep:
        row = [r for r in sweep if r["n"] == W.n]
        if row:
            forms["multipole_fp64"] = world * row[0]["multipole_fp64_mh_steps_per_s"]
    if rb32:
        forms["batched_fp64"] = world * rb64["value"]
        forms["batched_fp32_eval"] = world * rb32["value"]
        detail["batched_config"] = {
            "workload": "64 chains, N log-uniform [1000, 50000], rho=0.1, ~20 per finest cell, "
                        "p=10, h=0.3, beta=1, seed i for chain i",
            "proposals_per_chain_per_step": args.batch_steps, "ctas_per_chain": rb32["ctas"],
            "nf_cols": rb32["nf_cols"], "ctas_per_chain_fp64": rb64["ctas"],
            "nf_cols_fp64": rb64["nf_cols"], "setup_s": rb32["setup_s"], "tune_s": rb32["tune_s"],
            "acceptance": rb32["acceptance"],
            "fp64_arithmetic": "FP64, except the speculative contributions' irregular recurrence in "
                               "pair-of-floats arithmetic (~46 bits) on the FP32 pipe; FP64 accumulators"}
    # every form as a fraction of its roofline (rate x speed-of-light step time)
    bw, bw_src = hbm_peak_bytes()
    fr = {"fp64": value * roofline_step_time(W.p, W.levels, nbar, r64["nu"], False)}
    if r32:
        fr["fp32_eval"] = forms["fp32_eval"] * roofline_step_time(W.p, W.levels, nbar, r32["nu"], True)
    if rb32:
        for key, rb, f32 in (("batched_fp32_eval", rb32, True), ("batched_fp64", rb64, False)):
            ts = [roofline_step_time(10, L, n / 8 ** (L - 1), rb["acceptance"], f32)
                  for n, L in zip(rb["sizes"], rb["levels"])]
            fr[key] = forms[key] * statistics.mean(ts)
    detail["roofline_peaks"] = (f"FP64 {FP64_PEAK_FLOPS / 1e12:.2f} and FP32 {FP32_PEAK_FLOPS / 1e12:.1f} "
                                f"TFLOP/s derived (unit counts x 2070 MHz), HBM {bw / 1e9:.0f} GB/s {bw_src}")
    detail.update(cpu_baseline_batched=cpu_batched, precision_form=prec_stats, huge=huge,
                  size_sweep=sweep, nacl_full_mc=nacl,
                  paper_context={"value": 1000.0, "unit": UNIT,
                                 "hardware": "1 core of an Intel Xeon E5-2650v2",
                                 "workload": "NaCl-like, N ~ 1e5, 12 expansion terms (p = 11), L = 4, "
                                             "periodic, with Lennard-Jones",
                                 "note": "the paper's cost of about 1 ms per MH step (Sec. 2; setting "
                                         "of Sec. 5.3): context only, another machine and workload"})
    if huge:
        forms["n1e6_fp64"] = huge["fp64_mh_steps_per_s"]
        forms["n1e6_fp32_eval"] = huge["fp32_eval_mh_steps_per_s"]
    print(json.dumps({"detail": detail}), flush=True)
    line = compact_line(value, 1000 * r64["total"] / args.steps, args, world, r64, e2e, roof, cpu,
                        forms, fr, prec_stats, W.name)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def accuracy_study(args):
    """Relative error of the acceptance probability, dP = |P - P*| / P*,
    P = exp(-beta dE), against the number of expansion terms (Sec. 5.1):
    perturbed 22^3 NaCl crystals at 273 K, `--accuracy-configs` crystals x
    `--accuracy-moves` proposals (none accepted); P* from the local method at
    p = 15, the largest order of this build (tests/test_gpu_accuracy.py
    checks that reference against the p = 25 evaluation the paper uses).
    Local method in FP64 and FP32-eval, multipole method in FP64, p = 3..14."""
    import numpy as np

    from paper_2006_16622_gb300 import mcfmm
    from paper_2006_16622_gb300.workloads import NACL_BETA, perturbed_nacl, study_moves

    mcfmm.load()
    m, L = 22, 4
    forms = [("local_fp64", mcfmm.FP64, mcfmm.SETUP_P2L),
             ("local_fp32_eval", mcfmm.FP32_EVAL, mcfmm.SETUP_P2L),
             ("multipole_fp64", mcfmm.FP64, mcfmm.SETUP_MULTIPOLE)]
    ps = list(range(3, 15))
    errs = {name: {p: [] for p in ps} for name, _, _ in forms}
    t0 = time.perf_counter()
    for cfg in range(args.accuracy_configs):
        pos, q, a = perturbed_nacl(m, seed=cfg)
        js, rn = study_moves(len(q), a, pos, args.accuracy_moves, seed=cfg)

        def dEs(p, prec, mode):
            ctx = mcfmm.Context(pos, q, a, L, p, precision=prec)
            ctx.setup(mode)
            out = np.array([ctx.propose(int(j), r) for j, r in zip(js, rn)])
            ctx.close()
            return out

        ref = np.exp(-NACL_BETA * dEs(15, mcfmm.FP64, mcfmm.SETUP_P2L))
        for name, prec, mode in forms:
            for p in ps:
                P = np.exp(-NACL_BETA * dEs(p, prec, mode))
                errs[name][p].append(np.abs(P - ref) / np.abs(ref))
    out = {"metric": "mean relative error of the acceptance probability vs expansion order",
           "workload": f"perturbed {m}^3 NaCl, spacing 3.3 A, T = 273 K, h = 0.25 A, L = {L}",
           "samples": args.accuracy_configs * args.accuracy_moves, "reference": "local FP64, p = 15",
           "mean_delta_p": {}, "p11": {}, "seconds": None}
    for name, _, _ in forms:
        out["mean_delta_p"][name] = {p: float(np.mean(np.concatenate(errs[name][p]))) for p in ps}
        e = np.concatenate(errs[name][11])
        out["p11"][name] = {"median": float(np.median(e)), "p90": float(np.percentile(e, 90)),
                            "p99": float(np.percentile(e, 99)), "max": float(e.max()),
                            "fraction_below_1e-3": float(np.mean(e <= 1e-3))}
    out["seconds"] = time.perf_counter() - t0
    print(json.dumps(out), flush=True)


def model_levels(n, alpha):
    """L = floor(log8(alpha N)), at least 2 (Sec. 5.1's rule for the levels)."""
    import math
    return max(2, int(math.floor(math.log(alpha * n) / math.log(8.0) + 1e-12)))


def performance_model(f, n, L):
    """T = tau + gamma L + kappa N / N_cell + sigma N, N_cell = 8^(L-1) (Sec. 5.4)."""
    return f["tau"] + f["gamma"] * L + f["kappa"] * n / 8.0 ** (L - 1) + f["sigma"] * n


def fit_performance_model(rows, key):
    """Non-negative least-squares fit of the Sec. 5.4 model to rows of
    {"n", "levels", key} (every term of the model is a cost; the columns are
    scaled to unit norm for the solve).  Returns tau, gamma, kappa, sigma and
    the rms residual."""
    import numpy as np
    X = np.array([[1.0, r["levels"], r["n"] / 8.0 ** (r["levels"] - 1), r["n"]] for r in rows])
    y = np.array([r[key] for r in rows], dtype=np.float64)
    scale = np.linalg.norm(X, axis=0)
    try:
        from scipy.optimize import nnls
        cs, _ = nnls(X / scale, y)
    except ImportError:  # pragma: no cover - scipy is part of the image
        cs = np.clip(np.linalg.lstsq(X / scale, y, rcond=None)[0], 0.0, None)
    coef = cs / scale
    resid = y - X @ coef
    return {"tau": float(coef[0]), "gamma": float(coef[1]), "kappa": float(coef[2]), "sigma": float(coef[3]),
            "rms_residual_us": float(np.sqrt(np.mean(resid ** 2)))}


def model_fit_study():
    """The performance model of Sec. 5.4, T(N) = tau + gamma L + kappa N/N_cell
    + sigma N with N_cell = 8^(L-1), fitted by least squares to the time per
    propose and per accept operation of both methods (FP64), measured in the
    setting of Sec. 5.2: uniform random +-1 charges at the density of the
    NaCl spacing (3.3 A), moves of +-0.25 A per axis, 12 expansion terms
    (p = 11), N = 1e3..1e6, levels from L = floor(log8(alpha N)) with
    alpha = 0.327 (local) and 0.138 (multipole), the optimal values of
    Sec. 5.1.  The local method runs its plain schedule, whose accept phase
    is Alg. L.2 after the decision (the speculative schedule moves that work
    into the propose phase); the multipole method runs Alg. M.1 / M.2.
    Times are the device timers of CTA 0 (propose: the proposal draw to the
    decision; accept: the accept phase and its barrier, per accepted move).
    Also the speed-up S(N) and its limit S_inf at nu = 0.438."""
    import numpy as np
    import torch

    from paper_2006_16622_gb300 import mcfmm
    from paper_2006_16622_gb300.workloads import uniform_system

    mcfmm.load()
    rho = 1.0 / 3.3 ** 3
    p, h, beta, nu = 11, 0.25, 1.0, 0.438
    sizes = [1000, 2000, 5000, 10_000, 20_000, 50_000, 100_000, 200_000, 500_000, 1_000_000]
    # local method twice: its plain schedule (the paper's split: Alg. L.2 in
    # the accept) and the speculative phased schedule of this implementation
    # (the contributions computed during the propose phase, the accept adds)
    methods = (("local", 0.327, mcfmm.SETUP_P2L, mcfmm.SCHEDULE_PLAIN),
               ("local_spec", 0.327, mcfmm.SETUP_P2L, mcfmm.SCHEDULE_PHASED),
               ("multipole", 0.138, mcfmm.SETUP_MULTIPOLE, None))
    rows = []
    t0 = time.perf_counter()
    for n in sizes:
        a = (n / rho) ** (1.0 / 3.0)
        pos, q = uniform_system(n, a, seed=n)
        for name, alpha, mode, sched in methods:
            L = model_levels(n, alpha)
            ctx = mcfmm.Context(pos, q, a, L, p, precision=mcfmm.FP64)
            ctx.setup(mode)
            if sched is not None:
                ctx.set_schedule(sched)
            ctx.run(2000, seed=1, beta=beta, half_width=h, stats=False)
            ctx.profile(True)
            ctx.profile_read()
            ctx.run(5000, seed=2, beta=beta, half_width=h, stats=False)
            pr = ctx.profile_read().astype(np.float64)
            ctx.profile(False)
            ctx.close()
            steps, acc = max(pr[5], 1.0), max(pr[6], 1.0)
            rows.append({"n": n, "method": name, "levels": L, "n_per_cell": n / 8.0 ** (L - 1),
                         "propose_us": (pr[0] + pr[1] + pr[2]) / steps / 1e3,
                         "accept_us": (pr[3] + pr[4]) / acc / 1e3, "acceptance": pr[6] / steps})
    torch.cuda.synchronize()
    fits = {}
    for name, _, _, _ in methods:
        rs = [r for r in rows if r["method"] == name]
        for stage in ("propose", "accept"):
            fits[f"{name}_{stage}"] = fit_performance_model(rs, f"{stage}_us")

    def T(name, stage, n, alpha):
        return performance_model(fits[f"{name}_{stage}"], n, model_levels(n, alpha))

    f = fits
    speedup, s_inf = {}, {}
    for loc in ("local", "local_spec"):
        sp = {}
        for n in sizes:
            mp = T("multipole", "propose", n, 0.138) + nu * T("multipole", "accept", n, 0.138)
            lo = T(loc, "propose", n, 0.327) + nu * T(loc, "accept", n, 0.327)
            sp[str(n)] = mp / lo
        speedup[loc] = sp
        den = f[f"{loc}_propose"]["gamma"] + nu * f[f"{loc}_accept"]["gamma"]
        num = f["multipole_propose"]["gamma"] + nu * f["multipole_accept"]["gamma"]
        s_inf[loc] = num / den if den > 0 else None
    # the measured ratio of the step times (propose + nu accept) per size
    measured = {}
    for loc in ("local", "local_spec"):
        m = {}
        for n in sizes:
            r_l = next(r for r in rows if r["n"] == n and r["method"] == loc)
            r_m = next(r for r in rows if r["n"] == n and r["method"] == "multipole")
            m[str(n)] = ((r_m["propose_us"] + nu * r_m["accept_us"])
                         / (r_l["propose_us"] + nu * r_l["accept_us"]))
        measured[loc] = m
    out = {"metric": "performance model of Sec. 5.4 fitted to GPU propose/accept times",
           "workload": "uniform +-1 charges, NaCl density (spacing 3.3 A), p = 11, h = 0.25 A, FP64",
           "rows": rows, "fits": fits, "speedup_nu_0.438": speedup, "s_inf": s_inf,
           "measured_speedup_nu_0.438": measured,
           "paper": {"s_inf": 2.02, "measured_speedup_range": [1.18, 1.34]},
           "seconds": time.perf_counter() - t0}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.accuracy:
        accuracy_study(args)
        return
    if args.model_fit:
        model_fit_study()
        return
    if args.profile:
        profile_launch(args)
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    gpu_arm(args)


if __name__ == "__main__":
    main()
