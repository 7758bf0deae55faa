"""One profiler-bracketed launch of the batched form, for ncu.

Builds the 64-chain benchmark batch (N log-uniform in [1000, 50000], density
0.1, ~20 charges per finest cell, p = 10), tunes its CTA split, runs three
warm-up launches and brackets one more launch with cudaProfilerStart/Stop,
so that `ncu --profile-from-start off -k regex:mc_batch_kernel -c 1` captures
exactly that launch.  Usage, from the repository root:

    python paper_2006_16622_gb300/batch_profile.py {fp64|fp32_eval} PROPOSALS_PER_CHAIN
"""
import os
import sys

sys.path.insert(0, os.getcwd())

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_2006_16622_gb300 import mcfmm  # noqa: E402
from paper_2006_16622_gb300.workloads import batched_systems, uniform_system  # noqa: E402


def main():
    mcfmm.load()
    prec = mcfmm.FP64 if sys.argv[1] == "fp64" else mcfmm.FP32_EVAL
    steps = int(sys.argv[2])
    ctxs = []
    for n, a, L, i in batched_systems(64, 1000, 50000, 0.1, 20.0):
        pos, q = uniform_system(n, a, seed=1000 + i)
        c = mcfmm.Context(pos, q, a, L, 10, precision=prec)
        c.setup()
        ctxs.append(c)
    b = mcfmm.Batch(ctxs)
    b.tune(trial_steps=300, beta=1.0, half_width=0.3)
    seeds = np.arange(64, dtype=np.uint64)
    for _ in range(3):
        b.run(steps, seeds, beta=1.0, half_width=0.3, stats=False)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    b.run(steps, seeds, beta=1.0, half_width=0.3, stats=False)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    ok = all(c.status() == 0 for c in ctxs)
    print("batch", sys.argv[1], steps, "ok" if ok else "FAILED", b.info()[1], flush=True)
    sys.exit(0 if ok else 1)


if __name__ == "__main__":
    main()
