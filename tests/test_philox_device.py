"""The GPU path's proposal stream (csrc/mc_philox.cuh) on the CPU.

The device header is compiled for the host with g++ (the CUDA intrinsics it
uses are integer high multiplies and round-to-nearest double operations):
its Philox4x32-10 reproduces the generator's published known-answer values
(tests/golden/philox_kat.txt), and its proposals (particle, displacement,
acceptance uniform) equal the oracle's bit for bit over a few thousand
steps, several seeds, chains and sizes, both through the whole-proposal
form and the per-axis form the kernels use.  No GPU.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.usefixtures("oracle_lib")

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "paper_2006_16622_gb300", "csrc", "mc_philox.cuh")

HARNESS = r"""
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#define __device__
#define __forceinline__ inline
static inline uint32_t __umulhi(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline double __dadd_rn(double a, double b) { return a + b; }
static inline double __dsub_rn(double a, double b) { return a - b; }
#include "HEADER"

int main(int argc, char** argv) {
  // known-answer mode: counter and key words from the command line
  if (argc == 7) {
    uint32_t c[4];
    for (int i = 0; i < 4; i++) c[i] = (uint32_t)strtoul(argv[1 + i], nullptr, 16);
    philox4x32_10(c, (uint32_t)strtoul(argv[5], nullptr, 16), (uint32_t)strtoul(argv[6], nullptr, 16));
    std::printf("%08x %08x %08x %08x\n", c[0], c[1], c[2], c[3]);
    return 0;
  }
  // proposal mode: seed chain n h steps; one line per step
  const unsigned long long seed = strtoull(argv[1], nullptr, 10);
  const uint32_t chain = (uint32_t)strtoul(argv[2], nullptr, 10);
  const int n = atoi(argv[3]);
  const double h = atof(argv[4]);
  const long long steps = atoll(argv[5]);
  for (long long s = 0; s < steps; s++) {
    int j, ja;
    double d[3], u, da[3], ua = 0;
    mc_proposal(seed, (unsigned long long)s, chain, n, h, &j, d, &u);
    for (int a = 0; a < 3; a++) mc_proposal_axis(seed, (unsigned long long)s, chain, n, h, a, &ja, &da[a], a == 0 ? &ua : nullptr);
    const int same = (ja == j && da[0] == d[0] && da[1] == d[1] && da[2] == d[2] && ua == u) ? 1 : 0;
    std::printf("%d %a %a %a %a %d\n", j, d[0], d[1], d[2], u, same);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("philox")
    src = d / "philox.cpp"
    src.write_text(HARNESS.replace("HEADER", os.path.abspath(HEADER)))
    out = d / "philox"
    r = subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-o", str(out), str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return str(out)


def test_device_philox_known_answers(exe):
    path = os.path.join(HERE, "golden", "philox_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        out = subprocess.run([exe] + r[:6], check=True, capture_output=True, text=True).stdout.split()
        assert out == r[6:10], (r, out)


@pytest.mark.parametrize("seed,chain,n,h", [(0, 0, 1000, 0.5), (7, 3, 100000, 0.3), (2**40 + 5, 63, 48920, 0.25)])
def test_device_proposals_equal_oracle(exe, seed, chain, n, h):
    steps = 2000
    out = subprocess.run([exe, str(seed), str(chain), str(n), repr(h), str(steps)], check=True,
                         capture_output=True, text=True).stdout.splitlines()
    assert len(out) == steps
    for s, line in enumerate(out):
        f = line.split()
        j, d, u, same = int(f[0]), [float.fromhex(v) for v in f[1:4]], float.fromhex(f[4]), int(f[5])
        jo, do, uo = O.proposal(n, h, seed=seed, step=s, chain=chain)
        assert same == 1, s
        assert j == jo and 0 <= j < n, (s, j, jo)
        assert np.array_equal(np.array(d), do), (s, d, do)
        assert u == uo, (s, u, uo)
