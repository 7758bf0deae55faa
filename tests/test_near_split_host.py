"""The near-field split of the chain kernels (csrc/mc_geom.cuh near_part) on
the CPU: the device header is compiled for the host with g++, its item map
printed for both kernels' item counts (the barrier-free chain: 54 P items,
2 P per cell when r and r' share their finest cell; the phased chain: 27 or
54 P items, 1 or 2 P per shared cell), and the slot loop of the near item
(slot 32 part + lane, stepping by 32 nparts, 32 lanes) emulated: for every
split P = 1..4 and cell occupancy, each slot of each near cell is summed
exactly once for each side (Alg. 1 over the 27 near cells, old and new
position).  No GPU.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "paper_2006_16622_gb300", "csrc", "mc_geom.cuh")

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#define __device__
#define __forceinline__ inline
struct Dim { unsigned x; };
#define threadIdx (Dim{0u})
#define blockDim (Dim{1u})
#include "HEADER"

int main(int argc, char** argv) {
  const int nitems = atoi(argv[1]);
  const bool same = atoi(argv[2]) != 0;
  const int nparts = atoi(argv[3]), nsame = atoi(argv[4]);
  for (int k0 = 0; k0 < nitems; k0++) {
    const NearPart r = near_part(k0, same, nparts, nsame);
    std::printf("%d %d %d %d\n", r.k, r.side, r.part, r.nparts);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("near")
    src = d / "h.cpp"
    src.write_text(HARNESS.replace("HEADER", os.path.abspath(HEADER)))
    exe = d / "h"
    subprocess.run([gxx, "-std=c++17", "-O1", "-o", str(exe), str(src)], check=True)

    def run(nitems, same, nparts, nsame):
        out = subprocess.run([str(exe), str(nitems), str(int(same)), str(nparts), str(nsame)],
                             check=True, capture_output=True, text=True).stdout
        return [tuple(int(v) for v in line.split()) for line in out.splitlines()]

    return run


def _coverage(items, cnt):
    """(cell, side) -> list of slots summed, side 2 counting for both sides"""
    cov = {}
    for k, side, part, nparts in items:
        if k < 0:
            continue
        for lane in range(32):
            s = 32 * part + lane
            while s < cnt:
                for sd in ((0, 1) if side == 2 else (side,)):
                    cov.setdefault((k, sd), []).append(s)
                s += 32 * nparts
    return cov


@pytest.mark.parametrize("kernel", ["barrier-free", "phased"])
@pytest.mark.parametrize("P", [1, 2, 3, 4])
@pytest.mark.parametrize("same", [False, True])
def test_every_slot_once(harness, kernel, P, same):
    if kernel == "barrier-free":
        nsame = 2 * P
        nitems = 54 * P
    else:
        nsame = 1 if P == 1 else 2 * P
        nitems = 27 * nsame if same else 54 * P
    items = harness(nitems, same, P, nsame)
    assert len(items) == nitems
    for cnt in (0, 1, 31, 32, 33, 63, 64, 65, 100, 190, 255, 256, 384):
        cov = _coverage(items, cnt)
        for k in range(27):
            for sd in (0, 1):
                got = sorted(cov.get((k, sd), []))
                assert got == list(range(cnt)), (kernel, P, same, cnt, k, sd)
        assert set(cov) <= {(k, sd) for k in range(27) for sd in (0, 1)}
