"""The GPU path's interaction-list geometry (csrc/mc_geom.cuh) on the CPU.

The device header is compiled for the host with g++ and compared with the
oracle's interaction lists (Sec. 3.1, with the periodic images of
Sec. 3.4), cell by cell:

  - the per-parity offset table holds the 189 offsets of every cell's list;
  - on levels with at most 4 cells per axis, the 189 accept entries of a
    list (small_entry) are the oracle's (canonical cell, image shift)
    entries, images repeated, and in free space exactly its in-box cells;
  - on larger levels the accept items of a move from cell alpha to alpha'
    (large_item) own every cell of IL(alpha) u IL(alpha') exactly once, an
    item of the alpha' list owning its own targets, an item of the alpha
    list only those outside IL(alpha').
No GPU.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2006_16622_gb300.workloads import uniform_system

pytestmark = pytest.mark.usefixtures("oracle_lib")

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

static unsigned short il[8][189];

int main(int argc, char** argv) {
  il_table_init(il);
  const int mode = atoi(argv[1]);
  if (mode == 0) {  // the offset table
    for (int par = 0; par < 8; par++)
      for (int k = 0; k < 189; k++) {
        int ox, oy, oz;
        il_unpack(il[par][k], &ox, &oy, &oz);
        std::printf("%d %d %d %d\n", par, ox, oy, oz);
      }
    return 0;
  }
  const int nl = atoi(argv[2]);
  const bool pbc = atoi(argv[3]) != 0;
  const int co[3] = {atoi(argv[4]), atoi(argv[5]), atoi(argv[6])};
  const int cn[3] = {atoi(argv[7]), atoi(argv[8]), atoi(argv[9])};
  if (mode == 1) {  // small-level entries of the list of co
    for (int k = 0; k < 189; k++) {
      const SmallEntry se = small_entry(il, co, nl, pbc, k);
      std::printf("%d %d %d %d %d %d %d\n", se.valid ? 1 : 0, se.t3[0], se.t3[1], se.t3[2],
                  co[0] + se.o[0], co[1] + se.o[1], co[2] + se.o[2]);
    }
    return 0;
  }
  // mode 2: large-level items of a move from co to cn
  const bool samel = co[0] == cn[0] && co[1] == cn[1] && co[2] == cn[2];
  const int items = samel ? 189 : 378;
  for (int k = 0; k < items; k++) {
    const LargeItem it = large_item(il, co, cn, nl, pbc, samel, k);
    std::printf("%d %d %d %d %d\n", it.owner ? 1 : 0, it.from_new ? 1 : 0, it.tc[0], it.tc[1], it.tc[2]);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("geom")
    src = d / "geom.cpp"
    src.write_text(HARNESS.replace("HEADER", os.path.abspath(HEADER)))
    out = d / "geom"
    r = subprocess.run([gxx, "-O2", "-std=c++17", "-o", str(out), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return str(out)


def _run(exe, *args):
    out = subprocess.run([exe] + [str(a) for a in args], check=True, capture_output=True, text=True).stdout
    return np.array([[int(v) for v in ln.split()] for ln in out.splitlines()])


def _systems():
    pos, q = uniform_system(64, 16.0, seed=2)
    # levels 2..5: 2, 4, 8 and 16 cells per axis
    return {bc: O.System(pos, q, 16.0, 5, 2, bc=bc) for bc in (O.BC_PBC, O.BC_FREE)}


def _oracle_entries(s, level, c):
    """(canonical cell, extended cell) of every entry of the oracle's list."""
    n = 1 << (level - 1)
    out = []
    for lin, sx, sy, sz in s.interaction_list(level, c):
        b = (lin // (n * n), (lin // n) % n, lin % n)
        out.append((b, (b[0] + sx * n, b[1] + sy * n, b[2] + sz * n)))
    return out


def test_offset_table_matches_oracle_lists(exe):
    tab = _run(exe, 0)
    s = _systems()[O.BC_PBC]
    level, n = 5, 16
    for par in range(8):
        c = (4 + ((par >> 2) & 1), 8 + ((par >> 1) & 1), 6 + (par & 1))
        dev = sorted(tuple(r[1:]) for r in tab if r[0] == par)
        ora = sorted(tuple(e[k] - c[k] for k in range(3)) for _, e in _oracle_entries(s, level, c))
        assert len(dev) == 189 and len(set(dev)) == 189
        assert dev == ora, par


@pytest.mark.parametrize("bc", ["pbc", "free"])
def test_small_level_entries_match_oracle(exe, bc):
    s = _systems()[O.BC_PBC if bc == "pbc" else O.BC_FREE]
    rng = np.random.default_rng(4)
    for level in (2, 3):
        if bc == "free" and level < 3:
            continue  # free space: no lists below level 3
        n = 1 << (level - 1)
        for _ in range(6):
            c = tuple(int(v) for v in rng.integers(0, n, 3))
            rows = _run(exe, 1, n, 1 if bc == "pbc" else 0, *c, *c)
            dev = sorted((tuple(r[1:4]), tuple(r[4:7])) for r in rows if r[0] == 1)
            ora = sorted(_oracle_entries(s, level, c))
            assert dev == ora, (level, c)


@pytest.mark.parametrize("bc", ["pbc", "free"])
def test_large_level_items_own_the_union_once(exe, bc):
    s = _systems()[O.BC_PBC if bc == "pbc" else O.BC_FREE]
    rng = np.random.default_rng(5)
    for level in (4, 5):
        n = 1 << (level - 1)
        for t in range(12):
            co = rng.integers(0, n, 3)
            step = rng.integers(-1, 2, 3) if t % 3 else np.zeros(3, dtype=int)
            cn = (co + step) % n if bc == "pbc" else np.clip(co + step, 0, n - 1)
            co, cn = tuple(int(v) for v in co), tuple(int(v) for v in cn)
            rows = _run(exe, 2, n, 1 if bc == "pbc" else 0, *co, *cn)
            owned = [tuple(r[2:5]) for r in rows if r[0] == 1]
            il_o = {b for b, _ in _oracle_entries(s, level, co)}
            il_n = {b for b, _ in _oracle_entries(s, level, cn)}
            assert len(owned) == len(set(owned)), (level, co, cn)
            assert set(owned) == il_o | il_n, (level, co, cn)
            for r in rows:
                if r[0] == 1 and r[1] == 0:
                    assert tuple(r[2:5]) not in il_n
