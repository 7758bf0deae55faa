"""The allocation-free entry point mc_p2l_level_noalloc.

Some callers cannot let a library allocate device memory (they hand out
every byte from their own pool, or allocation would stall the device at the
wrong time).  They call mc_p2l_level_noalloc with buffers they own; it keeps
its intermediate sums in a fixed device array of the library.  Its level
expansions must equal the oracle's Alg. L.3 expansions and the ones mc_setup
stores, within the array tolerance of the other parity tests, on two calls in
a row (the second call reuses the scratch the first one left behind), and
the calls after the first must leave the device's free memory unchanged.
This file sorts last so that a run that stops at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import oracle as O
from paper_2006_16622_gb300 import mcfmm
from paper_2006_16622_gb300.workloads import uniform_system

pytestmark = pytest.mark.gpu

ARR_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    mcfmm.load()


def _by_finest_cell(pos, q, box, levels):
    """charges grouped by finest cell (the library's cell rule) + offsets"""
    nL = 1 << (levels - 1)
    c = np.minimum(np.floor(pos * (nL / box)).astype(np.int64), nL - 1)
    cell = (c[:, 0] * nL + c[:, 1]) * nL + c[:, 2]
    order = np.argsort(cell, kind="stable")
    part = np.ascontiguousarray(np.concatenate([pos[order], q[order, None]], axis=1))
    start = np.searchsorted(cell[order], np.arange(nL ** 3 + 1)).astype(np.int32)
    return part, start


@pytest.mark.parametrize("bc", [mcfmm.BC_PBC, mcfmm.BC_FREE])
def test_noalloc_level_expansions_match_oracle(bc):
    import torch
    n, a, L, p = 3000, 14.0, 4, 8
    pos, q = uniform_system(n, a, seed=21)
    orc = O.System(pos, q, a, L, p, bc=bc)
    orc.setup()
    ctx = mcfmm.Context(pos, q, a, L, p, bc=bc)
    ctx.setup()
    part, start = _by_finest_cell(pos, q, a, L)
    d_part = torch.tensor(part, dtype=torch.float64, device="cuda")
    d_start = torch.tensor(start, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    lmin = 2 if bc == mcfmm.BC_PBC else 3
    levels = list(range(lmin, L + 1))
    # every output buffer exists before the first call, so nothing but the
    # entry point itself runs between the free-memory readings
    outs = {lv: torch.empty(((1 << (lv - 1)) ** 3, (p + 1) ** 2), dtype=torch.float64,
                            device="cuda") for lv in levels}
    free_after_first = None
    for call in range(2):
        for level in levels:
            outs[level].fill_(float("nan"))
            torch.cuda.synchronize()
            if free_after_first is not None:
                assert torch.cuda.mem_get_info()[0] == free_after_first, (call, level)
            rc = mcfmm.p2l_level_noalloc(d_part.data_ptr(), d_start.data_ptr(), n, a, L, level,
                                         p, bc, outs[level].data_ptr(), stream)
            assert rc == mcfmm.MC_OK, rc
            torch.cuda.synchronize()
            if free_after_first is None:
                # the first call may load the module's code; later ones add nothing
                free_after_first = torch.cuda.mem_get_info()[0]
            else:
                assert torch.cuda.mem_get_info()[0] == free_after_first, (call, level)
            got = outs[level].cpu().numpy()
            assert np.all(np.isfinite(got))
            want = orc.local(level)
            scale = np.max(np.abs(want))
            assert np.max(np.abs(got - want)) <= ARR_TOL * scale, (call, level)
            assert np.max(np.abs(got - ctx.local(level))) <= ARR_TOL * scale, (call, level)
    ctx.close()


def test_noalloc_refuses_levels_beyond_the_scratch():
    import torch
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    s = torch.zeros(8, dtype=torch.int32, device="cuda")
    # level 6 at p = 8: 32768 cells x 81 coefficients > 2^20 doubles
    rc = mcfmm.p2l_level_noalloc(d.data_ptr(), s.data_ptr(), 0, 10.0, 6, 6, 8, mcfmm.BC_PBC,
                                 d.data_ptr(), None)
    assert rc == -12
    assert mcfmm.load().mc_strerror(rc).decode().startswith("request exceeds")
