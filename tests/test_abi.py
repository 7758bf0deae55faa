"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point that include/mcfmm.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2006_16622_gb300 import build
    return build.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "mcfmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mc_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["mc_init", "mc_setup", "mc_propose", "mc_accept", "mc_run", "mc_energy"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(\w+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in _declared():
        assert hasattr(lib, n)


def test_binding_rejects_bad_arguments_without_gpu(libpath):
    import numpy as np
    from paper_2006_16622_gb300 import mcfmm
    lib = mcfmm.load()
    h = ctypes.c_void_p()
    pos = np.zeros((2, 3))
    q = np.array([1.0, -1.0])
    P = mcfmm._ptr
    # argument checks run before any CUDA call
    assert lib.mc_init(ctypes.byref(h), 2, P(pos), P(q), 1.0, 1, 4, 0, 0, 0, None) == -4
    assert lib.mc_init(ctypes.byref(h), 2, P(pos), P(q), 1.0, 3, 16, 0, 0, 0, None) == -9
    assert lib.mc_init(ctypes.byref(h), 2, P(pos + 2.0), P(q), 1.0, 3, 4, 0, 0, 0, None) == -5
    assert lib.mc_init(ctypes.byref(h), 2, P(pos), P(np.array([1.0, 1.0])), 1.0, 3, 4, 0, 0, 0,
                       None) == -2
    assert lib.mc_init(ctypes.byref(h), 0, P(pos), P(q), 1.0, 3, 4, 0, 0, 0, None) == -1
    assert lib.mc_strerror(-7).decode().startswith("device-side wait")
