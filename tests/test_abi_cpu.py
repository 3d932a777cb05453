"""Host-side checks of the C ABI that need no GPU.

The library is compiled here (nvcc cross-compiles for sm_103a), loaded with
ctypes, and must export every function declared in include/blockoa.h.
Argument validation happens on the host before any CUDA call, so invalid
calls are exercised without a device.
"""
import ctypes as ct
import os
import re

import pytest

from paper_2510_23221_gb300 import blockoa as bo
from paper_2510_23221_gb300 import build as bld

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:int|void|long long|const char \*)\s*(blockoa_\w+)\s*\(", text, re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    bld.build()
    return bo.library()


def test_header_declares_the_boundary():
    names = _declared()
    for core in ("blockoa_assemble", "blockoa_block_solve", "blockoa_combine", "blockoa_apply_operator"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    raw = ct.CDLL(bo.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(raw, n)]
    assert not missing, missing
    assert set(bo.EXPORTED) <= set(_declared())


def test_library_resolves_all_its_own_symbols(lib):
    """Every symbol the library references is defined or comes from a system
    or CUDA library: loading with immediate binding fails otherwise (ctypes
    binds lazily, so a missing internal definition would only surface at the
    first call on a GPU)."""
    import subprocess
    import sys
    code = f"import ctypes, os; ctypes.CDLL({bo.LIB_PATH!r}, mode=os.RTLD_NOW)"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]


def test_status_strings(lib):
    assert bo.status_string(bo.OK) == "ok"
    assert "invalid" in bo.status_string(bo.ERR_INVALID)
    assert "converge" in bo.status_string(bo.ERR_NOT_CONVERGED)
    assert bo.status_string(12345) == "unknown status"


def test_invalid_arguments_rejected_on_host(lib):
    h = ct.c_void_p()
    assert lib.blockoa_assemble(None, 1, None, ct.byref(h)) == bo.ERR_INVALID
    assert lib.blockoa_assemble((bo.ChipDesc * 1)(), 0, None, ct.byref(h)) == bo.ERR_INVALID
    bad = bo.ChipDesc()
    bad.nx = 0
    assert lib.blockoa_assemble((bo.ChipDesc * 1)(bad), 1, None, ct.byref(h)) == bo.ERR_INVALID
    assert h.value is None
    assert lib.blockoa_block_solve(None, None, None, 4, None, None, None) == bo.ERR_INVALID
    assert lib.blockoa_combine(None, None, None, None, 4, 4, bo.FP64, None) == bo.ERR_INVALID
    assert lib.blockoa_apply_operator(None, None, None, 4, bo.FP64, None) == bo.ERR_INVALID
    assert lib.blockoa_pair_check(None, None, None, 4, bo.FP64, None, None) == bo.ERR_INVALID
    assert lib.blockoa_pair_check_static(None, None, None, 4, bo.FP64, None, None) == bo.ERR_INVALID
    assert lib.blockoa_residual_ratio(None, None, None, 4, None, None) == bo.ERR_INVALID
    assert lib.blockoa_inject_chip_status(None, 0, bo.ERR_TIMEOUT, 0) == bo.ERR_INVALID
    assert lib.blockoa_build_rhs(None, None, None, 4, None) == bo.ERR_INVALID
    assert lib.blockoa_build_rhs_volume(None, None, None, 4, None) == bo.ERR_INVALID
    assert lib.blockoa_export_conductances(None, 0, None, None, None, None) == bo.ERR_INVALID
    assert lib.blockoa_reassemble(None, None, 1, None) == bo.ERR_INVALID
    lib.blockoa_destroy(None)


def test_bad_chip_descriptors_rejected(lib):
    import numpy as np
    keep = []
    from paper_2510_23221_gb300 import synth
    chip = synth.random_small_chip(1, 3, 3, 2)
    for field, value in (("dx", -1.0), ("h_top", float("nan")), ("dy", 0.0), ("h_side", -1.0),
                         ("h_bottom", float("-inf")), ("dx", float("inf"))):
        d = bo._desc(chip, keep)
        setattr(d, field, value)
        h = ct.c_void_p()
        assert lib.blockoa_assemble((bo.ChipDesc * 1)(d), 1, None, ct.byref(h)) == bo.ERR_INVALID
    d = bo._desc(chip, keep)
    kneg = np.array([1.0, -2.0])
    keep.append(kneg)
    d.layer_k = kneg.ctypes.data_as(ct.POINTER(ct.c_double))
    h = ct.c_void_p()
    assert lib.blockoa_assemble((bo.ChipDesc * 1)(d), 1, None, ct.byref(h)) == bo.ERR_INVALID
