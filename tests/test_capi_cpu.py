"""CPU-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point include/gb3fmm.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gb3fmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1405_2255_gb300 import build
    build.build()
    from paper_1405_2255_gb300 import gb3fmm
    return gb3fmm.load()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("fmm_create", "fmm_evaluate", "fmm_evaluate_host", "fmm_evaluate_batch", "fmm_direct",
                 "fmm_destroy", "fmm_strerror", "fmm_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_1405_2255_gb300 import gb3fmm
    assert sorted(gb3fmm.EXPORTS) == _declared()


def test_host_only_calls(lib):
    from paper_1405_2255_gb300 import gb3fmm
    assert "sm_103a" in gb3fmm.fmm_version()
    assert gb3fmm.fmm_strerror(gb3fmm.FMM_E_INVALID) == "invalid argument or input"
    p = gb3fmm.fmm_default_params()
    assert p.p == 8 and p.eps == 1e-7 and p.mac == gb3fmm.FMM_MAC_A and p.precision == gb3fmm.FMM_PREC_MIXED


def test_create_rejects_bad_params(lib):
    from paper_1405_2255_gb300 import gb3fmm
    p = gb3fmm.fmm_default_params()
    p.p = 0
    h = ctypes.c_void_p()
    assert lib.fmm_create(ctypes.byref(h), ctypes.byref(p), 0) == gb3fmm.FMM_E_INVALID
    p = gb3fmm.fmm_default_params()
    p.eps = -1.0
    assert lib.fmm_create(ctypes.byref(h), ctypes.byref(p), 0) == gb3fmm.FMM_E_INVALID


def test_footprint_is_host_only_and_monotone(lib):
    from paper_1405_2255_gb300 import gb3fmm
    fp = [gb3fmm.fmm_footprint_bytes(n) for n in (0, 1, 1000, 10**5, 10**6, 10**7)]
    assert all(b > a for a, b in zip(fp, fp[1:]))
    # larger expansions and smaller leaves need more room per particle
    assert gb3fmm.fmm_footprint_bytes(10**6, p=12) > gb3fmm.fmm_footprint_bytes(10**6, p=8)
    assert gb3fmm.fmm_footprint_bytes(10**6, leaf_size=16) > gb3fmm.fmm_footprint_bytes(10**6, leaf_size=64)
    assert gb3fmm.fmm_footprint_bytes(-1) == -1
    assert gb3fmm.fmm_footprint_bytes(10, p=0) == -1
