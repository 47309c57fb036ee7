"""The C-ABI library loads without a GPU and exports every entry point include/fmm.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        names += re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(fmm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2009_00767_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("fmm_plan", "fmm_potential", "fmm_sync", "fmm_plan_destroy", "fmm_status_string",
                 "fmm_direct_targets", "fmm_potential_host", "fmm_plan_stats", "fmm_set_stream"):
        assert name in d


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol(lib):
    from paper_2009_00767_gb300 import binding
    assert set(_declared()) <= set(binding.SIGNATURES)


def test_status_strings_and_host_side_argument_checks(lib):
    from paper_2009_00767_gb300 import binding as b
    assert b.status_string(b.FMM_OK) == "ok"
    assert "outside" in b.status_string(b.FMM_ERR_OUT_OF_BOX)
    assert b.status_string(999) == "unknown status"
    h = ctypes.c_void_p()
    L = b.library()
    # rejected before any CUDA call: bad n, levels, p, box, precision, null out
    assert L.fmm_plan(ctypes.byref(h), 0, 3, 8, 5.0, 0, None) == b.FMM_ERR_INVALID_ARG
    assert L.fmm_plan(ctypes.byref(h), 10, 13, 8, 5.0, 0, None) == b.FMM_ERR_INVALID_ARG
    assert L.fmm_plan(ctypes.byref(h), 10, 3, 0, 5.0, 0, None) == b.FMM_ERR_INVALID_ARG
    assert L.fmm_plan(ctypes.byref(h), 10, 3, 41, 5.0, 0, None) == b.FMM_ERR_INVALID_ARG
    assert L.fmm_plan(ctypes.byref(h), 10, 3, 8, -1.0, 0, None) == b.FMM_ERR_INVALID_ARG
    assert L.fmm_plan(ctypes.byref(h), 10, 3, 8, float("nan"), 0, None) == b.FMM_ERR_INVALID_ARG
    assert L.fmm_plan(ctypes.byref(h), 10, 3, 8, 5.0, 99, None) == b.FMM_ERR_INVALID_ARG
    d = ctypes.c_double(1.0)
    assert L.fmm_probe_peak(7, ctypes.byref(d), None) == b.FMM_ERR_INVALID_ARG
    assert L.fmm_probe_peak(-1, ctypes.byref(d), None) == b.FMM_ERR_INVALID_ARG
    assert L.fmm_probe_peak(0, None, None) == b.FMM_ERR_INVALID_ARG
    assert L.fmm_plan(None, 10, 3, 8, 5.0, 0, None) == b.FMM_ERR_INVALID_ARG
    assert L.fmm_potential(None, None, None, None) == b.FMM_ERR_INVALID_ARG
    assert L.fmm_sync(None) == b.FMM_ERR_INVALID_ARG
    assert L.fmm_direct_targets(-1, None, None, 0, None, None, None) == b.FMM_ERR_INVALID_ARG
    L.fmm_plan_destroy(None)
