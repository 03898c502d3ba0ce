"""The C-ABI library builds, loads, and exports every function include/iwfpm.h declares."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "iwfpm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(iwf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_04507_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_core_entry_points():
    names = _declared()
    for must in ["iwf_plan_create", "iwf_plan_destroy", "iwf_apply", "iwf_set_potential",
                 "iwf_window", "iwf_last_error"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_mirrors_header(lib):
    from paper_2404_04507_gb300 import capi
    missing = [n for n in _declared() if not hasattr(capi, n)]
    assert not missing, f"binding lacks: {missing}"


def test_calls_fail_cleanly_without_gpu_or_args(lib):
    from paper_2404_04507_gb300 import capi
    h = ctypes.c_void_p()
    st = capi.iwf_plan_create(ctypes.byref(h), 1, 2, None, None, None, None)
    assert st == -1 and h.value is None
    assert b"NULL" in capi.iwf_last_error()
    assert capi.iwf_version() >= 100
