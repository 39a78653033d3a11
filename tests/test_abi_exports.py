"""The C-ABI library loads and exports every entry point include/qmccpw.h
declares (CPU only: no GPU call is made; the argument checks exercised here
return before the library touches CUDA)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            names.update(re.findall(r"^\s*(?:const\s+char\s*\*|int)\s*(qmccpw_\w+)\s*\(", text, re.M))
    return names


@pytest.fixture(scope="module")
def qlib():
    from paper_2209_11337_gb300 import build, qmccpw
    build.build()
    return qmccpw


def test_header_declares_the_plan_greeks_free_entry_points():
    names = declared_functions()
    for must in ("qmccpw_plan", "qmccpw_greeks", "qmccpw_free"):
        assert must in names


def test_library_exports_every_declared_symbol(qlib):
    L = qlib.library()
    names = declared_functions()
    assert names, "no declarations found"
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    assert set(qlib.EXPORTS) >= names


def test_plan_rejects_bad_descriptors_before_touching_the_device(qlib):
    L = qlib.library()
    h = ctypes.c_void_p()
    for d_max, r_max, reserved in ((0, 8, 0), (qlib.QMCCPW_D_LIMIT + 1, 8, 0), (64, 1, 0),
                                   (64, qlib.QMCCPW_R_LIMIT + 1, 0), (64, 8, 7)):
        desc = qlib.qmccpw_plan_desc(0, d_max, r_max, reserved, 1, None, 0)
        assert L.qmccpw_plan(ctypes.byref(h), ctypes.byref(desc)) == qlib.QMCCPW_ERR_INVALID_ARG
        assert qlib.qmccpw_last_error()
    assert L.qmccpw_plan(None, None) == qlib.QMCCPW_ERR_INVALID_ARG
    assert L.qmccpw_free(None) == qlib.QMCCPW_OK
    res = qlib.qmccpw_result()
    assert L.qmccpw_greeks(None, None, None, 1, 2, 0, 0, ctypes.byref(res)) == qlib.QMCCPW_ERR_INVALID_ARG
    assert qlib.qmccpw_version().startswith("qmccpw")


def test_binding_has_no_cpu_fallback(qlib, monkeypatch):
    monkeypatch.setattr(qlib, "_lib", None)
    monkeypatch.setattr(qlib, "LIB_PATH", "/nonexistent/libqmccpw.so")
    with pytest.raises(qlib.QmcCpwError):
        qlib.qmccpw_plan()
