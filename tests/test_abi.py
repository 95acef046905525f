"""The C ABI library builds, loads and exports every entry point include/tdh.h declares;
argument checks that return before any CUDA call behave as documented (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1604_07486_gb300 import build
    import paper_1604_07486_gb300 as tdh
    build.build()
    return tdh.lib()


def _declared():
    names = set()
    with open(os.path.join(ROOT, "include", "tdh.h")) as f:
        text = f.read()
    for m in re.finditer(r"^\s*(?:int|const char\*)\s+(tdh_\w+)\s*\(", text, re.M):
        names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"tdh_plan_create", "tdh_plan_execute", "tdh_plan_destroy"} <= names
    for name in names:
        assert hasattr(lib, name), name
    import paper_1604_07486_gb300 as tdh
    assert names == set(tdh.EXPORTS)


def test_error_codes_without_device(lib):
    import paper_1604_07486_gb300 as tdh
    p = tdh._Params()
    p.prec = tdh.FP32
    h = ctypes.c_void_p()
    assert lib.tdh_plan_create(99, 100, ctypes.byref(p), 1e-7, ctypes.byref(h)) == -1
    assert b"kind" in lib.tdh_last_error()
    assert lib.tdh_plan_create(0, 0, ctypes.byref(p), 1e-7, ctypes.byref(h)) == -1
    assert lib.tdh_plan_create(0, 10, ctypes.byref(p), 0.0, ctypes.byref(h)) == -1
    assert lib.tdh_plan_create(0, 10, None, 1e-7, ctypes.byref(h)) == -1
    p.prec = 7
    assert lib.tdh_plan_create(0, 10, ctypes.byref(p), 1e-7, ctypes.byref(h)) == -1
    assert lib.tdh_plan_destroy(None) == 0
    assert lib.tdh_plan_execute(None, None, None, 1, None) == -1
    assert lib.tdh_plan_query(None, None, None) == -1
    K = ctypes.c_int64()
    assert lib.tdh_pchol(None, 10, 0, 1e-7, 4, None, None, ctypes.byref(K), None) == -1
    assert lib.tdh_symbols(0, 0, None, None, None, None, None, None) == -1


def test_product_path_has_no_oracle_dependency():
    """The package never imports, links or runs anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_1604_07486_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.replace("Oracle", ""), f
