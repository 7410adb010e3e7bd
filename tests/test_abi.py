"""The C ABI loads and exports every entry point include/cng.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2510_05975_gb300.cng as cng

    return cng.lib()


def declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(cngx?_\w+)\s*\(", text, re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert {"cng_build", "cng_search", "cng_free"} <= names
    for name in sorted(names):
        assert hasattr(lib, name), name


def test_binding_covers_exports(lib):
    import paper_2510_05975_gb300.cng as cng

    assert set(cng.EXPORTS) <= declared()


def test_last_error_without_gpu(lib):
    import ctypes

    import paper_2510_05975_gb300.cng as cng

    # an invalid call is rejected before any device work
    p = cng.BuildParams(1.2, 0.0, 0, 10, 0, 0, 1e-5, 32, 0, 0)
    h = ctypes.c_void_p()
    rc = lib.cng_build(None, 0, 100, 8, ctypes.byref(p), None, ctypes.byref(h), None)
    assert rc == cng.CNG_E_INVAL
    assert "non-NULL" in cng.cng_last_error()
