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


def test_tune_tau_rejects_bad_arguments_without_gpu(lib):
    import ctypes

    import numpy as np

    import paper_2510_05975_gb300.cng as cng

    X = np.zeros((100, 8), np.float32)
    Q = np.zeros((5, 8), np.float32)
    gt = np.zeros((5, 4), np.int32)
    p = cng.BuildParams(1.2, 0.0, 8, 16, 0, 0, 1e-5, 32, 0, 0)
    best, nt = ctypes.c_double(), ctypes.c_int32()
    trials = (cng.TauTrial * 8)()

    def call(Ls, target):
        L = np.asarray(Ls, np.int32)
        return lib.cng_tune_tau(X.ctypes.data, 0, 100, 8, ctypes.byref(p), Q.ctypes.data, 5, 4,
                                gt.ctypes.data, L.ctypes.data, len(L), target, None,
                                ctypes.byref(best), trials, 8, ctypes.byref(nt))

    assert call([16, 8], 0.9) == cng.CNG_E_INVAL      # widths must ascend
    assert "ascend" in cng.cng_last_error()
    assert call([2, 8], 0.9) == cng.CNG_E_INVAL       # every width >= k
    assert call([8, 16], 0.0) == cng.CNG_E_INVAL      # 0 < target <= 1
    assert call([8, 16], 1.5) == cng.CNG_E_INVAL
