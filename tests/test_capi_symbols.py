"""The C-ABI library loads and exports every function include/itpp.h declares.

Runs without a GPU: loading the library and the calls checked here
(argument validation, status strings, version) touch no device.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(itpp_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    import paper_2601_14400_gb300 as p
    if not os.path.exists(p.LIB_PATH):
        p.build()
    return p


def test_every_declared_symbol_is_exported(lib):
    L = ctypes.CDLL(lib.LIB_PATH)
    declared = _declared()
    assert "itpp_create" in declared and "itpp_apply_trotter_layer" in declared
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b(itpp_\w+)\b", out))
    assert declared <= exported


def test_binding_covers_the_header(lib):
    assert set(lib.exported_names()) == _declared()


def test_status_strings_and_version(lib):
    L = lib.lib()
    assert L.itpp_version().decode().startswith("itpp-gb300")
    for s in range(9):
        assert L.itpp_status_string(s)
    assert L.itpp_status_string(0).decode() == "ok"


def test_create_rejects_bad_arguments_before_touching_a_device(lib):
    L = lib.lib()
    h = ctypes.c_void_p()
    p = lib.itpp_params()
    p.delta = 1e-6
    p.cap_M = 100
    gx = np.zeros(1, np.uint64)
    gz = np.zeros(1, np.uint64)
    al = np.array([-1.0])
    u64 = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    f64 = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.itpp_create(0, u64(gx), u64(gz), f64(al), 1, 0.1, ctypes.byref(p), None,
                         ctypes.byref(h)) == 1
    assert L.itpp_create(129, u64(gx), u64(gz), f64(al), 1, 0.1, ctypes.byref(p), None,
                         ctypes.byref(h)) == 1
    p.delta = -1.0
    assert L.itpp_create(8, u64(gx), u64(gz), f64(al), 1, 0.1, ctypes.byref(p), None,
                         ctypes.byref(h)) == 1
    p.delta = 1e-6
    gx[0] = np.uint64(1) << np.uint64(9)         # bit >= n
    assert L.itpp_create(8, u64(gx), u64(gz), f64(al), 1, 0.1, ctypes.byref(p), None,
                         ctypes.byref(h)) == 1
    assert L.itpp_destroy(None) == 0
