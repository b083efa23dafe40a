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
    for s in range(10):
        assert L.itpp_status_string(s)
    assert L.itpp_status_string(9).decode() != "unknown status"
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


@pytest.mark.parametrize("W", [1, 2])
def test_sort_terms_gives_the_canonical_order(lib, W):
    # the host-only canonical sort against numpy's lexicographic sort; words
    # drawn from a few values so that keys share leading words
    rng = np.random.default_rng(7 + W)
    n = 5000
    pool = np.array([0, 1, 2, 1 << 40, (1 << 63) + 5, (1 << 64) - 1], dtype=np.uint64)
    x = pool[rng.integers(0, len(pool), (n, W))]
    z = pool[rng.integers(0, len(pool), (n, W))]
    keys = np.unique(np.concatenate([x, z], axis=1), axis=0)
    rng.shuffle(keys)
    x, z = keys[:, :W].copy(), keys[:, W:].copy()
    c = rng.standard_normal(x.shape[0])
    order = np.lexsort(tuple(z[:, w] for w in range(W - 1, -1, -1)) +
                       tuple(x[:, w] for w in range(W - 1, -1, -1)))
    sx, sz, sc = lib.sort_terms(x, z, c)
    assert np.array_equal(sx, x[order]) and np.array_equal(sz, z[order])
    assert np.array_equal(sc.view(np.uint64), c[order].view(np.uint64))


def test_sort_save_load_reject_bad_arguments(lib):
    L = lib.lib()
    u64 = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    f64 = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    x = np.zeros(3, np.uint64)
    c = np.zeros(3)
    assert L.itpp_sort_terms(3, u64(x), u64(x), f64(c), 1) == 1
    assert L.itpp_sort_terms(1, None, None, None, 1) == 1
    assert L.itpp_sort_terms(2, None, None, None, 0) == 0
    assert L.itpp_save(None, b"state.bin") == 1
    assert L.itpp_load(None, b"state.bin") == 1
    assert L.itpp_get_terms_sorted(None, u64(x), u64(x), f64(c), 3, u64(x)) == 1
