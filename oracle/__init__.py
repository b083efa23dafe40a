"""CPU oracle for imaginary-time Pauli propagation -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and the two
share no code: this package holds a plain C++ restatement of Algorithm 1
(``itpp_oracle.cpp``, loaded through ctypes) and dense-matrix references
(``dense.py``).  ``build()`` compiles the C++ file in place.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "itpp_oracle.cpp")
_LIB = os.path.join(_HERE, "lib", "liboracle.so")

_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with -O2 and no floating-point contraction."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", _LIB + ".tmp", _SRC]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_create.restype = ctypes.c_void_p
        L.oracle_create.argtypes = [ctypes.c_int, ctypes.c_int, _u64p, _u64p, _f64p,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                    ctypes.c_int]
        L.oracle_destroy.argtypes = [ctypes.c_void_p]
        L.oracle_apply_gate.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.oracle_apply_layers.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.oracle_count.restype = ctypes.c_uint64
        L.oracle_count.argtypes = [ctypes.c_void_p]
        L.oracle_get_terms.argtypes = [ctypes.c_void_p, _u64p, _u64p, _f64p]
        L.oracle_set_terms.argtypes = [ctypes.c_void_p, ctypes.c_uint64, _u64p, _u64p, _f64p]
        L.oracle_set_max_weight.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.oracle_expect_psd.argtypes = [ctypes.c_void_p, _u64p, _u64p, _f64p, ctypes.c_int,
                                        _f64p]
        L.oracle_coeffs.argtypes = [ctypes.c_void_p, _u64p, _u64p, ctypes.c_int, _f64p]
        L.oracle_expect.restype = ctypes.c_double
        L.oracle_expect.argtypes = [ctypes.c_void_p, _u64p, _u64p, _f64p, ctypes.c_int]
        L.oracle_record.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.oracle_frozen_value.argtypes = [ctypes.c_void_p, _f64p, _u64p, _u64p, _f64p,
                                          ctypes.c_int, _f64p]
        L.oracle_adjoint.argtypes = [ctypes.c_void_p, _u64p, _u64p, _f64p, ctypes.c_int,
                                     _f64p, _f64p]
        L.oracle_commutes.argtypes = [ctypes.c_int, _u64p, _u64p, _u64p, _u64p]
        L.oracle_pauli_product.argtypes = [ctypes.c_int, _u64p, _u64p, _u64p, _u64p,
                                           _u64p, _u64p]
        _lib = L
    return _lib


def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(_u64p)


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_f64p)


class OracleError(RuntimeError):
    pass


class Oracle:
    """One propagation: state starts at the identity (Algorithm 1)."""

    def __init__(self, n, gate_x, gate_z, alpha, dtau, delta, cap_M=0, cap_policy=0,
                 max_weight=0):
        self.n = int(n)
        self.W = (self.n + 63) // 64
        gx, pgx = _u64(gate_x)
        gz, pgz = _u64(gate_z)
        al, pal = _f64(alpha)
        self._h = lib().oracle_create(self.n, int(al.shape[0]), pgx, pgz, pal,
                                      float(dtau), float(delta), int(cap_M),
                                      int(cap_policy))
        if not self._h:
            raise OracleError("oracle_create rejected its arguments")
        if max_weight:
            self._check(lib().oracle_set_max_weight(self._h, int(max_weight)))

    @classmethod
    def from_workload(cls, wl):
        return cls(wl.H.n, wl.H.gate_x, wl.H.gate_z, wl.H.alpha, wl.dtau, wl.delta,
                   wl.cap_M, wl.cap_policy)

    def close(self):
        if self._h:
            lib().oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st:
            raise OracleError(f"oracle status {st}")

    def apply_gate(self, k):
        self._check(lib().oracle_apply_gate(self._h, int(k)))

    def apply_layers(self, n_layers):
        self._check(lib().oracle_apply_layers(self._h, int(n_layers)))

    def count(self):
        return int(lib().oracle_count(self._h))

    def terms(self):
        """(x[count, W], z[count, W], c[count]) in ascending key order."""
        m = self.count()
        x = np.zeros((m, self.W), dtype=np.uint64)
        z = np.zeros((m, self.W), dtype=np.uint64)
        c = np.zeros(m)
        lib().oracle_get_terms(self._h, x.ctypes.data_as(_u64p), z.ctypes.data_as(_u64p),
                               c.ctypes.data_as(_f64p))
        return x, z, c

    def set_terms(self, x, z, c):
        x, px = _u64(x)
        z, pz = _u64(z)
        c, pc = _f64(c)
        self._check(lib().oracle_set_terms(self._h, int(c.shape[0]), px, pz, pc))

    def coeffs(self, ox, oz):
        ox, pox = _u64(ox)
        oz, poz = _u64(oz)
        m = ox.shape[0]
        out = np.zeros(m)
        lib().oracle_coeffs(self._h, pox, poz, m, out.ctypes.data_as(_f64p))
        return out

    def expect(self, obs):
        ox, pox = _u64(obs.x)
        oz, poz = _u64(obs.z)
        ow, pow_ = _f64(obs.w)
        return float(lib().oracle_expect(self._h, pox, poz, pow_, int(ow.shape[0])))


    def expect_psd(self, obs):
        """(<O>_{2 tau}, Tr[(O rho) rho] / 2^n, Tr[rho^2] / 2^n, imaginary
        residual) of the squared state, Sec. II.C."""
        ox, pox = _u64(obs.x)
        oz, poz = _u64(obs.z)
        ow, pow_ = _f64(obs.w)
        out = np.zeros(4)
        self._check(lib().oracle_expect_psd(self._h, pox, poz, pow_, int(ow.shape[0]),
                                            out.ctypes.data_as(_f64p)))
        return float(out[0]), float(out[1]), float(out[2]), float(out[3])


class FrozenAdjoint:
    """Frozen-support forward and its adjoint on top of an Oracle."""

    def __init__(self, o: "Oracle", n_layers: int):
        self.o = o
        o._check(lib().oracle_record(o._h, int(n_layers)))

    def value(self, obs, alpha=None):
        ox, pox = _u64(obs.x)
        oz, poz = _u64(obs.z)
        ow, pow_ = _f64(obs.w)
        f = ctypes.c_double()
        pa = None
        if alpha is not None:
            al, pa = _f64(alpha)
        self.o._check(lib().oracle_frozen_value(self.o._h, pa, pox, poz, pow_, int(ow.shape[0]),
                                                ctypes.byref(f)))
        return f.value

    def grad_alpha(self, obs, n_gates):
        ox, pox = _u64(obs.x)
        oz, poz = _u64(obs.z)
        ow, pow_ = _f64(obs.w)
        g = np.zeros(n_gates)
        f = ctypes.c_double()
        self.o._check(lib().oracle_adjoint(self.o._h, pox, poz, pow_, int(ow.shape[0]),
                                           g.ctypes.data_as(_f64p), ctypes.byref(f)))
        return f.value, g


def commutes(W, px, pz, qx, qz) -> bool:
    a = [_u64(v) for v in (px, pz, qx, qz)]
    return bool(lib().oracle_commutes(int(W), *[p for _, p in a]))


def pauli_product(W, qx, qz, px, pz):
    """Q*P = i^e R: returns (e, rx, rz)."""
    a = [_u64(v) for v in (qx, qz, px, pz)]
    rx = np.zeros(W, dtype=np.uint64)
    rz = np.zeros(W, dtype=np.uint64)
    e = lib().oracle_pauli_product(int(W), *[p for _, p in a], rx.ctypes.data_as(_u64p),
                                   rz.ctypes.data_as(_u64p))
    return int(e), rx, rz
