"""GB300 imaginary-time Pauli propagation: thin Python binding of the C ABI.

The functions below carry the C names of ``include/itpp.h`` and only marshal
arguments (numpy host arrays, device pointers as integers, CUDA streams as
integers); every step of the propagation runs in the sm_103a kernels of
``lib/libitpp_gb300.so``.  Importing this package without the built library
raises immediately -- there is no fallback.

``Propagator`` is a convenience wrapper holding one handle.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libitpp_gb300.so")

_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p

ITPP_OK = 0
STATUS_NAMES = {0: "ok", 1: "ERR_ARG", 2: "ERR_ALLOC", 3: "ERR_CAPACITY",
                4: "ERR_HASH_PROBE", 5: "ERR_TIMEOUT", 6: "ERR_TRACE_ZERO",
                7: "ERR_CUDA", 8: "ERR_STATE", 9: "ERR_IO"}


class itpp_params(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("cap_M", ctypes.c_uint64),
                ("cap_policy", ctypes.c_int), ("merge_path", ctypes.c_int),
                ("table_load_pct", ctypes.c_int), ("block_threads", ctypes.c_int),
                ("items_per_thread", ctypes.c_int), ("max_weight", ctypes.c_int),
                ("trotter_order", ctypes.c_int), ("partition_target", ctypes.c_int),
                ("reserved", ctypes.c_int * 2)]


class itpp_stats(ctypes.Structure):
    _fields_ = [("gates_applied", ctypes.c_uint64), ("terms_in", ctypes.c_uint64),
                ("terms_out", ctypes.c_uint64), ("peak_terms", ctypes.c_uint64),
                ("cap_events", ctypes.c_uint64), ("count", ctypes.c_uint64),
                ("table_probes", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("repartitions", ctypes.c_uint64), ("select_candidates", ctypes.c_uint64),
                ("select_range", ctypes.c_uint64), ("select_full", ctypes.c_uint64),
                ("long_partitions", ctypes.c_uint64), ("error_site", ctypes.c_uint64),
                ("merge_retries", ctypes.c_uint64)]


class ItppError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: {STATUS_NAMES.get(self.status, self.status)}")


_lib = None

# (name, restype, argtypes) of every exported function of include/itpp.h
class itpp_tune_result(ctypes.Structure):
    _fields_ = [("main_block", ctypes.c_int), ("main_grid", ctypes.c_int),
                ("insert_grid", ctypes.c_int), ("table_load_pct", ctypes.c_int),
                ("ms_per_probe", ctypes.c_double), ("ms_per_probe_default", ctypes.c_double),
                ("candidates", ctypes.c_int), ("partition_target", ctypes.c_int),
                ("reserved", ctypes.c_int * 2)]


_SIGNATURES = [
    ("itpp_create", ctypes.c_int, [ctypes.c_int, _u64p, _u64p, _f64p, ctypes.c_int,
                                   ctypes.c_double, ctypes.POINTER(itpp_params), _vp,
                                   ctypes.POINTER(_vp)]),
    ("itpp_destroy", ctypes.c_int, [_vp]),
    ("itpp_apply_trotter_layer", ctypes.c_int, [_vp, ctypes.c_int]),
    ("itpp_apply_gate", ctypes.c_int, [_vp, ctypes.c_int]),
    ("itpp_truncate", ctypes.c_int, [_vp, ctypes.c_double]),
    ("itpp_expect", ctypes.c_int, [_vp, _u64p, _u64p, _f64p, ctypes.c_int, _f64p]),
    ("itpp_expect_psd", ctypes.c_int, [_vp, _u64p, _u64p, _f64p, ctypes.c_int, _f64p]),
    ("itpp_coeffs", ctypes.c_int, [_vp, _u64p, _u64p, ctypes.c_int, _f64p]),
    ("itpp_expect_device", ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
    ("itpp_synchronize", ctypes.c_int, [_vp]),
    ("itpp_get_count", ctypes.c_int, [_vp, _u64p]),
    ("itpp_get_terms", ctypes.c_int, [_vp, _u64p, _u64p, _f64p, ctypes.c_uint64, _u64p]),
    ("itpp_set_terms", ctypes.c_int, [_vp, _u64p, _u64p, _f64p, ctypes.c_uint64]),
    ("itpp_sort_terms", ctypes.c_int, [ctypes.c_int, _u64p, _u64p, _f64p, ctypes.c_uint64]),
    ("itpp_get_terms_sorted", ctypes.c_int, [_vp, _u64p, _u64p, _f64p, ctypes.c_uint64, _u64p]),
    ("itpp_save", ctypes.c_int, [_vp, ctypes.c_char_p]),
    ("itpp_load", ctypes.c_int, [_vp, ctypes.c_char_p]),
    ("itpp_get_stats", ctypes.c_int, [_vp, ctypes.POINTER(itpp_stats)]),
    ("itpp_profile_enable", ctypes.c_int, [_vp, ctypes.c_int]),
    ("itpp_profile_read", ctypes.c_int, [_vp, ctypes.c_int, _u64p, _f64p]),
    ("itpp_set_alpha", ctypes.c_int, [_vp, _f64p]),
    ("itpp_reset", ctypes.c_int, [_vp]),
    ("itpp_adjoint", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _u64p, _u64p, _f64p,
                                    ctypes.c_int, _f64p, _f64p]),
    ("itpp_frozen_value", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _f64p, _u64p, _u64p,
                                         _f64p, ctypes.c_int, _f64p]),
    ("itpp_batch_create", ctypes.c_int, [ctypes.c_int, _i32p, _i32p, _u64p, _u64p, _f64p,
                                         ctypes.c_double, ctypes.POINTER(itpp_params), _vp,
                                         ctypes.POINTER(_vp)]),
    ("itpp_batch_destroy", ctypes.c_int, [_vp]),
    ("itpp_batch_apply_trotter_layer", ctypes.c_int, [_vp, ctypes.c_int]),
    ("itpp_batch_synchronize", ctypes.c_int, [_vp]),
    ("itpp_batch_autotune", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(itpp_tune_result)]),
    ("itpp_batch_get_counts", ctypes.c_int, [_vp, _u64p, _i32p]),
    ("itpp_batch_get_stats", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(itpp_stats)]),
    ("itpp_batch_get_terms", ctypes.c_int, [_vp, ctypes.c_int, _u64p, _u64p, _f64p,
                                            ctypes.c_uint64, _u64p]),
    ("itpp_batch_expect", ctypes.c_int, [_vp, ctypes.c_int, _u64p, _u64p, _f64p, ctypes.c_int,
                                         _f64p]),
    ("itpp_gate_apply_noalloc", ctypes.c_int, [ctypes.c_int, _u64p, _u64p, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, _vp, _vp,
                                               ctypes.c_uint64, _vp, _vp, ctypes.c_uint64, _vp,
                                               _vp, _vp]),
    ("itpp_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("itpp_version", ctypes.c_char_p, []),
]


def exported_names():
    return [s[0] for s in _SIGNATURES]


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                              "(the CUDA extension is required; there is no fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def itpp_gate_apply_noalloc(n, gate_x, gate_z, alpha, dtau, delta, d_keys_in, d_coef_in,
                            n_in, d_keys_out, d_coef_out, out_capacity, d_n_out,
                            d_trace_out=None, stream=None):
    """One gate on caller-owned device buffers (integers: device addresses),
    with no device allocation; see include/itpp.h."""
    gx, pgx = _u64(gate_x)
    gz, pgz = _u64(gate_z)
    st = lib().itpp_gate_apply_noalloc(int(n), pgx, pgz, float(alpha), float(dtau),
                                       float(delta), d_keys_in, d_coef_in, int(n_in),
                                       d_keys_out, d_coef_out, int(out_capacity), d_n_out,
                                       d_trace_out, _stream_ptr(stream))
    _check(st, "itpp_gate_apply_noalloc")


def sort_terms(x, z, c):
    """Copies of host arrays (x[count, W], z[count, W], c[count]) sorted into
    the canonical order by itpp_sort_terms."""
    x = np.array(x, dtype=np.uint64, order="C", copy=True)
    z = np.array(z, dtype=np.uint64, order="C", copy=True)
    c = np.array(c, dtype=np.float64, order="C", copy=True)
    W = x.shape[1] if x.ndim == 2 else 1
    _check(lib().itpp_sort_terms(W, x.ctypes.data_as(_u64p), z.ctypes.data_as(_u64p),
                                 c.ctypes.data_as(_f64p), int(c.shape[0])), "itpp_sort_terms")
    return x, z, c


def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(_u64p)


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_f64p)


def _check(st, where):
    if st != ITPP_OK:
        raise ItppError(st, where)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)   # torch.cuda.Stream


class Propagator:
    """One ITPP propagation on the current CUDA device (C handle owner)."""

    def __init__(self, n, gate_x, gate_z, alpha, dtau, delta, cap_M, cap_policy=0,
                 merge_path=0, stream=None, table_load_pct=0, block_threads=0,
                 items_per_thread=0, max_weight=0, trotter_order=1, partition_target=0):
        self.n = int(n)
        self.W = (self.n + 63) // 64
        gx, pgx = _u64(gate_x)
        gz, pgz = _u64(gate_z)
        al, pal = _f64(alpha)
        self.n_gates = int(al.shape[0])
        p = itpp_params()
        p.delta = float(delta)
        p.cap_M = int(cap_M)
        p.cap_policy = int(cap_policy)
        p.merge_path = int(merge_path)
        p.table_load_pct = int(table_load_pct)
        p.block_threads = int(block_threads)
        p.items_per_thread = int(items_per_thread)
        p.max_weight = int(max_weight)
        p.trotter_order = int(trotter_order)
        p.partition_target = int(partition_target)
        h = _vp()
        st = lib().itpp_create(self.n, pgx, pgz, pal, self.n_gates, float(dtau),
                               ctypes.byref(p), _stream_ptr(stream), ctypes.byref(h))
        _check(st, "itpp_create")
        self._h = h

    @classmethod
    def from_workload(cls, wl, **kw):
        return cls(wl.H.n, wl.H.gate_x, wl.H.gate_z, wl.H.alpha, wl.dtau, wl.delta,
                   wl.cap_M, wl.cap_policy, **kw)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().itpp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def apply_trotter_layer(self, n_layers=1):
        _check(lib().itpp_apply_trotter_layer(self._h, int(n_layers)), "itpp_apply_trotter_layer")

    def apply_gate(self, k):
        _check(lib().itpp_apply_gate(self._h, int(k)), "itpp_apply_gate")

    def truncate(self, delta):
        _check(lib().itpp_truncate(self._h, float(delta)), "itpp_truncate")

    def synchronize(self):
        _check(lib().itpp_synchronize(self._h), "itpp_synchronize")

    def count(self):
        c = ctypes.c_uint64()
        _check(lib().itpp_get_count(self._h, ctypes.byref(c)), "itpp_get_count")
        return int(c.value)

    def terms(self):
        """(x[count, W], z[count, W], c[count]), order unspecified."""
        n = self.count()
        x = np.zeros((n, self.W), dtype=np.uint64)
        z = np.zeros((n, self.W), dtype=np.uint64)
        c = np.zeros(n)
        got = ctypes.c_uint64()
        _check(lib().itpp_get_terms(self._h, x.ctypes.data_as(_u64p), z.ctypes.data_as(_u64p),
                                    c.ctypes.data_as(_f64p), n, ctypes.byref(got)),
               "itpp_get_terms")
        return x, z, c

    def sorted_terms(self):
        """Terms in the canonical order (ascending: x words, then z words),
        from itpp_get_terms_sorted."""
        n = self.count()
        x = np.zeros((n, self.W), dtype=np.uint64)
        z = np.zeros((n, self.W), dtype=np.uint64)
        c = np.zeros(n)
        got = ctypes.c_uint64()
        _check(lib().itpp_get_terms_sorted(self._h, x.ctypes.data_as(_u64p),
                                           z.ctypes.data_as(_u64p), c.ctypes.data_as(_f64p),
                                           n, ctypes.byref(got)), "itpp_get_terms_sorted")
        return x, z, c

    def save(self, path):
        """Checkpoint the state to a file (see itpp_save)."""
        _check(lib().itpp_save(self._h, os.fsencode(path)), "itpp_save")

    def load(self, path):
        """Replace the state by a checkpoint written by save (see itpp_load)."""
        _check(lib().itpp_load(self._h, os.fsencode(path)), "itpp_load")

    def set_terms(self, x, z, c):
        x, px = _u64(x)
        z, pz = _u64(z)
        c, pc = _f64(c)
        _check(lib().itpp_set_terms(self._h, px, pz, pc, int(c.shape[0])), "itpp_set_terms")

    def expect(self, obs):
        ox, pox = _u64(obs.x)
        oz, poz = _u64(obs.z)
        ow, pow_ = _f64(obs.w)
        out = ctypes.c_double()
        _check(lib().itpp_expect(self._h, pox, poz, pow_, int(ow.shape[0]), ctypes.byref(out)),
               "itpp_expect")
        return float(out.value)

    def expect_psd(self, obs):
        """(<O>_{2 tau}, Tr[(O rho) rho] / 2^n, Tr[rho^2] / 2^n) of the squared
        state (Sec. II.C); see include/itpp.h."""
        ox, pox = _u64(obs.x)
        oz, poz = _u64(obs.z)
        ow, pow_ = _f64(obs.w)
        out = np.zeros(3)
        _check(lib().itpp_expect_psd(self._h, pox, poz, pow_, int(ow.shape[0]),
                                     out.ctypes.data_as(_f64p)), "itpp_expect_psd")
        return float(out[0]), float(out[1]), float(out[2])

    def coeffs(self, ox, oz):
        ox, pox = _u64(ox)
        oz, poz = _u64(oz)
        m = ox.shape[0]
        out = np.zeros(m)
        _check(lib().itpp_coeffs(self._h, pox, poz, m, out.ctypes.data_as(_f64p)), "itpp_coeffs")
        return out

    def stats(self, check=True):
        """Device counters; with check=False the counters are returned even
        when the handle holds an error (then "status" names it)."""
        s = itpp_stats()
        st = lib().itpp_get_stats(self._h, ctypes.byref(s))
        if check:
            _check(st, "itpp_get_stats")
        d = {k: int(getattr(s, k)) for k, _ in itpp_stats._fields_}
        d["status"] = int(st)
        return d

    def reset(self):
        _check(lib().itpp_reset(self._h), "itpp_reset")

    def set_alpha(self, alpha):
        al, pal = _f64(alpha)
        _check(lib().itpp_set_alpha(self._h, pal), "itpp_set_alpha")

    def adjoint(self, n_layers, obs, ckpt_every=10):
        """(f, df/dalpha) for f = sum_j w_j c_{P_j} after n_layers layers
        from the identity, support frozen; see include/itpp.h."""
        ox, pox = _u64(obs.x)
        oz, poz = _u64(obs.z)
        ow, pow_ = _f64(obs.w)
        g = np.zeros(self.n_gates)
        f = ctypes.c_double()
        _check(lib().itpp_adjoint(self._h, int(n_layers), int(ckpt_every), pox, poz, pow_,
                                  int(ow.shape[0]), g.ctypes.data_as(_f64p), ctypes.byref(f)),
               "itpp_adjoint")
        return f.value, g

    def frozen_value(self, n_layers, obs, alpha_eval, ckpt_every=10):
        """f = sum_j w_j c_{P_j} of the frozen-support forward (the support of
        this handle's coefficients) evaluated at alpha_eval; see include/itpp.h."""
        ox, pox = _u64(obs.x)
        oz, poz = _u64(obs.z)
        ow, pow_ = _f64(obs.w)
        al, pal = _f64(np.asarray(alpha_eval, dtype=np.float64))
        f = ctypes.c_double()
        _check(lib().itpp_frozen_value(self._h, int(n_layers), int(ckpt_every), pal, pox, poz,
                                       pow_, int(ow.shape[0]), ctypes.byref(f)),
               "itpp_frozen_value")
        return f.value

    def profile_enable(self, on=True):
        _check(lib().itpp_profile_enable(self._h, 1 if on else 0), "itpp_profile_enable")

    def profile_read(self, kid):
        n = ctypes.c_uint64()
        ms = ctypes.c_double()
        _check(lib().itpp_profile_read(self._h, int(kid), ctypes.byref(n), ctypes.byref(ms)),
               "itpp_profile_read")
        return int(n.value), float(ms.value)


class BatchPropagator:
    """B independent ITPP propagations advanced in shared launches."""

    def __init__(self, hams, dtau, delta, cap_M, cap_policy=0, stream=None, table_load_pct=0,
                 max_weight=0, merge_path=0, partition_target=0):
        self.B = len(hams)
        self.ns = [int(H.n) for H in hams]
        self.W = (max(self.ns) + 63) // 64
        W = self.W
        gx = np.concatenate([_pad_words(H.gate_x, W) for H in hams])
        gz = np.concatenate([_pad_words(H.gate_z, W) for H in hams])
        al = np.concatenate([np.asarray(H.alpha, dtype=np.float64) for H in hams])
        n = np.asarray(self.ns, dtype=np.int32)
        ng = np.asarray([H.n_gates for H in hams], dtype=np.int32)
        gx, pgx = _u64(gx)
        gz, pgz = _u64(gz)
        al, pal = _f64(al)
        p = itpp_params()
        p.delta = float(delta)
        p.cap_M = int(cap_M)
        p.cap_policy = int(cap_policy)
        p.table_load_pct = int(table_load_pct)
        p.max_weight = int(max_weight)
        p.merge_path = int(merge_path)
        p.partition_target = int(partition_target)
        h = _vp()
        st = lib().itpp_batch_create(self.B, n.ctypes.data_as(_i32p), ng.ctypes.data_as(_i32p),
                                     pgx, pgz, pal, float(dtau), ctypes.byref(p),
                                     _stream_ptr(stream), ctypes.byref(h))
        _check(st, "itpp_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().itpp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, probe_layers=2):
        """Time launch shapes (and partition sizes or table loads) on this
        batch, keep the fastest (every instance is reset to the identity).
        Returns the choice."""
        r = itpp_tune_result()
        _check(lib().itpp_batch_autotune(self._h, int(probe_layers), ctypes.byref(r)),
               "itpp_batch_autotune")
        return {k: getattr(r, k) for k, _ in itpp_tune_result._fields_ if k != "reserved"}

    def apply_trotter_layer(self, n_layers=1):
        _check(lib().itpp_batch_apply_trotter_layer(self._h, int(n_layers)),
               "itpp_batch_apply_trotter_layer")

    def synchronize(self):
        _check(lib().itpp_batch_synchronize(self._h), "itpp_batch_synchronize")

    def counts(self):
        c = np.zeros(self.B, dtype=np.uint64)
        s = np.zeros(self.B, dtype=np.int32)
        lib().itpp_batch_get_counts(self._h, c.ctypes.data_as(_u64p), s.ctypes.data_as(_i32p))
        return c.astype(np.int64), s

    def stats(self, b):
        s = itpp_stats()
        _check(lib().itpp_batch_get_stats(self._h, int(b), ctypes.byref(s)), "itpp_batch_get_stats")
        return {k: int(getattr(s, k)) for k, _ in itpp_stats._fields_}

    def terms(self, b):
        got = ctypes.c_uint64()
        c_all, _ = self.counts()
        n = int(c_all[b])
        x = np.zeros((n, self.W), dtype=np.uint64)
        z = np.zeros((n, self.W), dtype=np.uint64)
        c = np.zeros(n)
        _check(lib().itpp_batch_get_terms(self._h, int(b), x.ctypes.data_as(_u64p),
                                          z.ctypes.data_as(_u64p), c.ctypes.data_as(_f64p), n,
                                          ctypes.byref(got)), "itpp_batch_get_terms")
        return x, z, c

    def expect(self, b, obs):
        ox, pox = _u64(_pad_words(obs.x, self.W))
        oz, poz = _u64(_pad_words(obs.z, self.W))
        ow, pow_ = _f64(obs.w)
        out = ctypes.c_double()
        _check(lib().itpp_batch_expect(self._h, int(b), pox, poz, pow_, int(ow.shape[0]),
                                       ctypes.byref(out)), "itpp_batch_expect")
        return float(out.value)


def _pad_words(a, W):
    a = np.asarray(a, dtype=np.uint64)
    if a.shape[1] == W:
        return a
    out = np.zeros((a.shape[0], W), dtype=np.uint64)
    out[:, :a.shape[1]] = a
    return out
