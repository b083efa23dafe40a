"""itpp_gate_apply_noalloc: one gate for callers that cannot allocate.

Callers running inside a memory pool that owns the whole device, or on a host
path that must not pay cudaMalloc's implicit synchronisation, can apply a
gate to their own buffers through this entry point; its scratch is a static
device array inside the library.  These checks call it through the C ABI
twice in a row (the second call reads the first call's output, so the shared
scratch is reused) and compare each result with the CPU oracle applying the
same gate to the same input, and with the allocating entry point
(itpp_apply_gate + itpp_get_terms): string sets equal, coefficients equal in
every bit, the bar of the other parity tests.  The returned trace is the
identity's merged coefficient before the rescaling, checked bit for bit
against the propagation rule on the oracle's input (the identity's own child
cosh(theta) plus its partner Q's child c_Q (-sinh(theta))).  Around a call
after the first, neither the device's free memory nor the caching
allocator's usage may change.  The file sorts last so a failure here stops a
-x run only after every other test has run.
"""
import ctypes
import glob
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
import workloads as wl
from tests._compare import assert_same_state

pytestmark = pytest.mark.gpu

itpp = pytest.importorskip("paper_2601_14400_gb300")
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def itpp_max(W):
    return 262144 if W == 1 else 131072


def _to_device_keys(x, z):
    """(count, W) x and z planes -> device AoS keys: x[0..W-1], z[0..W-1]."""
    keys = np.ascontiguousarray(np.concatenate([x, z], axis=1))
    return torch.from_numpy(keys.view(np.int64)).cuda()


def _from_device(d_keys, d_coef, count, W):
    k = d_keys[:count].cpu().numpy().view(np.uint64).reshape(count, 2 * W)
    return k[:, :W].copy(), k[:, W:].copy(), d_coef[:count].cpu().numpy().copy()


def _sorted(p):
    from tests._compare import sort_terms
    return sort_terms(*p.terms())


def _expected_trace(o, H, k, dtau):
    """c_I after gate k before rescaling: cosh(theta) * 1 + c_Q * (-sinh(theta))
    (Q Q = +I, so the sign is +1), theta = alpha_k dtau, on the oracle's input."""
    theta = H.alpha[k] * dtau
    c_q = float(o.coeffs(H.gate_x[k][None], H.gate_z[k][None])[0])
    return 1.0 * math.cosh(theta) + c_q * (-math.sinh(theta))


class _Call:
    """Output buffers of one call, allocated before it (the call allocates nothing)."""

    def __init__(self, cap, W):
        self.keys = torch.zeros((cap, 2 * W), dtype=torch.int64, device="cuda")
        self.coef = torch.zeros(cap, dtype=torch.float64, device="cuda")
        self.n = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.tr = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.cap = cap


@pytest.mark.parametrize("n,layers,gates,delta", [(10, 2, (3, 12), 1e-6),
                                                  (70, 1, (5, 80), 1e-3)])
def test_noalloc_two_calls_match_oracle_and_allocating_path(n, layers, gates, delta):
    torch.cuda.set_device(0)
    H = wl.tfim_1d(n, 1.0, 0.9, periodic=True)
    W = H.W
    dtau = 0.1
    ref = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta, 1 << 18)
    ref.apply_trotter_layer(layers)
    o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta)
    x, z, c = ref.terms()
    o.set_terms(x, z, c)
    d_keys = _to_device_keys(x, z)
    d_coef = torch.from_numpy(c).cuda()
    count = c.shape[0]
    assert count <= itpp_max(W)
    stream = torch.cuda.current_stream()
    for call, k in enumerate(gates):
        out = _Call(2 * count, W)
        want_tr = _expected_trace(o, H, k, dtau)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        used0 = torch.cuda.memory_allocated()
        itpp.itpp_gate_apply_noalloc(n, H.gate_x[k], H.gate_z[k], H.alpha[k], dtau, delta,
                                     d_keys.data_ptr(), d_coef.data_ptr(), count,
                                     out.keys.data_ptr(), out.coef.data_ptr(), out.cap,
                                     out.n.data_ptr(), out.tr.data_ptr(), stream)
        torch.cuda.synchronize()
        if call > 0:   # the first call may load the module and set the scratch aside
            assert torch.cuda.mem_get_info()[0] == free0, "device memory changed"
            assert torch.cuda.memory_allocated() == used0, "caching allocator grew"
        got_n = int(out.n.item())
        assert 0 < got_n <= out.cap
        got = _from_device(out.keys, out.coef, got_n, W)
        o.apply_gate(k)
        assert_same_state(got, o.terms(), f"gate {k} vs oracle")
        ref.apply_gate(k)
        assert_same_state(got, _sorted(ref), f"gate {k} vs allocating path")
        got_tr = float(out.tr.item())
        assert np.float64(got_tr).view(np.uint64) == np.float64(want_tr).view(np.uint64), \
            (got_tr, want_tr)
        d_keys, d_coef, count = out.keys, out.coef, got_n
    ref.close()
    o.close()


def test_noalloc_input_without_identity_is_reported():
    torch.cuda.set_device(0)
    H = wl.tfim_1d(8, 1.0, 1.0)
    X, Z, C = wl.synthetic_state(8, 500, 17, delta=1e-6)
    keep = ~((X[:, 0] == 0) & (Z[:, 0] == 0))         # drop the identity
    X, Z, C = X[keep], Z[keep], C[keep]
    d_keys, d_coef = _to_device_keys(X, Z), torch.from_numpy(C).cuda()
    out = _Call(2 * C.shape[0], 1)
    itpp.itpp_gate_apply_noalloc(8, H.gate_x[0], H.gate_z[0], H.alpha[0], 0.1, 1e-6,
                                 d_keys.data_ptr(), d_coef.data_ptr(), C.shape[0],
                                 out.keys.data_ptr(), out.coef.data_ptr(), out.cap,
                                 out.n.data_ptr(), out.tr.data_ptr(),
                                 torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert np.int64(out.n.item()).view(np.uint64) == np.uint64(2**64 - 1)
    assert math.isnan(float(out.tr.item()))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch.cuda.set_device(0)
    H = wl.tfim_1d(8, 1.0, 1.0)
    n_big = int(itpp_max(1)) + 1
    buf = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(itpp.ItppError) as e:
        itpp.itpp_gate_apply_noalloc(8, H.gate_x[0], H.gate_z[0], H.alpha[0], 0.1, 1e-6,
                                     buf.data_ptr(), buf.data_ptr(), n_big, buf.data_ptr(),
                                     buf.data_ptr(), 2 * n_big, buf.data_ptr(), None, None)
    assert e.value.status == 3
    with pytest.raises(itpp.ItppError) as e:      # output room below 2 * n_in
        itpp.itpp_gate_apply_noalloc(8, H.gate_x[0], H.gate_z[0], H.alpha[0], 0.1, 1e-6,
                                     buf.data_ptr(), buf.data_ptr(), 4, buf.data_ptr(),
                                     buf.data_ptr(), 7, buf.data_ptr(), None, None)
    assert e.value.status == 3


def _harness(tmp_path):
    """The entry point built with a generation hook, from the library's objects."""
    from paper_2601_14400_gb300 import _build
    objs = [p for p in sorted(glob.glob(os.path.join(_build.LIBDIR, "obj", "*.o")))
            if not os.path.basename(p).startswith("itpp_noalloc")]
    assert objs, "library objects missing (build first)"
    so = str(tmp_path / "libnoalloc_harness.so")
    cmd = [_build.nvcc()] + _build.ARCH + list(_build.NVCC_FLAGS) + [
        "-shared", os.path.join(ROOT, "tests", "noalloc_gen_harness.cu")] + objs + ["-o", so]
    subprocess.run(cmd, check=True, capture_output=True)
    L = ctypes.CDLL(so)
    L.itpp_test_noalloc_set_generation.argtypes = [ctypes.c_uint]
    L.itpp_gate_apply_noalloc.argtypes = [
        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
        ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
        ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return L


def test_noalloc_generation_wrap_clears_the_table(tmp_path):
    """Call 1 leaves slots tagged with generation 1; the counter is then set
    to 2^32 - 1, so call 2 wraps.  Call 2 applies the same gate to the same
    strings with other coefficients: a slot of call 1 taken for live would
    hand it call 1's partner coefficients."""
    torch.cuda.set_device(0)
    L = _harness(tmp_path)
    H = wl.tfim_1d(10, 1.0, 0.8, periodic=True)
    dtau, delta, k = 0.1, 1e-6, 4
    ref = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta, 1 << 18)
    ref.apply_trotter_layer(2)
    x, z, c = ref.terms()
    ref.close()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(coef):
        o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta)
        o.set_terms(x, z, coef)
        out = _Call(2 * coef.shape[0], 1)
        d_keys, d_coef = _to_device_keys(x, z), torch.from_numpy(coef).cuda()
        gx = np.ascontiguousarray(H.gate_x[k], dtype=np.uint64)
        gz = np.ascontiguousarray(H.gate_z[k], dtype=np.uint64)
        st = L.itpp_gate_apply_noalloc(
            H.n, gx.ctypes.data, gz.ctypes.data, float(H.alpha[k]), dtau, delta,
            d_keys.data_ptr(), d_coef.data_ptr(), coef.shape[0], out.keys.data_ptr(),
            out.coef.data_ptr(), out.cap, out.n.data_ptr(), out.tr.data_ptr(), stream)
        assert st == 0
        torch.cuda.synchronize()
        got_n = int(out.n.item())
        assert 0 < got_n <= out.cap
        o.apply_gate(k)
        assert_same_state(_from_device(out.keys, out.coef, got_n, 1), o.terms(), "wrap")
        o.close()

    assert L.itpp_test_noalloc_set_generation(0) == 0
    call(c)
    assert L.itpp_test_noalloc_set_generation(0xFFFFFFFF) == 0
    c2 = c * 0.5
    c2[(x[:, 0] == 0) & (z[:, 0] == 0)] = 1.0
    call(c2)
