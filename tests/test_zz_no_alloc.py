"""itpp_gate_apply_noalloc: one gate for callers that cannot allocate.

Callers running inside a memory pool that owns the whole device, or on a host
path that must not pay cudaMalloc's implicit synchronisation, can apply a
gate to their own buffers through this entry point; its scratch is a static
device array inside the library.  These checks call it through the C ABI
twice in a row (the second call reads the first call's output, so the shared
scratch is reused) and compare each result with the allocating entry point
(itpp_apply_gate + itpp_get_terms): string sets equal, coefficients equal in
every bit, the bar of the other parity tests.  The file sorts last so a
failure here stops a -x run only after every other test has run.
"""
import numpy as np
import pytest

import workloads as wl
from tests._compare import assert_same_state

pytestmark = pytest.mark.gpu

itpp = pytest.importorskip("paper_2601_14400_gb300")
torch = pytest.importorskip("torch")


def _to_device_keys(x, z):
    """(count, W) x and z planes -> device AoS keys: x[0..W-1], z[0..W-1]."""
    keys = np.ascontiguousarray(np.concatenate([x, z], axis=1))
    return torch.from_numpy(keys.view(np.int64)).cuda()


def _from_device(d_keys, d_coef, count, W):
    k = d_keys[:count].cpu().numpy().view(np.uint64).reshape(count, 2 * W)
    return k[:, :W].copy(), k[:, W:].copy(), d_coef[:count].cpu().numpy().copy()


@pytest.mark.parametrize("n,layers,gates,delta", [(10, 2, (3, 12), 1e-6),
                                                  (70, 1, (5, 80), 1e-3)])
def test_noalloc_two_calls_match_allocating_path(n, layers, gates, delta):
    torch.cuda.set_device(0)
    H = wl.tfim_1d(n, 1.0, 0.9, periodic=True)
    W = H.W
    dtau = 0.1
    ref = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta, 1 << 18)
    ref.apply_trotter_layer(layers)
    x, z, c = ref.terms()
    d_keys = _to_device_keys(x, z)
    d_coef = torch.from_numpy(c).cuda()
    count = c.shape[0]
    assert count <= itpp_max(W)
    stream = torch.cuda.current_stream()
    for k in gates:
        cap = 2 * count
        out_keys = torch.zeros((cap, 2 * W), dtype=torch.int64, device="cuda")
        out_coef = torch.zeros(cap, dtype=torch.float64, device="cuda")
        d_n = torch.zeros(1, dtype=torch.int64, device="cuda")
        d_tr = torch.zeros(1, dtype=torch.float64, device="cuda")
        itpp.itpp_gate_apply_noalloc(
            n, H.gate_x[k], H.gate_z[k], H.alpha[k], dtau, delta,
            d_keys.data_ptr(), d_coef.data_ptr(), count, out_keys.data_ptr(),
            out_coef.data_ptr(), cap, d_n.data_ptr(), d_tr.data_ptr(), stream)
        torch.cuda.synchronize()
        got_n = int(d_n.item())
        assert 0 < got_n <= cap
        ref.apply_gate(k)
        assert_same_state(_from_device(out_keys, out_coef, got_n, W), _sorted(ref), f"gate {k}")
        assert float(d_tr.item()) > 0.0
        d_keys, d_coef, count = out_keys, out_coef, got_n
    ref.close()


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


def itpp_max(W):
    return 262144 if W == 1 else 131072


def _sorted(p):
    from tests._compare import sort_terms
    return sort_terms(*p.terms())
