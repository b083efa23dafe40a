"""GPU adjoint (frozen-support gradients) vs the oracle's adjoint.

The oracle's adjoint is pinned on the CPU against central differences of the
frozen forward, the dense Trotter derivative and the exact thermal
derivative; here the GPU sweep must match it to 1e-10 of the largest
gradient component (the reductions run in a different order).
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

itpp = pytest.importorskip("paper_2601_14400_gb300")
torch = pytest.importorskip("torch")


def _both(H, dtau, delta, layers, obs, ckpt):
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta, 1 << 20)
    f_g, grad_g = g.adjoint(layers, obs, ckpt_every=ckpt)
    o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta)
    f_o, grad_o = oracle.FrozenAdjoint(o, layers).grad_alpha(obs, H.n_gates)
    return g, (f_g, grad_g), (f_o, grad_o)


def _close(a, b, tol=1e-10):
    scale = max(np.max(np.abs(b)), 1e-300)
    assert np.max(np.abs(a - b)) <= tol * scale, (np.max(np.abs(a - b)), scale)


@pytest.mark.parametrize("obs_kind", ["zz", "energy"])
def test_adjoint_n10_subcase_matches_oracle(obs_kind):
    H = wl.adjoint_chain(10)
    O = (wl.zz_observables(10, [(4, 5)])[0] if obs_kind == "zz"
         else wl.energy_observable(H))
    g, (f_g, d_g), (f_o, d_o) = _both(H, 0.02, 1e-6, 5, O, ckpt=2)
    assert abs(f_g - f_o) <= 1e-12 * max(1.0, abs(f_o))
    _close(d_g, d_o)


@pytest.mark.parametrize("M", [500, 3000])
def test_adjoint_with_top_m_bound_matches_oracle(M):
    # frozen support = the kept top-M set of every step
    H = wl.adjoint_chain(10)
    O = wl.energy_observable(H)
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.05, 1e-9, M, 1)
    f_g, d_g = g.adjoint(4, O, ckpt_every=2)
    assert g.stats()["cap_events"] > 0
    o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, 0.05, 1e-9, M, 1)
    f_o, d_o = oracle.FrozenAdjoint(o, 4).grad_alpha(O, H.n_gates)
    assert abs(f_g - f_o) <= 1e-12 * max(1.0, abs(f_o))
    _close(d_g, d_o)


def test_adjoint_checkpoint_interval_does_not_change_the_gradient():
    H = wl.tfim_1d(8, 1.0, 0.8, periodic=True)
    O = wl.zz_observables(8, [(0, 1)])[0]
    grads = []
    for ck in (1, 2, 5):
        g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.05, 1e-6, 1 << 18)
        grads.append(g.adjoint(5, O, ckpt_every=ck)[1])
    _close(grads[1], grads[0], 1e-13)
    _close(grads[2], grads[0], 1e-13)


def test_adjoint_two_words_matches_oracle():
    H = wl.random_pauli_hamiltonian(70, 14, 9, max_weight=3)
    O = wl.Observable(70, H.gate_x[:3].copy(), H.gate_z[:3].copy(), np.array([0.7, -1.1, 0.4]))
    g, (f_g, d_g), (f_o, d_o) = _both(H, 0.1, 1e-4, 3, O, ckpt=1)
    _close(d_g, d_o)


def test_adjoint_leaves_the_forward_state():
    H = wl.tfim_1d(6, 1.0, 1.0)
    O = wl.energy_observable(H)
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.05, 1e-8, 1 << 16)
    f, _ = g.adjoint(4, O, ckpt_every=2)
    o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, 0.05, 1e-8)
    o.apply_layers(4)
    from tests._compare import assert_same_state
    assert_same_state(g.terms(), o.terms(), "after adjoint")
    assert abs(f - o.expect(O)) <= 1e-12 * abs(o.expect(O))


def test_autograd_energy_gradient_wrt_fields_and_couplings():
    from paper_2601_14400_gb300.autograd import thermal_coefficients
    n, dtau, layers = 8, 0.05, 6
    Jv = torch.tensor(np.linspace(0.9, 1.1, n - 1), dtype=torch.float64, requires_grad=True)
    hv = torch.tensor(np.linspace(0.8, 1.2, n), dtype=torch.float64, requires_grad=True)
    H = wl.tfim_1d(n, Jv.detach().numpy(), hv.detach().numpy())
    prop = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, dtau, 1e-9, 1 << 18)
    alpha = torch.cat([-Jv, -hv])                      # Trotter order: bonds, then fields
    c = thermal_coefficients(alpha, prop, layers, H.gate_x, H.gate_z, ckpt_every=3)
    energy = (alpha * c).sum()                          # <H> = sum_k alpha_k c_{Q_k}
    energy.backward()
    # oracle: explicit term + frozen adjoint, chain rule d alpha / d(J, h) = -1
    o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, dtau, 1e-9)
    f_o, g_o = oracle.FrozenAdjoint(o, layers).grad_alpha(wl.energy_observable(H), H.n_gates)
    c_o = o.coeffs(H.gate_x, H.gate_z)
    d_alpha = c_o + g_o
    want_J, want_h = -d_alpha[:n - 1], -d_alpha[n - 1:]
    assert abs(float(energy) - f_o) <= 1e-12 * abs(f_o)
    _close(Jv.grad.numpy(), want_J)
    _close(hv.grad.numpy(), want_h)


@pytest.mark.parametrize("obs_kind", ["energy", "zz"])
def test_adjoint_cfg5_size_prefix_matches_oracle(obs_kind):
    """The gradient workload at its own size (n = 32, 63 parameters, per-site
    fields and couplings from its seed, dtau = 0.02, |c| <= 1e-7 dropped) on a
    two-layer prefix with at most 2^14 terms (top-M, the frozen support of a
    step is its kept set): GPU adjoint against the oracle's, 1e-10 of the
    largest component, for d<H>/d alpha and d<Z15 Z16>/d alpha."""
    w = wl.WORKLOADS["adjoint_n32"]
    H = w.H
    O = w.observables["energy"] if obs_kind == "energy" else w.observables["Z15Z16"]
    M, layers = 1 << 14, 2
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, w.dtau, w.delta, M, 1)
    f_g, d_g = g.adjoint(layers, O, ckpt_every=1)
    assert g.stats()["cap_events"] > 0
    o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, w.dtau, w.delta, M, 1)
    f_o, d_o = oracle.FrozenAdjoint(o, layers).grad_alpha(O, H.n_gates)
    assert abs(f_g - f_o) <= 1e-12 * max(1.0, abs(f_o))
    assert H.n_gates == 63
    _close(d_g, d_o)


def test_frozen_value_at_alpha_is_the_forward_value():
    H = wl.adjoint_chain(10)
    O = wl.energy_observable(H)
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.05, 1e-6, 1 << 12, 1)
    f_adj, _ = g.adjoint(4, O, ckpt_every=2)
    f_frz = g.frozen_value(4, O, H.alpha, ckpt_every=2)
    assert abs(f_frz - f_adj) <= 1e-12 * abs(f_adj)
    o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, 0.05, 1e-6, 1 << 12, 1)
    fa = oracle.FrozenAdjoint(o, 4)
    a = H.alpha.copy()
    a[3] += 0.01
    assert abs(g.frozen_value(4, O, a, ckpt_every=2) - fa.value(O, a)) <= 1e-11 * abs(f_adj)


@pytest.mark.parametrize("obs_kind", ["energy", "zz"])
def test_adjoint_cfg5_full_size_central_differences(obs_kind):
    """The gradient workload in full (n = 32, 63 parameters, 50 layers,
    snapshots every 10 layers, |c| <= 1e-7 dropped, at most 2^20 terms):
    the adjoint gradient of <H> (without its explicit term) and of
    <Z15 Z16> against central differences (step 1e-5) of the frozen-support
    forward at six parameters, 1e-7 relative to the largest component."""
    w = wl.WORKLOADS["adjoint_n32"]
    H = w.H
    O = w.observables["energy"] if obs_kind == "energy" else w.observables["Z15Z16"]
    g = itpp.Propagator.from_workload(w)
    f, grad = g.adjoint(w.n_layers, O, ckpt_every=10)
    eps = 1e-5
    scale = np.max(np.abs(grad))
    for k in (0, 15, 30, 31, 47, 62):
        vals = []
        for sgn in (1, -1):
            a = H.alpha.copy()
            a[k] += sgn * eps
            vals.append(g.frozen_value(w.n_layers, O, a, ckpt_every=10))
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - grad[k]) <= 1e-7 * scale, (k, fd, grad[k], scale)
