"""PSD-restored observable <O>_{2 tau} (Sec. II.C) on the GPU against the oracle.

The oracle expands O rho in the Pauli basis and overlaps it with rho, as the
paper describes (pinned against dense matrices and a closed form); the GPU
sums only the commuting pairs through a hash table of the state.  The two
agree to 1e-10 relative; the state and the following gates are unchanged.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from tests._compare import assert_same_state

pytestmark = pytest.mark.gpu

itpp = pytest.importorskip("paper_2601_14400_gb300")


def _close(a, b, tol=1e-10):
    assert abs(a - b) <= tol * max(1.0, abs(b)), (a, b)


@pytest.mark.parametrize("merge_path", [0, 1, 2])
def test_psd_observables_match_oracle(merge_path):
    H = wl.tfim_1d(10, 1.0, 0.9, periodic=True)      # at most C(20,10) terms
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.1, 1e-6, 1 << 18,
                        merge_path=merge_path)
    o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, 0.1, 1e-6, 1 << 18)
    g.apply_trotter_layer(3)
    o.apply_layers(3)
    for O in (wl.energy_observable(H), wl.zz_observables(10, [(0, 1), (3, 7)])[1],
              wl.x_observables(10)[5]):
        v, num, pur = g.expect_psd(O)
        ov, onum, opur, oimag = o.expect_psd(O)
        _close(v, ov)
        _close(num, onum)
        _close(pur, opur)
    # the state is untouched and later gates still match
    g.apply_trotter_layer(1)
    o.apply_layers(1)
    assert_same_state(g.terms(), o.terms(), f"after psd, path {merge_path}")


def test_psd_after_top_m_and_two_words():
    H = wl.tfim_2d(5, 1.0, 1.5)                       # n = 25, W = 1
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.05, 1e-9, 5000, 1)
    o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, 0.05, 1e-9, 5000, 1)
    g.apply_trotter_layer(2)
    o.apply_layers(2)
    assert g.stats()["cap_events"] > 0
    E = wl.energy_observable(H)
    _close(g.expect_psd(E)[0], o.expect_psd(E)[0])
    H2 = wl.random_pauli_hamiltonian(70, 12, 4, max_weight=3)   # W = 2
    g2 = itpp.Propagator(H2.n, H2.gate_x, H2.gate_z, H2.alpha, 0.1, 1e-5, 1 << 18)
    o2 = oracle.Oracle(H2.n, H2.gate_x, H2.gate_z, H2.alpha, 0.1, 1e-5, 1 << 18)
    g2.apply_trotter_layer(2)
    o2.apply_layers(2)
    O2 = wl.Observable(70, H2.gate_x[:5].copy(), H2.gate_z[:5].copy(),
                       np.array([0.3, -1.2, 0.8, 0.5, -0.1]))
    v, num, pur = g2.expect_psd(O2)
    ov, onum, opur, _ = o2.expect_psd(O2)
    _close(v, ov)
    _close(pur, opur)


def test_psd_twice_the_imaginary_time_on_gpu():
    # h = 0: the Trotter product is exact, the squared state is at beta = 2 tau
    import math
    n, J, tau, L = 10, 0.8, 0.35, 5
    H = wl.tfim_1d(n, J, 0.0)
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, tau / L, 0.0, 1 << 16)
    g.apply_trotter_layer(L)
    v, _, _ = g.expect_psd(wl.zz_observables(n, [(4, 5)])[0])
    assert abs(v - math.tanh(2 * tau * J)) < 1e-12
