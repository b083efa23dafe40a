"""K-truncation (Sec. II.C) and the K(N, eps0) scan of the scalability study.

K-truncation keeps the K largest |c| after every step: cap_policy 1 with
delta = 0.  The GPU run is bit-identical to the oracle's; a K above the
untruncated support changes nothing; and the scan finds the smallest K
(doubling from 2^9) whose thermal energy is within eps0 = 1e-2 of the exact
free-fermion value, for open TFIM chains (J = 1, h = 0.5) at the paper's
high temperatures.  The table is printed (pytest -s).
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from oracle import dense
from tests._compare import assert_same_state, sort_terms

pytestmark = pytest.mark.gpu

itpp = pytest.importorskip("paper_2601_14400_gb300")


def test_k_truncation_matches_oracle():
    H = wl.tfim_1d(14, 1.0, 0.5)
    K = 1 << 10
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.04, 0.0, K, 1)
    o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, 0.04, 0.0, K, 1)
    for layer in range(4):
        g.apply_trotter_layer(1)
        o.apply_layers(1)
        assert_same_state(g.terms(), o.terms(), f"K-truncation layer {layer}")
    assert g.count() == K and g.stats()["cap_events"] > 0


def test_k_above_support_is_untruncated():
    H = wl.tfim_1d(8, 1.0, 0.5)
    a = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.04, 0.0, 1 << 16, 1)
    b = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.04, 0.0, 1 << 16, 0)
    a.apply_trotter_layer(10)
    b.apply_trotter_layer(10)
    assert a.stats()["cap_events"] == 0
    assert_same_state(sort_terms(*a.terms()), sort_terms(*b.terms()), "K above the support")


def _rel_energy_error(N, beta, dtau, K):
    H = wl.tfim_1d(N, 1.0, 0.5)
    L = int(round(beta / dtau))
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, dtau, 0.0, K, 1)
    g.apply_trotter_layer(L)
    E = g.expect(wl.energy_observable(H))
    exact = dense.bdg_energy(np.ones(N - 1), np.full(N, 0.5), L * dtau)
    return abs(E - exact) / abs(exact)


@pytest.mark.parametrize("beta", [0.08, 0.24])
def test_k_scan_grows_slowly_at_high_temperature(beta):
    eps0, dtau = 1e-2, 0.02
    table = {}
    for N in (12, 16, 20):
        K = 1 << 9
        while _rel_energy_error(N, beta, dtau, K) > eps0:
            K <<= 1
            assert K <= 1 << 20, (N, beta)
        table[N] = K
    print(f"K(N, 1e-2) at beta={beta}: {table}")
    Ks = [table[N] for N in sorted(table)]
    assert all(a <= b for a, b in zip(Ks, Ks[1:]))
