"""Pauli weight cutoff (Sec. II.B) on the GPU against the oracle.

The oracle's cutoff is pinned against a dense projection onto the weight <= k
span after every gate (tests/test_oracle_pins.py); here every merge path,
the top-M bound and the batched path must match the oracle bit for bit.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from tests._compare import assert_same_state

pytestmark = pytest.mark.gpu

itpp = pytest.importorskip("paper_2601_14400_gb300")


@pytest.mark.parametrize("merge_path", [0, 1, 2])
@pytest.mark.parametrize("n,k,delta", [(12, 3, 1e-9), (40, 4, 1e-6), (70, 3, 1e-5)])
def test_weight_cutoff_matches_oracle(merge_path, n, k, delta):
    H = wl.tfim_1d(n, 1.0, 0.9, periodic=True)
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.1, delta, 1 << 20,
                        merge_path=merge_path, max_weight=k)
    o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, 0.1, delta, 1 << 20, 0, max_weight=k)
    for layer in range(3):
        g.apply_trotter_layer(1)
        o.apply_layers(1)
        assert_same_state(g.terms(), o.terms(), f"path {merge_path} k={k} layer {layer}")
    x, z, _ = g.terms()
    w = np.array([sum(bin(int(a) | int(b)).count("1") for a, b in zip(xr, zr))
                  for xr, zr in zip(x, z)])
    assert w.max() <= k


def test_weight_cutoff_with_top_m_and_random_hamiltonian():
    H = wl.random_pauli_hamiltonian(20, 12, 3, max_weight=3)
    # the cutoff alone keeps 439 / 700 / 778 terms: a bound of 300 fires
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.1, 1e-9, 300, 1, max_weight=5)
    o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, 0.1, 1e-9, 300, 1, max_weight=5)
    g.apply_trotter_layer(3)
    o.apply_layers(3)
    assert_same_state(g.terms(), o.terms(), "top-M with weight cutoff")
    assert g.stats()["cap_events"] > 0


def test_weight_cutoff_batched():
    hams = [wl.tfim_1d(10, 1.0, 0.7), wl.tfim_1d(16, 1.0, 1.2, periodic=True)]
    bp = itpp.BatchPropagator(hams, 0.05, 1e-8, 1 << 16, max_weight=3)
    bp.apply_trotter_layer(3)
    for b, H in enumerate(hams):
        o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, 0.05, 1e-8, 1 << 16, 0, max_weight=3)
        o.apply_layers(3)
        assert_same_state(bp.terms(b), o.terms(), f"instance {b}")


def test_weight_cutoff_rejects_bad_bound():
    H = wl.tfim_1d(8, 1.0, 1.0)
    with pytest.raises(itpp.ItppError):
        itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.1, 1e-6, 100, max_weight=-1)
    with pytest.raises(itpp.ItppError):
        itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.1, 1e-6, 100, max_weight=129)
