"""Sort-based merge (merge_path 1) against the oracle and the hash paths.

The sort path finds equal strings with a radix sort of the commuting terms'
children and a segmented reduce; every state must be bit-identical to the
oracle's (same string set, same coefficient bits) and to the hash paths.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from tests._compare import assert_same_state, rel_close, sort_terms

pytestmark = pytest.mark.gpu

itpp = pytest.importorskip("paper_2601_14400_gb300")


def _pair(H, dtau, delta, cap_M=1 << 16, cap_policy=0):
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta, cap_M, cap_policy,
                        merge_path=1)
    o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta, cap_M, cap_policy)
    return g, o


def test_sorted_tfim_n8_full_run():
    w = wl.WORKLOADS["tfim1d_n8_open"]
    g, o = _pair(w.H, w.dtau, w.delta, w.cap_M, w.cap_policy)
    for layer in range(w.n_layers):
        g.apply_trotter_layer(1)
        o.apply_layers(1)
        if layer % 5 == 4:
            assert_same_state(g.terms(), o.terms(), f"layer {layer}")
            for name, obs in w.observables.items():
                assert rel_close(g.expect(obs), o.expect(obs), 1e-10), name


@pytest.mark.parametrize("n,terms,seed,layers,delta", [
    (20, 12, 3, 3, 1e-6),      # W = 1
    (70, 14, 5, 2, 1e-4),      # W = 2
    (121, 10, 7, 2, 1e-3),     # W = 2, every digit of the upper words
])
def test_sorted_random_hamiltonian(n, terms, seed, layers, delta):
    H = wl.random_pauli_hamiltonian(n, terms, seed, max_weight=4)
    g, o = _pair(H, 0.1, delta, 1 << 18)
    g.apply_trotter_layer(layers)
    o.apply_layers(layers)
    assert_same_state(g.terms(), o.terms(), f"n={n}")


@pytest.mark.parametrize("n", [1, 7, 8, 9, 63, 64, 65, 128])
def test_sorted_word_and_digit_boundaries(n):
    # the pass plan skips digits above bit n: n on and off digit boundaries
    H = wl.tfim_1d(n, 1.0, 0.9, periodic=n > 2)
    g, o = _pair(H, 0.05, 2e-3, 1 << 18)
    g.apply_trotter_layer(2)
    o.apply_layers(2)
    assert_same_state(g.terms(), o.terms(), f"n={n}")


@pytest.mark.parametrize("M", [100, 2049])
def test_sorted_top_m(M):
    H = wl.tfim_1d(10, 1.0, 1.0, periodic=True)
    g, o = _pair(H, 0.1, 1e-9, cap_M=M, cap_policy=1)
    for layer in range(3):
        g.apply_trotter_layer(1)
        o.apply_layers(1)
        assert_same_state(g.terms(), o.terms(), f"M={M} layer {layer}")
    assert g.stats()["cap_events"] > 0


def test_sorted_edge_cases():
    H = wl.tfim_1d(5, 1.0, 1.0)
    g, o = _pair(H, 0.05, 0.5)                # everything but the identity dropped
    g.apply_trotter_layer(3)
    o.apply_layers(3)
    assert g.count() == 1
    assert_same_state(g.terms(), o.terms(), "delta=0.5")
    g, o = _pair(H, 0.1, 0.0)                 # delta = 0 keeps every nonzero child
    g.apply_trotter_layer(3)
    o.apply_layers(3)
    assert_same_state(g.terms(), o.terms(), "delta=0")
    H8 = wl.tfim_1d(8, 1.0, 1.0)
    g = itpp.Propagator(H8.n, H8.gate_x, H8.gate_z, H8.alpha, 0.1, 1e-9, 50, 0, merge_path=1)
    with pytest.raises(itpp.ItppError) as e:  # the bound as an error
        g.apply_trotter_layer(3)
        g.synchronize()
    assert e.value.status == 3


def test_sorted_synthetic_state_one_gate():
    n, M = 64, 20000 + 77
    X, Z, C = wl.synthetic_state(n, M, 2601, delta=1e-6)
    for q in (wl.two_site(n, 10, 11, "Z", "Z"), wl.single_site(n, 10, "X")):
        H = wl.Hamiltonian(n, q[0][None], q[1][None], np.array([-1.0]))
        g, o = _pair(H, 0.1, 1e-6, cap_M=2 * M + 2)
        g.set_terms(X, Z, C)
        o.set_terms(X, Z, C)
        g.apply_gate(0)
        o.apply_gate(0)
        assert_same_state(g.terms(), o.terms(), "synthetic")


@pytest.mark.parametrize("n,delta", [(64, 1e-4), (100, 2e-4)])
def test_all_three_merge_paths_identical(n, delta):
    H = wl.tfim_1d(n, 1.0, 1.0, periodic=True)
    states = []
    for path in (0, 1, 2):
        p = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.05, delta, 1 << 22,
                            merge_path=path)
        p.apply_trotter_layer(2)
        states.append(sort_terms(*p.terms()))
    assert states[0][2].shape[0] > 20000
    assert_same_state(states[1], states[0], "sort vs partitioned")
    assert_same_state(states[2], states[0], "global table vs partitioned")
