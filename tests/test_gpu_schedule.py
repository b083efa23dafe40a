"""Symmetric (Strang) layer schedule on the GPU against the oracle.

With trotter_order = 2 the library builds the symmetric product of each
layer itself; the oracle runs the same schedule written out as a gate list
(workloads.strang_schedule, pinned on the CPU).  States are bit-identical,
and the adjoint's per-term gradients are the schedule's per-gate gradients
folded back (d alpha_gate / d alpha = 1/2 for the halves).
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from tests._compare import assert_same_state

pytestmark = pytest.mark.gpu

itpp = pytest.importorskip("paper_2601_14400_gb300")


@pytest.mark.parametrize("merge_path", [0, 2])
def test_strang_layers_match_oracle(merge_path):
    H = wl.tfim_1d(16, 1.0, 0.9, periodic=True)      # 0.32M terms after 3 layers
    S = wl.strang_schedule(H)
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.05, 1e-6, 1 << 20,
                        merge_path=merge_path, trotter_order=2)
    o = oracle.Oracle(S.n, S.gate_x, S.gate_z, S.alpha, 0.05, 1e-6, 1 << 20)
    for layer in range(3):
        g.apply_trotter_layer(1)
        o.apply_layers(1)
        assert_same_state(g.terms(), o.terms(), f"layer {layer}")


def test_strang_adjoint_folds_per_term():
    H = wl.adjoint_chain(8)
    S = wl.strang_schedule(H)
    O = wl.energy_observable(H)
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.05, 1e-8, 1 << 18, trotter_order=2)
    f_g, d_g = g.adjoint(3, O, ckpt_every=2)
    o = oracle.Oracle(S.n, S.gate_x, S.gate_z, S.alpha, 0.05, 1e-8)
    f_o, d_sched = oracle.FrozenAdjoint(o, 3).grad_alpha(O, S.n_gates)
    G = H.n_gates
    want = np.zeros(G)
    for j in range(S.n_gates):
        k = j if j < G else 2 * G - 2 - j
        want[k] += d_sched[j] * (1.0 if j == G - 1 else 0.5)
    assert abs(f_g - f_o) <= 1e-12 * abs(f_o)
    assert np.max(np.abs(d_g - want)) <= 1e-10 * np.max(np.abs(want))


def test_trotter_order_validation():
    H = wl.tfim_1d(6, 1.0, 1.0)
    with pytest.raises(itpp.ItppError):
        itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.1, 1e-6, 100, trotter_order=3)
