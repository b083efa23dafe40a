"""Batched propagation vs the oracle, instance by instance, through the C ABI.

Every instance of a batch must equal its own plain propagation bit for bit
(string set and coefficient bits), so each is compared with the oracle run
on that instance's Hamiltonian alone.  Both merges of the batch: the
partitioned one (merge_path 0; with partition_target 2048 every partition
passes the staging capacity and takes the sub-pass path) and the global
table (merge_path 2).
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from tests._compare import assert_same_state, rel_close

pytestmark = pytest.mark.gpu

itpp = pytest.importorskip("paper_2601_14400_gb300")


def _oracles(hams, dtau, delta, cap_M, cap_policy):
    return [oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta, cap_M, cap_policy)
            for H in hams]


def _check_all(bp, ors, hams, what):
    for b, (o, H) in enumerate(zip(ors, hams)):
        x, z, c = bp.terms(b)
        ox, oz, oc = o.terms()
        # oracle strings have H.W words; the batch uses the widest W
        W = ox.shape[1]
        assert not x[:, W:].any() and not z[:, W:].any()
        assert_same_state((x[:, :W], z[:, :W], c), (ox, oz, oc), f"{what} instance {b}")


PATHS = [(0, 0), (0, 2048), (2, 0)]


@pytest.mark.parametrize("merge_path,target", PATHS)
def test_batch_mixed_chains_bit_exact(merge_path, target):
    hams = [wl.tfim_1d(8, 1.0, 0.7), wl.tfim_1d(12, 1.0, 1.3, periodic=True),
            wl.tfim_1d(5, 0.8, 2.0), wl.tfim_1d(16, 1.0, 0.5), wl.tfim_1d(1, 1.0, 1.0),
            wl.tfim_2d(3, 1.0, 1.5)]
    dtau, delta = 0.05, 1e-5
    bp = itpp.BatchPropagator(hams, dtau, delta, 1 << 18, merge_path=merge_path,
                              partition_target=target)
    ors = _oracles(hams, dtau, delta, 1 << 18, 0)
    for layer in range(3):
        bp.apply_trotter_layer(1)
        for o in ors:
            o.apply_layers(1)
        _check_all(bp, ors, hams, f"layer {layer}")
    for b, (o, H) in enumerate(zip(ors, hams)):
        E = wl.energy_observable(H)
        got, want = bp.expect(b, E), o.expect(E)
        scale = float(np.sum(np.abs(E.w * o.coeffs(E.x, E.z))))
        assert rel_close(got, want, 1e-10, scale)
    bp.synchronize()


@pytest.mark.parametrize("merge_path,target", PATHS)
def test_batch_two_words_and_random_hamiltonians(merge_path, target):
    hams = [wl.random_pauli_hamiltonian(70, 20, 1, max_weight=3),
            wl.random_pauli_hamiltonian(10, 12, 2), wl.tfim_1d(100, 1.0, 1.0, periodic=True)]
    dtau, delta = 0.1, 5e-3
    bp = itpp.BatchPropagator(hams, dtau, delta, 1 << 17, merge_path=merge_path,
                              partition_target=target)
    ors = _oracles(hams, dtau, delta, 1 << 17, 0)
    bp.apply_trotter_layer(2)
    for o in ors:
        o.apply_layers(2)
    _check_all(bp, ors, hams, "W=2")


@pytest.mark.parametrize("merge_path", [0, 2])
@pytest.mark.parametrize("M", [300, 2000])
def test_batch_top_m_bit_exact(M, merge_path):
    hams = [wl.tfim_1d(10, 1.0, 1.0, periodic=True), wl.tfim_1d(14, 1.0, 0.6),
            wl.tfim_1d(6, 1.0, 2.0)]
    dtau, delta = 0.1, 1e-9
    bp = itpp.BatchPropagator(hams, dtau, delta, M, cap_policy=1, merge_path=merge_path)
    ors = _oracles(hams, dtau, delta, M, 1)
    for layer in range(3):
        bp.apply_trotter_layer(1)
        for o in ors:
            o.apply_layers(1)
        _check_all(bp, ors, hams, f"M={M} layer {layer}")
    assert any(bp.stats(b)["cap_events"] > 0 for b in range(len(hams)))


@pytest.mark.parametrize("merge_path", [0, 2])
def test_batch_instance_error_is_isolated(merge_path):
    hams = [wl.tfim_1d(12, 1.0, 1.0), wl.tfim_1d(3, 1.0, 1.0)]
    bp = itpp.BatchPropagator(hams, 0.1, 1e-9, 60, cap_policy=0, merge_path=merge_path)
    bp.apply_trotter_layer(3)
    counts, statuses = bp.counts()
    assert statuses[0] == 3          # the 12-site chain passes 60 terms
    assert statuses[1] == 0          # the 3-site chain holds at most C(6,3) = 20
    o = oracle.Oracle(3, hams[1].gate_x, hams[1].gate_z, hams[1].alpha, 0.1, 1e-9, 60, 0)
    o.apply_layers(3)
    x, z, c = bp.terms(1)
    assert_same_state((x, z, c), o.terms(), "healthy instance")
    with pytest.raises(itpp.ItppError):
        bp.synchronize()


def test_field_sweep_recipe_sampled_instances():
    ns, hs = wl.batch_field_sweep()
    hams = [wl.tfim_1d(n, 1.0, h) for n, h in zip(ns, hs)]
    dtau, delta, M = 0.02, 1e-7, 4096
    bp = itpp.BatchPropagator(hams, dtau, delta, M, cap_policy=1)
    bp.apply_trotter_layer(1)
    counts, statuses = bp.counts()
    assert (statuses == 0).all() and (counts > 0).all() and (counts <= M).all()
    for b in (0, 1, len(hams) - 2, len(hams) - 1):
        H = hams[b]
        o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta, M, 1)
        o.apply_layers(1)
        assert_same_state(bp.terms(b), o.terms(), f"sweep instance {b} (n={H.n})")


@pytest.mark.parametrize("merge_path", [0, 2])
def test_autotune_keeps_results_bit_identical(merge_path):
    # the tuner resets every instance and installs the fastest shape; any
    # shape gives the plain run's states
    hams = [wl.tfim_1d(10, 1.0, 0.7), wl.tfim_1d(14, 1.0, 1.3, periodic=True),
            wl.tfim_1d(6, 0.8, 2.0), wl.tfim_2d(3, 1.0, 1.5)]
    dtau, delta = 0.05, 1e-6
    bp = itpp.BatchPropagator(hams, dtau, delta, 1 << 16, 1, merge_path=merge_path)
    bp.apply_trotter_layer(2)             # state before tuning is discarded
    r = bp.autotune(probe_layers=2)
    assert r["main_block"] in (128, 256, 512)
    assert r["insert_grid"] in (4, 8, 16)
    if merge_path == 0:
        assert 1 <= r["main_grid"] <= 8 and r["table_load_pct"] == 0
        assert r["partition_target"] in (350, 500, 700, 1000)
    else:
        assert r["main_grid"] in (2, 4, 8) and 25 <= r["table_load_pct"] <= 65
        assert r["partition_target"] == 0
    assert r["candidates"] >= 8 and r["ms_per_probe"] <= r["ms_per_probe_default"]
    counts, _ = bp.counts()
    assert all(int(c) == 1 for c in counts)           # back at the identity
    assert all(bp.stats(b)["gates_applied"] == 0 for b in range(len(hams)))
    ors = _oracles(hams, dtau, delta, 1 << 16, 1)
    for layer in range(3):
        bp.apply_trotter_layer(1)
        for o in ors:
            o.apply_layers(1)
    _check_all(bp, ors, hams, "after autotune")
