"""GPU path vs the CPU oracle, element by element, through the C ABI.

Bar: string sets identical and coefficients identical in every bit (the
merge has at most two addends per string, so the GPU and the oracle round
the same operations); observables within 1e-10 of the oracle relative to
sum_j |w_j c_j| (the sums are ordered differently).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as wl
from tests._compare import assert_same_state, rel_close

pytestmark = pytest.mark.gpu

itpp = pytest.importorskip("paper_2601_14400_gb300")


def _pair(H, dtau, delta, cap_M=1 << 16, cap_policy=0, **kw):
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta, cap_M, cap_policy, **kw)
    o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta, cap_M, cap_policy)
    return g, o


def _obs_check(g, o, obs):
    got = g.expect(obs)
    want = o.expect(obs)
    cs = o.coeffs(obs.x, obs.z)
    scale = float(np.sum(np.abs(obs.w * cs)))
    assert rel_close(got, want, 1e-10, scale), (got, want)
    gc = g.coeffs(obs.x, obs.z)
    assert np.array_equal(gc.view(np.uint64), cs.view(np.uint64))


# ---------------------------------------------------------------------------
# The n = 8 chain workload, in full, with per-layer observables
# ---------------------------------------------------------------------------
def test_tfim_n8_full_run_bit_exact():
    w = wl.WORKLOADS["tfim1d_n8_open"]
    g, o = _pair(w.H, w.dtau, w.delta, w.cap_M, w.cap_policy)
    for layer in range(w.n_layers):
        g.apply_trotter_layer(1)
        o.apply_layers(1)
        assert_same_state(g.terms(), o.terms(), f"layer {layer}")
        for name, obs in w.observables.items():
            _obs_check(g, o, obs)
    st = g.stats()
    assert st["gates_applied"] == w.n_layers * w.H.n_gates


@pytest.mark.parametrize("k_steps", [1, 2, 3, 15, 16, 40])
def test_single_gates_bit_exact(k_steps):
    H = wl.tfim_1d(6, 1.0, 0.7, periodic=True)
    g, o = _pair(H, 0.1, 1e-9)
    for s in range(k_steps):
        k = s % H.n_gates
        g.apply_gate(k)
        o.apply_gate(k)
    assert_same_state(g.terms(), o.terms(), f"after {k_steps} gates")


# ---------------------------------------------------------------------------
# General Pauli Hamiltonians and word boundaries (W = 1 and 2)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,terms,seed,layers,delta", [
    (10, 12, 1, 3, 1e-6), (33, 20, 2, 2, 1e-5), (64, 24, 3, 2, 1e-5),
    (65, 24, 4, 2, 1e-5), (100, 30, 5, 2, 1e-4), (128, 30, 6, 2, 1e-4)])
def test_random_hamiltonian_bit_exact(n, terms, seed, layers, delta):
    H = wl.random_pauli_hamiltonian(n, terms, seed, max_weight=4)
    g, o = _pair(H, 0.15, delta, cap_M=1 << 18)
    for layer in range(layers):
        g.apply_trotter_layer(1)
        o.apply_layers(1)
        assert_same_state(g.terms(), o.terms(), f"n={n} layer {layer}")


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 127, 128])
def test_tfim_word_boundaries(n):
    periodic = n >= 3
    H = wl.tfim_1d(n, 1.0, 1.0, periodic=periodic)
    g, o = _pair(H, 0.05, 2e-3, cap_M=1 << 18)
    g.apply_trotter_layer(2)
    o.apply_layers(2)
    assert_same_state(g.terms(), o.terms(), f"n={n}")
    _obs_check(g, o, wl.energy_observable(H))


def test_tfim_2d_prefix_bit_exact():
    H = wl.tfim_2d(5, 1.0, 3.04)     # n = 25
    g, o = _pair(H, 0.02, 1e-4, cap_M=1 << 20)
    for layer in range(2):
        g.apply_trotter_layer(1)
        o.apply_layers(1)
    assert_same_state(g.terms(), o.terms(), "2d")
    _obs_check(g, o, wl.energy_observable(H))


def test_tfim_11x11_gate_prefix_bit_exact():
    # the 11x11 workload itself (W = 2): all 220 bonds and the first fields
    w = wl.WORKLOADS["tfim2d_11x11"]
    g, o = _pair(w.H, w.dtau, w.delta, cap_M=1 << 22)
    for k in range(236):
        g.apply_gate(k)
        o.apply_gate(k)
    assert_same_state(g.terms(), o.terms(), "11x11")
    for obs in w.observables.values():
        _obs_check(g, o, obs)


# ---------------------------------------------------------------------------
# Synthetic states spanning many tiles with a ragged tail, one gate each
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,M", [(64, (1 << 15) + 77), (121, (1 << 14) + 5), (20, 3001)])
@pytest.mark.parametrize("which", ["zz", "x", "y"])
def test_synthetic_state_one_gate(n, M, which):
    X, Z, C = wl.synthetic_state(n, M, 2601 + n, delta=1e-6)
    if which == "zz":
        gx, gz = wl.two_site(n, 3, 4, "Z", "Z")
    elif which == "x":
        gx, gz = wl.single_site(n, 5, "X")
    else:
        gx, gz = wl.two_site(n, 0, n - 1, "Y", "X")
    H = wl.Hamiltonian(n, gx[None], gz[None], np.array([-0.7]))
    g, o = _pair(H, 0.05, 1e-6, cap_M=2 * M + 2)
    g.set_terms(X, Z, C)
    o.set_terms(X, Z, C)
    assert_same_state(g.terms(), o.terms(), "loaded")
    g.apply_gate(0)
    o.apply_gate(0)
    assert_same_state(g.terms(), o.terms(), f"{which} gate")


# ---------------------------------------------------------------------------
# Edge cases and degenerate inputs
# ---------------------------------------------------------------------------
def test_identity_only_and_delta_zero():
    H = wl.tfim_1d(4, 1.0, 1.0)
    g, o = _pair(H, 0.1, 0.0)
    assert g.count() == 1
    x, z, c = g.terms()
    assert c[0] == 1.0 and not x.any() and not z.any()
    g.apply_trotter_layer(3)
    o.apply_layers(3)
    assert_same_state(g.terms(), o.terms(), "delta=0")


def test_negative_zero_delta_is_zero():
    # the threshold is compared on bit patterns: -0.0 must act as +0.0
    H = wl.tfim_1d(5, 1.0, 0.7)
    g, o = _pair(H, 0.1, -0.0)
    g.apply_trotter_layer(3)
    o.apply_layers(3)
    assert_same_state(g.terms(), o.terms(), "delta=-0")
    g.truncate(-0.0)
    assert_same_state(g.terms(), o.terms(), "truncate(-0)")


def test_everything_truncated_but_identity():
    H = wl.tfim_1d(5, 1.0, 1.0)
    g, o = _pair(H, 0.05, 0.5)
    g.apply_trotter_layer(4)
    o.apply_layers(4)
    assert g.count() == 1
    assert_same_state(g.terms(), o.terms(), "delta=0.5")


def test_explicit_truncate():
    w = wl.WORKLOADS["tfim1d_n8_open"]
    g, o = _pair(w.H, w.dtau, 0.0)
    g.apply_trotter_layer(5)
    o.apply_layers(5)
    g.truncate(1e-3)
    x, z, c = o.terms()
    keep = np.abs(c) > 1e-3
    assert_same_state(g.terms(), (x[keep], z[keep], c[keep]), "truncate")
    with pytest.raises(itpp.ItppError):
        g.truncate(2.0)      # would drop the identity
        g.synchronize()


def test_cap_policy_error():
    H = wl.tfim_1d(8, 1.0, 1.0)
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.1, 1e-9, 50, 0)
    with pytest.raises(itpp.ItppError) as e:
        g.apply_trotter_layer(3)
        g.synchronize()
    assert e.value.status == 3
    with pytest.raises(itpp.ItppError):
        g.count()


@pytest.mark.parametrize("M", [100, 1000, 2049])
def test_cap_policy_topM_bit_exact(M):
    H = wl.tfim_1d(10, 1.0, 1.0, periodic=True)
    g, o = _pair(H, 0.1, 1e-9, cap_M=M, cap_policy=1)
    for layer in range(4):
        g.apply_trotter_layer(1)
        o.apply_layers(1)
        assert_same_state(g.terms(), o.terms(), f"M={M} layer {layer}")
    assert g.stats()["cap_events"] > 0


def test_cap_policy_topM_with_exact_ties():
    n, M = 16, 500
    X, Z, C = wl.synthetic_state(n, 2000, 9, delta=1e-3)
    C[1:] = np.sign(C[1:]) * 2.0 ** np.round(np.log2(np.abs(C[1:])))   # many equal |c|
    gx, gz = wl.single_site(n, 2, "X")
    H = wl.Hamiltonian(n, gx[None], gz[None], np.array([-1.0]))
    g, o = _pair(H, 0.1, 1e-9, cap_M=M, cap_policy=1)
    g.set_terms(X[:M], Z[:M], C[:M])
    o.set_terms(X[:M], Z[:M], C[:M])
    g.apply_gate(0)
    o.apply_gate(0)
    assert_same_state(g.terms(), o.terms(), "ties")


@pytest.mark.parametrize("cap_M", [4_000_001, 4_500_000])
def test_cap_policy_topM_large_tie_class(cap_M):
    # 4M strings with |c| = 1/2: after a ZZ gate about 2M children share
    # each of three magnitudes, so the first digit of the select holds about
    # 2M candidates, more than the gather's shared stages hold (the overflow
    # path writes them straight to the list).  cap_M = 4M + 1 keeps exactly
    # the two upper classes; 4.5M cuts inside the third, where the key
    # tie-break decides among 2M equal magnitudes.
    n, M = 64, 4_000_000
    X, Z, C = wl.synthetic_state(n, M, 1461, delta=1e-6)
    C[1:] = np.where(C[1:] < 0, -0.5, 0.5)
    gx, gz = wl.two_site(n, 10, 11, "Z", "Z")
    H = wl.Hamiltonian(n, gx[None], gz[None], np.array([-1.0]))
    g, o = _pair(H, 0.1, 1e-12, cap_M=cap_M, cap_policy=1)
    g.set_terms(X, Z, C)
    o.set_terms(X, Z, C)
    g.apply_gate(0)
    o.apply_gate(0)
    st = g.stats()
    assert st["select_candidates"] > 1_900_000 and st["cap_events"] == 1
    assert_same_state(g.terms(), o.terms(), f"cap_M={cap_M}")


def test_set_terms_validation():
    H = wl.tfim_1d(8, 1.0, 1.0)
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.1, 1e-9, 1000, 0)
    X, Z, C = wl.synthetic_state(8, 20, 1)
    with pytest.raises(itpp.ItppError) as e:      # duplicate key
        g.set_terms(np.concatenate([X, X[3:4]]), np.concatenate([Z, Z[3:4]]),
                    np.concatenate([C, C[3:4]]))
    assert e.value.status == 1
    with pytest.raises(itpp.ItppError) as e:      # identity missing
        g.set_terms(X[1:], Z[1:], C[1:])
    assert e.value.status == 6
    Xb = X.copy()
    Xb[2, 0] |= np.uint64(1) << np.uint64(9)       # bit >= n
    with pytest.raises(itpp.ItppError) as e:
        g.set_terms(Xb, Z, C)
    assert e.value.status == 1
    g.set_terms(X, Z, C)                          # still usable afterwards
    assert g.count() == 21


def test_create_validation():
    H = wl.tfim_1d(8, 1.0, 1.0)
    bad = H.gate_x.copy()
    bad[0, 0] |= np.uint64(1) << np.uint64(40)
    for args in [dict(delta=-1.0), dict(cap_M=0), dict(cap_policy=3)]:
        kw = dict(delta=1e-6, cap_M=100, cap_policy=0)
        kw.update(args)
        with pytest.raises(itpp.ItppError):
            itpp.Propagator(8, H.gate_x, H.gate_z, H.alpha, 0.1, kw["delta"], kw["cap_M"],
                            kw["cap_policy"])
    with pytest.raises(itpp.ItppError):
        itpp.Propagator(8, bad, H.gate_z, H.alpha, 0.1, 1e-6, 100)


def test_non_finite_inputs_rejected():
    """NaN or inf coefficients, and gate weights cosh / sinh that overflow
    (|alpha dtau| beyond about 710), are argument errors."""
    H = wl.tfim_1d(8, 1.0, 1.0)
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.1, 1e-9, 1000, 0)
    X, Z, C = wl.synthetic_state(8, 20, 1)
    for bad in (np.nan, np.inf, -np.inf):
        Cb = C.copy()
        Cb[5] = bad
        with pytest.raises(itpp.ItppError) as e:
            g.set_terms(X, Z, Cb)
        assert e.value.status == 1
    g.set_terms(X, Z, C)                          # still usable afterwards
    assert g.count() == 21
    with pytest.raises(itpp.ItppError) as e:
        g.set_alpha(np.full_like(H.alpha, 1e4))   # theta = 1e3: cosh overflows
    assert e.value.status == 1
    g.close()
    with pytest.raises(itpp.ItppError):
        itpp.Propagator(H.n, H.gate_x, H.gate_z, np.full_like(H.alpha, -1e4), 0.1, 1e-9, 1000)


def test_overflowing_child_is_a_device_error():
    """A finite coefficient near the largest double times cosh(1) overflows to
    inf: the gate reports ITPP_ERR_STATE instead of carrying an inf on."""
    H = wl.tfim_1d(4, 10.0, 1.0)                 # bonds: alpha = -10, theta = -1
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.1, 1e-9, 1000, 0)
    X = np.zeros((2, 1), dtype=np.uint64)
    Z = np.array([[0], [1]], dtype=np.uint64)    # I and Z_0, which commutes with Z_0 Z_1
    g.set_terms(X, Z, np.array([1.0, 1.7e308]))   # times cosh(1): 2.6e308 > DBL_MAX
    g.apply_gate(0)
    with pytest.raises(itpp.ItppError) as e:
        g.synchronize()
    assert e.value.status == 8
    g.close()


@pytest.mark.parametrize("block,ipt,load", [(128, 1, 25), (256, 4, 75), (512, 2, 50)])
def test_launch_shapes_give_identical_states(block, ipt, load):
    H = wl.tfim_1d(12, 1.0, 1.0, periodic=True)
    g, o = _pair(H, 0.05, 1e-7, cap_M=1 << 18, block_threads=block, items_per_thread=ipt,
                 table_load_pct=load, merge_path=2)
    g.apply_trotter_layer(3)
    o.apply_layers(3)
    assert_same_state(g.terms(), o.terms(), f"block={block} ipt={ipt} load={load}")


@pytest.mark.parametrize("n,cap_policy,delta", [(10, 0, 1e-7), (12, 1, 1e-7), (70, 0, 1e-3)])
@pytest.mark.parametrize("block,ipt", [(128, 1), (512, 2)])
def test_partitioned_merge_windows_and_long_partitions(n, cap_policy, delta, block, ipt):
    # 128 x 1 holds 128 items in registers and the scatter aims at 2048
    # terms per partition: every partition takes the long path, in sub-passes
    # (one per 1024 terms) that each hold one hash class of the pairs
    H = wl.tfim_1d(n, 1.0, 0.9, periodic=True)
    cap = 3000 if cap_policy else 1 << 20
    g, o = _pair(H, 0.1, delta, cap_M=cap, cap_policy=cap_policy, block_threads=block,
                 items_per_thread=ipt, merge_path=0,
                 partition_target=2048 if block == 128 else 0)
    for layer in range(3):
        g.apply_trotter_layer(1)
        o.apply_layers(1)
        st = g.stats(check=False)
        assert st["status"] == 0, (st["status"], st["error_site"])
        assert_same_state(g.terms(), o.terms(), f"{block}x{ipt} layer {layer}")
    g.apply_gate(3)                  # a single gate: a window of its own
    o.apply_gate(3)
    g.apply_gate(4)                  # the next gate reuses no stale partition
    o.apply_gate(4)
    assert_same_state(g.terms(), o.terms(), "single gates")
    st = g.stats()
    assert st["repartitions"] >= 3 * 2     # at least one scatter per bond / field window
    if block == 128 and st["peak_terms"] > 2048:
        assert st["long_partitions"] > 0


@pytest.mark.parametrize("n,W_delta", [(64, 1e-4), (100, 2e-4)])
def test_merge_paths_identical(n, W_delta):
    # partitioned shared-memory merge vs one global table, many partitions
    H = wl.tfim_1d(n, 1.0, 1.0, periodic=True)
    a = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.05, W_delta, 1 << 22, merge_path=0)
    b = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.05, W_delta, 1 << 22, merge_path=2)
    a.apply_trotter_layer(2)
    b.apply_trotter_layer(2)
    assert a.count() > 20000
    from tests._compare import sort_terms
    assert_same_state(a.terms(), sort_terms(*b.terms()), f"n={n}")


# ---------------------------------------------------------------------------
# The paper's printed count: untruncated N = 12 support
# ---------------------------------------------------------------------------
def test_paper_untruncated_support_n12():
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "paper_numbers.json")))["untruncated_support_N12"]
    H = wl.tfim_1d(12, 1.0, 0.5)
    g = itpp.Propagator(12, H.gate_x, H.gate_z, H.alpha, 0.04, 0.0, 1 << 22)
    prev = -1
    for layer in range(500):        # tau = 20
        g.apply_trotter_layer(10)
        c = g.count()
        if c == prev:
            break
        prev = c
    assert g.count() == gold["value"]
    x, z, c = g.terms()
    ident = ~(x.any(axis=1) | z.any(axis=1))
    assert ident.sum() == 1 and c[ident][0] == 1.0


# ---------------------------------------------------------------------------
# The paper's printed pair (Sec. III.C) under the readings taken here
# ---------------------------------------------------------------------------
def test_paper_pair_workload_matches_the_oracle():
    """N = 12 open chain, J = 1, h = 0.5, dtau = 0.04, 500 layers, delta =
    2^-7 and 2^-8: the final count and the energy's coefficients equal the
    oracle's stored values bit for bit (tests/golden/make_paper_pair.py),
    and the energy agrees to 1e-12.  The paper's 42,466 terms at 2^-7 are
    not what this reading gives (189); the stored record says so."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "paper_pair_readings.json")))
    H = wl.tfim_1d(12, 1.0, 0.5)
    obs = wl.energy_observable(H)
    for case in gold["cases"]:
        g = itpp.Propagator(12, H.gate_x, H.gate_z, H.alpha, 0.04,
                            2.0 ** case["delta_log2"], 1 << 20)
        g.apply_trotter_layer(500)
        assert g.count() == case["final_terms"], case["delta_log2"]
        want = np.array([float.fromhex(h) for h in case["energy_term_coeffs_hex"]])
        got = g.coeffs(obs.x, obs.z)
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), case["delta_log2"]
        E = g.expect(obs)
        assert abs(E - case["energy"]) <= 1e-12 * abs(case["energy"])
        g.close()
    assert all(c["final_terms"] != 42466 for c in gold["cases"])


# ---------------------------------------------------------------------------
# Children below the select's predicted range, and the merge run again
# ---------------------------------------------------------------------------
def test_dropped_children_and_merge_retry_match_oracle():
    """With top-M the partitioned merge leaves children below the select's
    predicted range unwritten; when fewer than cap_M children are then kept
    (the threshold fell below the range: here after every coefficient of the
    Hamiltonian is cut to a fifth mid-run) the gate's merge runs again in
    full.  Both cases stay equal to the oracle bit for bit, and the second
    one occurs."""
    H = wl.tfim_1d(12, 1.0, 1.0, periodic=True)
    M, dtau, delta = 3000, 0.1, 1e-9
    g, o = _pair(H, dtau, delta, cap_M=M, cap_policy=1)
    for layer in range(4):
        g.apply_trotter_layer(1)
        o.apply_layers(1)
        assert_same_state(g.terms(), o.terms(), f"layer {layer}")
    assert g.stats()["cap_events"] > 0
    a2 = np.asarray(H.alpha) * 0.2
    g.set_alpha(a2)
    o2 = oracle.Oracle(H.n, H.gate_x, H.gate_z, a2, dtau, delta, M, 1)
    o2.set_terms(*o.terms())
    for layer in range(3):
        g.apply_trotter_layer(1)
        o2.apply_layers(1)
        assert_same_state(g.terms(), o2.terms(), f"after the cut, layer {layer}")
    st = g.stats()
    print("merge retries", st["merge_retries"], "full selects", st["select_full"])
    assert st["merge_retries"] > 0


# ---------------------------------------------------------------------------
# Dense states against the partition layout (no device error)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [16, 20, 24, 28, 32, 48])
def test_dense_chains_keep_within_partition_strides(n):
    """Open chains of the field-sweep recipe at a 2^18 bound (top-M), 50
    layers: the states are dense in the low-weight strings, so the groups of
    a window (the strings with one pattern outside it) are large; a group
    must always fit one partition's stride.  The run ends without a device
    error and the bound holds."""
    H = wl.tfim_1d(n, 1.0, 1.2)
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.02, 1e-7, 1 << 18, 1)
    g.apply_trotter_layer(50)
    g.synchronize()
    st = g.stats()
    assert st["status"] == 0 and 0 < g.count() <= 1 << 18
