"""Canonical-order export and file checkpoints through the C ABI.

`itpp_get_terms_sorted` must give the oracle's own export order (ascending
x words, then z words) with no sorting on the Python side, and a state saved
with `itpp_save` and resumed with `itpp_load` must continue bit for bit as
the handle that saved it (the coefficients are stored normalised, and
normalising on load multiplies by exactly 1).
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

itpp = pytest.importorskip("paper_2601_14400_gb300")


def _same_bits(a, b, what):
    ax, az, ac = a
    bx, bz, bc = b
    assert ax.shape == bx.shape, f"{what}: {ax.shape[0]} vs {bx.shape[0]} terms"
    assert np.array_equal(ax, bx) and np.array_equal(az, bz), f"{what}: keys differ"
    assert np.array_equal(ac.view(np.uint64), bc.view(np.uint64)), f"{what}: coefficients differ"


def _chain(n, periodic):
    return wl.tfim_1d(n, 1.0, 0.9, periodic=periodic)


# sizes the oracle finishes in seconds: 135k terms (W = 1), 9.7k (W = 2)
@pytest.mark.parametrize("n,periodic,delta,layers", [(16, False, 1e-4, 3), (70, True, 3e-3, 2)])
def test_sorted_export_is_the_oracle_order(n, periodic, delta, layers):
    H = _chain(n, periodic)
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, 0.1, delta, 1 << 20)
    o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, 0.1, delta, 1 << 20, 0)
    g.apply_trotter_layer(layers)
    o.apply_layers(layers)
    _same_bits(g.sorted_terms(), o.terms(), f"n={n}")


def test_save_load_resumes_bit_for_bit(tmp_path):
    H, dtau, delta = _chain(16, False), 0.1, 1e-3     # 69k terms after 5 layers
    mk = lambda: itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta, 1 << 20)
    g = mk()
    g.apply_trotter_layer(3)
    f1 = tmp_path / "layer3.itpp"
    g.save(f1)
    g.apply_trotter_layer(2)
    h = mk()
    h.load(f1)
    h.apply_trotter_layer(2)
    _same_bits(h.sorted_terms(), g.sorted_terms(), "resumed vs continued")
    o = oracle.Oracle(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta, 1 << 20, 0)
    o.apply_layers(5)
    _same_bits(h.sorted_terms(), o.terms(), "resumed vs oracle")
    # equal states give equal files (canonical order)
    fa, fb = tmp_path / "a.itpp", tmp_path / "b.itpp"
    g.save(fa)
    h.save(fb)
    assert fa.read_bytes() == fb.read_bytes()
    n_terms = g.count()
    assert fa.stat().st_size == 8 + 8 + 8 + n_terms * (8 + 8 + 8)


def test_load_rejects_foreign_and_damaged_files(tmp_path):
    H, dtau, delta = _chain(16, False), 0.1, 1e-3
    g = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta, 1 << 20)
    g.apply_trotter_layer(2)
    good = tmp_path / "good.itpp"
    g.save(good)
    before = g.sorted_terms()
    H17 = wl.tfim_1d(17, 1.0, 0.9)
    other = itpp.Propagator(H17.n, H17.gate_x, H17.gate_z, H17.alpha, dtau, delta, 1 << 20)
    with pytest.raises(itpp.ItppError) as e:       # another n
        other.load(good)
    assert e.value.status == 9
    data = good.read_bytes()
    bad = tmp_path / "bad.itpp"
    for blob in (b"NOTSTATE" + data[8:], data[:-5], b""):
        bad.write_bytes(blob)
        with pytest.raises(itpp.ItppError) as e:
            g.load(bad)
        assert e.value.status == 9
    with pytest.raises(itpp.ItppError) as e:
        g.load(tmp_path / "missing.itpp")
    assert e.value.status == 9
    small = itpp.Propagator(H.n, H.gate_x, H.gate_z, H.alpha, dtau, delta, 10)
    with pytest.raises(itpp.ItppError) as e:       # more terms than its bound
        small.load(good)
    assert e.value.status == 9
    _same_bits(g.sorted_terms(), before, "a failed load leaves the state")
