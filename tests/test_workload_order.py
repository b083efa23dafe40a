"""The gate order and weights of the TFIM workloads: the reading of the
Trotter order within a layer (ZZ bonds first, then X fields; the periodic
bond last among the bonds; 2D horizontal bonds row-major, then vertical
bonds row-major, then fields row-major) and of the sign of alpha (bonds -J,
fields -h).  The oracle and the GPU both take this list as input, so a
silent reordering would change every result; this pins it to the reading by
decoding each gate string back to its sites and letters.
"""
import numpy as np

import workloads as wl


def _letters(H, k):
    out = []
    for site in range(H.n):
        w, b = divmod(site, 64)
        x = (int(H.gate_x[k, w]) >> b) & 1
        z = (int(H.gate_z[k, w]) >> b) & 1
        if x or z:
            out.append((site, "IXZY"[x + 2 * z]))
    return out


def test_tfim_1d_order_and_signs():
    for n, periodic in [(8, False), (64, True), (65, True), (130, False)]:
        H = wl.tfim_1d(n, 1.3, 0.7, periodic=periodic)
        n_bonds = n if periodic else n - 1
        assert H.gate_x.shape[0] == n_bonds + n
        for k in range(n_bonds):
            assert _letters(H, k) == sorted([(k, "Z"), ((k + 1) % n, "Z")])
            assert H.alpha[k] == -1.3
        for i in range(n):
            assert _letters(H, n_bonds + i) == [(i, "X")]
            assert H.alpha[n_bonds + i] == -0.7
    assert wl.tfim_1d(64, periodic=True).gate_x.shape[0] == 128   # the bench layer


def test_tfim_2d_order_and_signs():
    L = 11
    H = wl.tfim_2d(L, 1.0, 3.04)
    n = L * L
    horiz = [(r * L + c, r * L + c + 1) for r in range(L) for c in range(L - 1)]
    vert = [(r * L + c, (r + 1) * L + c) for r in range(L - 1) for c in range(L)]
    assert len(horiz) + len(vert) == 220 and H.gate_x.shape[0] == 341
    for k, (a, b) in enumerate(horiz + vert):
        assert _letters(H, k) == [(a, "Z"), (b, "Z")]
        assert H.alpha[k] == -1.0
    for i in range(n):
        assert _letters(H, 220 + i) == [(i, "X")]
        assert H.alpha[220 + i] == -3.04
    assert H.W == 2
    top = np.uint64(121 - 64)          # bits >= 121 of the second word are clear
    assert np.all(H.gate_x[:, 1] >> top == 0) and np.all(H.gate_z[:, 1] >> top == 0)
