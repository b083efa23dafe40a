"""Comparison helpers for the GPU-vs-oracle parity tests."""
import numpy as np


def sort_terms(x, z, c):
    """Ascending key order: x words, then z words (the oracle's order)."""
    W = x.shape[1]
    keys = tuple(z[:, w] for w in range(W - 1, -1, -1)) + tuple(x[:, w] for w in range(W - 1, -1, -1))
    order = np.lexsort(keys)
    return x[order], z[order], c[order]


def assert_same_state(gpu, ora, what=""):
    """Bit-exact: identical string sets and identical coefficient bits."""
    gx, gz, gc = sort_terms(*gpu)
    ox, oz, oc = ora
    assert gx.shape == ox.shape, f"{what}: {gx.shape[0]} GPU terms vs {ox.shape[0]} oracle terms"
    assert np.array_equal(gx, ox) and np.array_equal(gz, oz), f"{what}: string sets differ"
    same = gc.view(np.uint64) == oc.view(np.uint64)
    if not same.all():
        i = int(np.argmin(same))
        rel = np.max(np.abs(gc - oc) / np.maximum(np.abs(oc), 1e-300))
        raise AssertionError(f"{what}: {int((~same).sum())} coefficients differ in bits; "
                             f"first at {i}: {gc[i]!r} vs {oc[i]!r}; max rel {rel:.3e}")


def rel_close(a, b, tol=1e-10, scale=None):
    s = max(abs(b), 1e-300) if scale is None else max(scale, 1e-300)
    return abs(a - b) <= tol * s
