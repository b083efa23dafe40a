"""One gate at the bench's full size, against the oracle on sampled strings.

The bench times the n = 64 chain at a bound of 2^26 terms with the top-M
select, in the library's default launch configuration.  At that size the
oracle cannot run the whole state in a test, but one gate only pairs a
string K with K.Q, so the oracle's value for K needs only K, K.Q and the
identity (whose partner Q is absent here).  The test therefore builds a
seeded state of exactly 2^26 strings with a known pair structure
(`workloads.paired_state`: strings that differ only in the gate's z bits),
runs the gate on the GPU over the whole state, runs the oracle over the
sub-state of 20k sampled pairs plus the identity (closed under the gate's
pairing, so every sampled output has the same value there as in the whole
state), and compares:

* every string the oracle keeps is on the GPU with identical coefficient
  bits, unless the top-M bound dropped it, in which case its magnitude is at
  most the smallest magnitude the GPU kept;
* every candidate string the oracle drops (below delta, or never produced)
  is absent on the GPU;
* the GPU keeps exactly 2^26 strings, with the identity at exactly 1.

The same check runs on the CPU with the oracle standing in for the GPU over
a small state, which pins the sub-state argument itself.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

PAIR_ZBITS = 0b11                 # the gate Z0 Z1 acts on z bits 0 and 1
DTAU, DELTA, ALPHA = 0.01, 1e-6, -1.0
FULL_M = 1 << 26
FULL_BASE = (FULL_M - 1) * 2 // 3  # 1 + n_base + n_base / 2 = 2^26 strings


def _gate():
    gx, gz = wl.two_site(64, 0, 1, "Z", "Z")
    assert int(gz[0]) == PAIR_ZBITS and int(gx[0]) == 0
    return gx, gz


def _oracle_on_sample(X, Z, C, base_row, pair_row, n_sample, seed):
    rng = np.random.default_rng(seed)
    js = rng.choice(base_row.shape[0], size=n_sample, replace=False)
    rows = np.concatenate([[0], base_row[js], pair_row[js][pair_row[js] >= 0]])
    gx, gz = _gate()
    o = oracle.Oracle(64, gx[None], gz[None], np.array([ALPHA]), DTAU, DELTA,
                      4 * rows.shape[0] + 16, 0)
    o.set_terms(X[rows], Z[rows], C[rows])
    o.apply_gate(0)
    # every string the sampled pairs can produce: the base and its pair key
    cand_x = np.concatenate([X[base_row[js], 0], X[base_row[js], 0]])
    cand_z = np.concatenate([Z[base_row[js], 0], Z[base_row[js], 0] | np.uint64(PAIR_ZBITS)])
    return o.terms(), (cand_x, cand_z)


def _lookup(sx, sz, qx, qz):
    """Rows of (qx, qz) in the canonically sorted (sx, sz), or -1.  A given x
    word occurs at most twice here (a base string and its pair key)."""
    lo = np.searchsorted(sx, qx, side="left")
    row = np.full(qx.shape[0], -1, dtype=np.int64)
    for off in (0, 1, 2):
        i = np.minimum(lo + off, sx.shape[0] - 1)
        hit = (lo + off < sx.shape[0]) & (sx[i] == qx) & (sz[i] == qz)
        row[hit] = i[hit]
    return row


def _check(got, M, expected, candidates):
    gx, gz, gc = got
    gx, gz = gx[:, 0], gz[:, 0]
    assert gc.shape[0] == M, f"{gc.shape[0]} strings kept, bound {M}"
    ident = (gx == 0) & (gz == 0)
    assert ident.sum() == 1 and gc[ident][0] == 1.0
    T = np.min(np.abs(gc))
    ex, ez, ec = expected
    ex, ez = ex[:, 0], ez[:, 0]
    keep = ~((ex == 0) & (ez == 0))
    ex, ez, ec = ex[keep], ez[keep], ec[keep]
    row = _lookup(gx, gz, ex, ez)
    found = row >= 0
    same = gc[row[found]].view(np.uint64) == ec[found].view(np.uint64)
    assert same.all(), f"{int((~same).sum())} of {int(found.sum())} sampled coefficients differ"
    dropped = ~found
    assert np.all(np.abs(ec[dropped]) <= T), "a string above the kept minimum is missing"
    # candidates the oracle does not keep must be absent
    cx, cz = candidates
    in_oracle = _lookup(ex, ez, cx, cz) >= 0
    assert np.all(_lookup(gx, gz, cx[~in_oracle], cz[~in_oracle]) < 0)
    return int(found.sum()), int(dropped.sum()), int((~in_oracle).sum())


def test_sub_state_argument_on_cpu():
    # oracle over the whole (small) state with the top-M bound = the "GPU"
    n_base = 3000
    X, Z, C, base_row, pair_row = wl.paired_state(n_base, 2601, PAIR_ZBITS)
    M = X.shape[0]
    gx, gz = _gate()
    whole = oracle.Oracle(64, gx[None], gz[None], np.array([ALPHA]), DTAU, DELTA, M, 1)
    whole.set_terms(X, Z, C)
    whole.apply_gate(0)
    expected, cand = _oracle_on_sample(X, Z, C, base_row, pair_row, 600, 7)
    kept, cut, absent = _check(whole.terms(), M, expected, cand)
    assert kept > 500 and cut > 10 and absent > 10


@pytest.mark.gpu
def test_full_size_gate_on_sampled_strings():
    itpp = pytest.importorskip("paper_2601_14400_gb300")
    X, Z, C, base_row, pair_row = wl.paired_state(FULL_BASE, 2601, PAIR_ZBITS)
    assert X.shape[0] == FULL_M
    gx, gz = _gate()
    # the bench's configuration: bound 2^26, top-M, default launch shapes
    g = itpp.Propagator(64, gx[None], gz[None], np.array([ALPHA]), DTAU, DELTA, FULL_M, 1)
    g.set_terms(X, Z, C)
    g.apply_gate(0)
    st = g.stats()
    assert st["cap_events"] == 1 and st["terms_in"] == FULL_M
    got = g.sorted_terms()
    expected, cand = _oracle_on_sample(X, Z, C, base_row, pair_row, 20000, 11)
    kept, cut, absent = _check(got, FULL_M, expected, cand)
    assert kept > 15000 and cut > 100 and absent > 100


def test_paired_state_structure():
    # the generator's promises the full-size check relies on, on a medium size
    n_base = 200_000
    X, Z, C, base_row, pair_row = wl.paired_state(n_base, 3, PAIR_ZBITS)
    N = X.shape[0]
    assert N == 1 + n_base + n_base // 2
    assert X[0, 0] == 0 and Z[0, 0] == 0 and C[0] == 1.0
    x, z = X[1:, 0], Z[1:, 0]
    assert np.all(x != 0)                                     # no second identity
    keys = np.stack([x, z], axis=1)
    assert np.unique(keys, axis=0).shape[0] == N - 1          # distinct strings
    bx = X[base_row, 0]
    assert np.unique(bx).shape[0] == n_base                   # x words distinct
    assert np.all(Z[base_row, 0] & np.uint64(PAIR_ZBITS) == 0)
    has = pair_row >= 0
    assert has.sum() == n_base // 2
    assert np.array_equal(X[pair_row[has], 0], bx[has])
    assert np.array_equal(Z[pair_row[has], 0], Z[base_row[has], 0] | np.uint64(PAIR_ZBITS))
    mags = np.abs(C[1:])
    assert mags.min() >= 1e-6 and mags.max() <= 1.0
