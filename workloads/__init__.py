"""Seeded, synthetic inputs shared by the tests, the bench and the smoke check.

This module builds *inputs only*: Hamiltonians as ordered lists of Pauli-string
gates with real coefficients, observables, and synthetic Pauli-sum states. It
holds none of the propagation arithmetic (no commutation tests, no products,
no weights); both the CUDA library and the CPU oracle receive these arrays and
do their own work on them.

Conventions (the bit layout of a Pauli string, Sec. II.B "bitstring
representation" in the introduction and Eq. (Observable_Pauli)):

* A string on ``n`` sites is a pair of masks ``(x, z)`` of ``W = ceil(n/64)``
  uint64 words each; site ``i`` is bit ``i % 64`` of word ``i // 64``.
  ``(x_i, z_i) = (0,0) I, (1,0) X, (0,1) Z, (1,1) Y``; the phase is the
  Hermitian one (``Y`` itself, not ``XZ``).
* A Hamiltonian ``H = sum_k alpha_k Q_k`` is given in Trotter order as arrays
  ``gate_x[n_gates, W]``, ``gate_z[n_gates, W]`` and ``alpha[n_gates]``.
  The transverse-field Ising model of Eq. (TFIM) is
  ``H = -J sum Z_i Z_{i+1} - h sum X_i``, so ``alpha = -J`` on bonds and
  ``alpha = -h`` on fields.
* Trotter order inside a layer (Algorithm 1 leaves it to the user): ZZ bonds
  first, then X fields.  1D: bonds ``(i, i+1)`` for ``i = 0..n-2``, the
  periodic bond ``(n-1, 0)`` last, then ``X_0..X_{n-1}``.  2D ``L x L`` (site
  ``r*L + c``): horizontal bonds row-major, vertical bonds row-major, then
  ``X`` row-major.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Hamiltonian", "n_words", "single_site", "two_site", "tfim_1d", "tfim_2d",
    "random_pauli_hamiltonian", "Observable", "energy_observable",
    "x_observables", "zz_observables", "synthetic_state", "WORKLOADS",
    "Workload", "batch_field_sweep", "adjoint_chain",
]


def n_words(n: int) -> int:
    """Words per mask for ``n`` sites (site ``i`` -> word ``i // 64``)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    return (n + 63) // 64


def _empty(count: int, W: int):
    return (np.zeros((count, W), dtype=np.uint64),
            np.zeros((count, W), dtype=np.uint64))


def _set_bit(mask_row: np.ndarray, site: int) -> None:
    mask_row[site // 64] |= np.uint64(1) << np.uint64(site % 64)


def single_site(n: int, site: int, letter: str):
    """(x, z) rows of one single-site Pauli ``letter`` in {X, Y, Z}."""
    W = n_words(n)
    x = np.zeros(W, dtype=np.uint64)
    z = np.zeros(W, dtype=np.uint64)
    if letter in ("X", "Y"):
        _set_bit(x, site)
    if letter in ("Z", "Y"):
        _set_bit(z, site)
    return x, z


def two_site(n: int, a: int, b: int, la: str, lb: str):
    xa, za = single_site(n, a, la)
    xb, zb = single_site(n, b, lb)
    return xa | xb, za | zb


@dataclass
class Hamiltonian:
    """Ordered gate list of a Pauli Hamiltonian ``sum_k alpha_k Q_k``."""
    n: int
    gate_x: np.ndarray          # (n_gates, W) uint64
    gate_z: np.ndarray          # (n_gates, W) uint64
    alpha: np.ndarray           # (n_gates,) float64
    labels: list = field(default_factory=list)   # human-readable, optional
    param: np.ndarray | None = None  # (n_gates,) int: parameter index of each gate

    @property
    def W(self) -> int:
        return n_words(self.n)

    @property
    def n_gates(self) -> int:
        return int(self.alpha.shape[0])


def tfim_1d(n: int, J=1.0, h=1.0, periodic: bool = False) -> Hamiltonian:
    """1D TFIM of Eq. (TFIM); ``J`` and ``h`` may be scalars or per-bond /
    per-site arrays (``len(J) = n-1`` open, ``n`` periodic; ``len(h) = n``).

    ``param`` numbers the couplings first (bond ``i`` -> ``i``) and then the
    fields (site ``i`` -> ``n_bonds + i``): the order of the gradient vector
    of the adjoint extension.
    """
    n_bonds = (n if periodic else n - 1) if n > 1 else 0
    if periodic and n < 3:
        raise ValueError("periodic chain needs n >= 3")
    Jv = np.broadcast_to(np.asarray(J, dtype=np.float64), (n_bonds,)).copy()
    hv = np.broadcast_to(np.asarray(h, dtype=np.float64), (n,)).copy()
    W = n_words(n)
    gx, gz = _empty(n_bonds + n, W)
    alpha = np.empty(n_bonds + n)
    labels, param = [], []
    k = 0
    for i in range(n_bonds):
        j = (i + 1) % n
        gx[k], gz[k] = two_site(n, i, j, "Z", "Z")
        alpha[k] = -Jv[i]
        labels.append(f"Z{i}Z{j}")
        param.append(i)
        k += 1
    for i in range(n):
        gx[k], gz[k] = single_site(n, i, "X")
        alpha[k] = -hv[i]
        labels.append(f"X{i}")
        param.append(n_bonds + i)
        k += 1
    return Hamiltonian(n, gx, gz, alpha, labels, np.asarray(param, dtype=np.int32))


def tfim_2d(L: int, J=1.0, h=1.0) -> Hamiltonian:
    """2D TFIM on an open ``L x L`` square lattice (site ``r*L + c``)."""
    n = L * L
    bonds = [(r * L + c, r * L + c + 1) for r in range(L) for c in range(L - 1)]
    bonds += [(r * L + c, (r + 1) * L + c) for r in range(L - 1) for c in range(L)]
    W = n_words(n)
    gx, gz = _empty(len(bonds) + n, W)
    alpha = np.empty(len(bonds) + n)
    labels, param = [], []
    for k, (a, b) in enumerate(bonds):
        gx[k], gz[k] = two_site(n, a, b, "Z", "Z")
        alpha[k] = -float(J)
        labels.append(f"Z{a}Z{b}")
        param.append(k)
    for i in range(n):
        k = len(bonds) + i
        gx[k], gz[k] = single_site(n, i, "X")
        alpha[k] = -float(h)
        labels.append(f"X{i}")
        param.append(k)
    return Hamiltonian(n, gx, gz, alpha, labels, np.asarray(param, dtype=np.int32))


def strang_schedule(H: Hamiltonian) -> Hamiltonian:
    """The symmetric second-order product of a Trotter layer (Sec. II.C,
    Strang splitting) written out as a gate list: terms 1..G-1 with half
    coefficients, term G whole, then terms G-1..1 with half coefficients."""
    G = H.n_gates
    if G < 2:
        return H
    idx = list(range(G - 1)) + [G - 1] + list(range(G - 2, -1, -1))
    scale = np.array([0.5] * (G - 1) + [1.0] + [0.5] * (G - 1))
    return Hamiltonian(H.n, H.gate_x[idx].copy(), H.gate_z[idx].copy(),
                       np.asarray(H.alpha, dtype=np.float64)[idx] * scale,
                       [H.labels[i] for i in idx] if H.labels else [],
                       H.param[idx] if H.param is not None else None)


def random_pauli_hamiltonian(n: int, n_terms: int, seed: int,
                             max_weight: int | None = None) -> Hamiltonian:
    """Random non-identity Pauli strings, letters uniform in {X, Y, Z} on a
    random set of sites, with ``alpha ~ U[-1, 1]``."""
    rng = np.random.default_rng(seed)
    W = n_words(n)
    gx, gz = _empty(n_terms, W)
    alpha = rng.uniform(-1.0, 1.0, n_terms)
    mw = n if max_weight is None else min(max_weight, n)
    for k in range(n_terms):
        wgt = int(rng.integers(1, mw + 1))
        for s in rng.choice(n, size=wgt, replace=False):
            letter = "XYZ"[int(rng.integers(0, 3))]
            x, z = single_site(n, int(s), letter)
            gx[k] |= x
            gz[k] |= z
    return Hamiltonian(n, gx, gz, alpha, [f"R{k}" for k in range(n_terms)],
                       np.arange(n_terms, dtype=np.int32))


@dataclass
class Observable:
    """Sparse Pauli sum ``O = sum_j w_j P_j`` (Eq. (Observable_Pauli))."""
    n: int
    x: np.ndarray   # (m, W) uint64
    z: np.ndarray   # (m, W) uint64
    w: np.ndarray   # (m,) float64
    labels: list = field(default_factory=list)


def energy_observable(H: Hamiltonian) -> Observable:
    """``H`` itself as an observable (weights ``alpha_k``)."""
    return Observable(H.n, H.gate_x.copy(), H.gate_z.copy(), H.alpha.copy(),
                      list(H.labels))


def x_observables(n: int) -> list:
    out = []
    for i in range(n):
        x, z = single_site(n, i, "X")
        out.append(Observable(n, x[None], z[None], np.ones(1), [f"X{i}"]))
    return out


def zz_observables(n: int, pairs) -> list:
    out = []
    for a, b in pairs:
        x, z = two_site(n, a, b, "Z", "Z")
        out.append(Observable(n, x[None], z[None], np.ones(1), [f"Z{a}Z{b}"]))
    return out


def stack_observables(obs: list) -> Observable:
    """Concatenate single observables (used to read many coefficients at once)."""
    n = obs[0].n
    return Observable(n, np.concatenate([o.x for o in obs]),
                      np.concatenate([o.z for o in obs]),
                      np.concatenate([o.w for o in obs]),
                      sum((o.labels for o in obs), []))


def _row_parity(a: np.ndarray) -> np.ndarray:
    """Parity of the popcount of each row of a (rows, W) uint64 array."""
    v = np.bitwise_xor.reduce(a, axis=1)
    for sh in (32, 16, 8, 4, 2, 1):
        v ^= v >> np.uint64(sh)
    return (v & np.uint64(1)).astype(bool)


def _lowest_set_bit(a: np.ndarray) -> np.ndarray:
    """Per row, a (rows, W) mask holding only the lowest set bit of the row."""
    out = np.zeros_like(a)
    done = np.zeros(a.shape[0], dtype=bool)
    for w in range(a.shape[1]):
        col = a[:, w]
        lb = col & (~col + np.uint64(1))
        take = (~done) & (col != 0)
        out[take, w] = lb[take]
        done |= take
    return out


def _first_occurrences(rows: np.ndarray) -> np.ndarray:
    """Sorted indices of the first occurrence of every distinct row: rows are
    grouped by a 64-bit mix of their words, and only rows whose mix repeats
    are compared in full (same result as ``np.unique(axis=0)``'s first
    indices, without sorting whole rows)."""
    h = np.zeros(rows.shape[0], dtype=np.uint64)
    with np.errstate(over="ignore"):
        for j in range(rows.shape[1]):
            h ^= rows[:, j] * np.uint64(0x9E3779B97F4A7C15 + 2 * j)
            h ^= h >> np.uint64(29)
            h *= np.uint64(0xBF58476D1CE4E5B9)
    order = np.argsort(h, kind="stable")
    hs = h[order]
    rep = np.zeros(rows.shape[0], dtype=bool)
    eq = hs[1:] == hs[:-1]
    rep[1:] |= eq
    rep[:-1] |= eq
    keep = np.ones(rows.shape[0], dtype=bool)
    if rep.any():
        sub = np.sort(order[rep])                      # rows whose mix repeats
        _, first = np.unique(rows[sub], axis=0, return_index=True)
        keep[sub] = False
        keep[sub[first]] = True
    return np.flatnonzero(keep)


def synthetic_state(n: int, M: int, seed: int, delta: float = 1e-6):
    """``M`` distinct random non-identity strings in the TFIM sector, plus
    the identity.

    Sector: bits ``>= n`` clear, ``popc(z)`` even, ``popc(x & z)`` even (the
    strings a real, spin-flip-symmetric density matrix of Eq. (TFIM) can
    hold).  Coefficients: uniform sign, ``|c|`` log-uniform in
    ``[delta, 1]``; the identity (all-zero key) is entry 0 with ``c = 1``.
    Returns ``(x, z, c)`` with shapes ``(M+1, W)``, ``(M+1, W)``, ``(M+1,)``,
    rows in random order after the identity.
    """
    rng = np.random.default_rng(seed)
    W = n_words(n)
    top = np.full(W, ~np.uint64(0), dtype=np.uint64)
    if n % 64:
        top[-1] = (np.uint64(1) << np.uint64(n % 64)) - np.uint64(1)
    if n < 64 and M > 4 ** n // 4:
        raise ValueError("too many strings requested for this n")
    keys = np.zeros((0, 2 * W), dtype=np.uint64)
    while keys.shape[0] < M:
        k = int(1.2 * (M - keys.shape[0])) + 64
        x = rng.integers(0, 2**64, size=(k, W), dtype=np.uint64) & top
        z = rng.integers(0, 2**64, size=(k, W), dtype=np.uint64) & top
        z[_row_parity(z), 0] ^= np.uint64(1)          # popc(z) even
        odd = _row_parity(x & z)                      # flip x where z is set
        x[odd] ^= _lowest_set_bit(z[odd])
        cand = np.concatenate([keys, np.concatenate([x, z], axis=1)])
        cand = cand[cand.any(axis=1)]                 # drop the identity
        keys = cand[_first_occurrences(cand)]
    keys = keys[:M]
    keys = keys[rng.permutation(M)]
    X = np.zeros((M + 1, W), dtype=np.uint64)
    Z = np.zeros((M + 1, W), dtype=np.uint64)
    X[1:] = keys[:, :W]
    Z[1:] = keys[:, W:]
    mag = np.exp(rng.uniform(math.log(delta), 0.0, M))
    sgn = np.where(rng.integers(0, 2, M) == 1, 1.0, -1.0)
    C = np.empty(M + 1)
    C[0] = 1.0
    C[1:] = sgn * mag
    return X, Z, C


def paired_state(n_base: int, seed: int, pair_zbits: int, pair_every: int = 2,
                 delta: float = 1e-6):
    """A large n = 64 state with a known pair structure, built without any
    deduplication (full-size single-gate checks).

    Base string j (j = 1..n_base): x = j * A mod 2^64 with A odd, so the x
    words alone are distinct and nonzero; z = j * B + D mod 2^64 with the bits
    of ``pair_zbits`` cleared.  Every ``pair_every``-th base string (j a
    multiple of it) also appears with those z bits set: the two rows differ
    only there, and no other row shares their x word.  Coefficients: sign
    uniform, ``|c|`` log-uniform in ``[delta, 1]``; the identity (c = 1) is
    row 0.  Returns ``(x, z, c, base_row, pair_row)``: x, z of shape
    ``(N, 1)``, and for base string j (index j - 1) its row and its pair's
    row (-1 when absent).
    """
    rng = np.random.default_rng(seed)
    A = np.uint64(0x9E3779B97F4A7C15)
    B = np.uint64(0xC2B2AE3D27D4EB4F)
    D = np.uint64(0x165667B19E3779F9)
    j = np.arange(1, n_base + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        bx = j * A
        bz = (j * B + D) & ~np.uint64(pair_zbits)
    paired = (j % np.uint64(pair_every)) == 0
    n_pair = int(paired.sum())
    N = 1 + n_base + n_pair
    X = np.zeros((N, 1), dtype=np.uint64)
    Z = np.zeros((N, 1), dtype=np.uint64)
    X[1:n_base + 1, 0] = bx
    Z[1:n_base + 1, 0] = bz
    X[n_base + 1:, 0] = bx[paired]
    Z[n_base + 1:, 0] = bz[paired] | np.uint64(pair_zbits)
    base_row = np.arange(1, n_base + 1, dtype=np.int64)
    pair_row = np.full(n_base, -1, dtype=np.int64)
    pair_row[paired] = np.arange(n_base + 1, N, dtype=np.int64)
    mag = np.exp(rng.uniform(math.log(delta), 0.0, N - 1))
    sgn = np.where(rng.integers(0, 2, N - 1) == 1, 1.0, -1.0)
    C = np.empty(N)
    C[0] = 1.0
    C[1:] = sgn * mag
    return X, Z, C, base_row, pair_row


# --------------------------------------------------------------------------
# The workloads the library is measured and checked on.
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    H: Hamiltonian
    dtau: float
    n_layers: int
    delta: float
    cap_M: int
    cap_policy: int          # 0 = error when exceeded, 1 = keep the top-M
    observables: dict
    note: str = ""


def _tfim1d_workload(name, n, J, h, periodic, dtau, n_layers, delta, cap_M,
                     cap_policy, zz_pairs, note):
    H = tfim_1d(n, J, h, periodic)
    obs = {"energy": energy_observable(H)}
    for o in x_observables(n):
        obs[o.labels[0]] = o
    for o in zz_observables(n, zz_pairs):
        obs[o.labels[0]] = o
    return Workload(name, H, dtau, n_layers, delta, cap_M, cap_policy, obs, note)


def batch_field_sweep(seed: int = 14400, B: int = 64):
    """64 open TFIM chains: ``n ~ U{16..64}``, ``h ~ U[0.5, 2]``, J = 1."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(16, 65, B)
    hs = rng.uniform(0.5, 2.0, B)
    return [int(v) for v in ns], [float(v) for v in hs]


def adjoint_chain(n: int = 32, seed: int = 1440):
    """Open chain with per-site fields ``h_i ~ U[0.8, 1.2]`` and couplings
    ``J_i ~ U[0.9, 1.1]`` (fields drawn first)."""
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.8, 1.2, n)
    J = rng.uniform(0.9, 1.1, n - 1)
    return tfim_1d(n, J, h, periodic=False)


def _build_workloads():
    w = {}
    w["tfim1d_n8_open"] = _tfim1d_workload(
        "tfim1d_n8_open", 8, 1.0, 1.0, False, 0.05, 20, 1e-8, 1 << 16, 0,
        [(i, i + 1) for i in range(7)],
        "n=8 open chain, J=h=1, dtau=0.05, 20 layers (beta=1), |c|<=1e-8 dropped")
    w["tfim1d_n64_periodic"] = _tfim1d_workload(
        "tfim1d_n64_periodic", 64, 1.0, 1.0, True, 0.01, 200, 1e-6, 1 << 26, 1,
        [(0, 1)],
        "n=64 periodic chain at h=J (critical), dtau=0.01, 200 layers (beta=2), "
        "|c|<=1e-6 dropped, at most 2^26 terms kept (top-M)")
    H2 = tfim_2d(11, 1.0, 3.04)
    obs2 = {"energy": energy_observable(H2)}
    c = 5 * 11 + 5
    for o in zz_observables(121, [(c, c + 1), (c, c + 11)]):
        obs2[o.labels[0]] = o
    w["tfim2d_11x11"] = Workload(
        "tfim2d_11x11", H2, 0.02, 30, 1e-5, 1 << 28, 1, obs2,
        "11x11 open square lattice, J=1, h=3.04, dtau=0.02, 30 layers (beta=0.6), "
        "|c|<=1e-5 dropped; the threshold alone exceeds 2^29 terms by the third "
        "layer, so at most 2^28 terms are kept (top-M)")
    Ha = adjoint_chain()
    obsa = {"energy": energy_observable(Ha)}
    for o in zz_observables(32, [(15, 16)]):
        obsa[o.labels[0]] = o
    w["adjoint_n32"] = Workload(
        "adjoint_n32", Ha, 0.02, 50, 1e-7, 1 << 20, 1, obsa,
        "n=32 open chain, h_i~U[0.8,1.2], J_i~U[0.9,1.1], dtau=0.02, 50 layers, "
        "|c|<=1e-7 dropped; the threshold alone passes 4.6e7 terms by layer 5 and "
        "2^27 by layer 7, so at most 2^20 terms are kept (top-M; the frozen support "
        "of a step is its kept set)")
    return w


WORKLOADS = _build_workloads()
