"""Dense-matrix references for small systems -- TEST INFRASTRUCTURE ONLY.

These are the definitions the propagated operator must reproduce, written
with plain matrices (no Pauli-string bookkeeping at all):

* ``trotter_rho`` -- the Trotterised thermal operator of Eq. (ThermalTrotter):
  every gate is ``V_k = expm(-(theta_k/2) Q_k)`` with ``theta_k = alpha_k dtau``
  (the first-order product of Sec. II.C), and Algorithm 1 applies
  ``rho <- V_k^dagger rho V_k`` gate after gate starting from ``rho = I``.
* ``pauli_coefficients`` -- Eq. (Observable_Pauli) inverted:
  ``c_P = Tr(P rho) / Tr(rho)`` (``Tr(P_a P_b) = 2^n delta_ab``), i.e. the
  expansion normalised so that the identity coefficient is one.
* ``thermal_expect`` -- Eq. (Expectation_Value) with ``beta`` the inverse
  temperature, by exact diagonalisation.
* ``bdg_energy`` -- the exact thermal energy of the open TFIM chain from free
  fermions (the Bogoliubov-de Gennes solution the paper benchmarks against,
  Sec. III).
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.linalg as sla

_I = np.eye(2, dtype=complex)
_X = np.array([[0, 1], [1, 0]], dtype=complex)
_Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
_Z = np.array([[1, 0], [0, -1]], dtype=complex)


def _bit(row, site):
    return (int(row[site // 64]) >> (site % 64)) & 1


def pauli_dense(x_row, z_row, n):
    """Dense 2^n x 2^n matrix of the string (x, z); site 0 is the leftmost
    tensor factor.  (x_i, z_i) = (1, 1) is Y itself."""
    M = np.ones((1, 1), dtype=complex)
    for i in range(n):
        a, b = _bit(x_row, i), _bit(z_row, i)
        s = {(0, 0): _I, (1, 0): _X, (0, 1): _Z, (1, 1): _Y}[(a, b)]
        M = np.kron(M, s)
    return M


def all_strings(n):
    """Every (x, z) pair of masks on n <= 64 sites, as (4^n, 1) arrays."""
    xs, zs = [], []
    for xv, zv in itertools.product(range(2 ** n), range(2 ** n)):
        xs.append(xv)
        zs.append(zv)
    return (np.asarray(xs, dtype=np.uint64)[:, None],
            np.asarray(zs, dtype=np.uint64)[:, None])


def hamiltonian_dense(H):
    D = 2 ** H.n
    M = np.zeros((D, D), dtype=complex)
    for k in range(H.n_gates):
        M += H.alpha[k] * pauli_dense(H.gate_x[k], H.gate_z[k], H.n)
    return M


def trotter_rho(H, dtau, n_layers, rho0=None, gates=None):
    """rho after ``n_layers`` layers of ``rho <- V_k^dagger rho V_k`` over the
    gates in order (``gates`` restricts to a prefix list of gate indices for
    a single layer).  Starts from the identity unless ``rho0`` is given."""
    D = 2 ** H.n
    rho = np.eye(D, dtype=complex) if rho0 is None else rho0.astype(complex)
    order = list(range(H.n_gates)) if gates is None else list(gates)
    Vs = [sla.expm(-0.5 * H.alpha[k] * dtau * pauli_dense(H.gate_x[k], H.gate_z[k], H.n))
          for k in range(H.n_gates)]
    for _ in range(n_layers):
        for k in order:
            V = Vs[k]
            rho = V.conj().T @ rho @ V
    return rho


def trotter_rho_weight_cut(H, dtau, n_layers, k):
    """The Trotter evolution with the Pauli weight cutoff of Sec. II.B after
    every gate, done on dense matrices: after each ``rho <- V^dagger rho V``
    the operator is projected onto the strings of weight <= k,
    ``rho <- sum_{w(P) <= k} Tr(P rho) / 2^n P``, then scaled to unit trace
    coefficient.  Brute force for small n (4^n projections per gate)."""
    D = 2 ** H.n
    xs, zs = all_strings(H.n)
    basis = [pauli_dense(xs[i], zs[i], H.n) for i in range(xs.shape[0])
             if sum(bin(int(a) | int(b)).count("1") for a, b in zip(xs[i], zs[i])) <= k]
    Vs = [sla.expm(-0.5 * H.alpha[j] * dtau * pauli_dense(H.gate_x[j], H.gate_z[j], H.n))
          for j in range(H.n_gates)]
    rho = np.eye(D, dtype=complex)
    for _ in range(n_layers):
        for V in Vs:
            rho = V.conj().T @ rho @ V
            proj = np.zeros_like(rho)
            for P in basis:
                proj += (np.trace(P @ rho) / D) * P
            rho = proj / (np.trace(proj) / D)
    return rho


def pauli_coefficients(rho, n):
    """{(x, z): c_P} for every string, c_P = Tr(P rho) / Tr(rho)."""
    tr = np.trace(rho)
    out = {}
    xs, zs = all_strings(n)
    for i in range(xs.shape[0]):
        P = pauli_dense(xs[i], zs[i], n)
        out[(int(xs[i, 0]), int(zs[i, 0]))] = np.trace(P @ rho) / tr
    return out


def thermal_expect(H, beta, O):
    """Tr[O e^{-beta H}] / Tr[e^{-beta H}] by exact diagonalisation."""
    Hd = hamiltonian_dense(H)
    w, U = np.linalg.eigh(Hd)
    p = np.exp(-beta * (w - w.min()))
    p /= p.sum()
    Od = np.zeros_like(Hd)
    for j in range(O.x.shape[0]):
        Od += O.w[j] * pauli_dense(O.x[j], O.z[j], H.n)
    Odiag = np.real(np.einsum("ij,ik,kj->j", U.conj(), Od, U))
    return float(p @ Odiag)


def bdg_energy(J, h, beta):
    """Thermal energy of H = -sum J_i Z_i Z_{i+1} - sum h_i X_i (open chain).

    A Jordan-Wigner map built on the X basis turns H into a free Majorana
    quadratic form with ``X_i ~ i g_{2i} g_{2i+1}`` and
    ``Z_i Z_{i+1} ~ i g_{2i+1} g_{2i+2}``; its mode energies are twice the
    singular values ``s_k`` of the bidiagonal matrix with ``h_i`` on the
    diagonal and ``J_i`` above it, and
    ``<H>_beta = - sum_k s_k tanh(beta s_k)``.
    """
    h = np.asarray(h, dtype=float)
    n = h.shape[0]
    J = np.broadcast_to(np.asarray(J, dtype=float), (n - 1,))
    M = np.diag(h) + np.diag(J, 1)
    s = np.linalg.svd(M, compute_uv=False)
    return float(-np.sum(s * np.tanh(beta * s)))


def bdg_ground_energy(J, h):
    h = np.asarray(h, dtype=float)
    n = h.shape[0]
    J = np.broadcast_to(np.asarray(J, dtype=float), (n - 1,))
    s = np.linalg.svd(np.diag(h) + np.diag(J, 1), compute_uv=False)
    return float(-np.sum(s))


def binom(a, b):
    return math.comb(a, b)
