"""Pauli-string Hamiltonians on L qubits: the spin chains of the paper's outlook.

The conclusions name OTOCs of sparse spin chains (such as those of
many-body-localisation studies) as the natural next use of the same GPU
machinery.  A spin Hamiltonian is a real combination of Pauli strings,
H = sum_t h_t P_t, which is also the form the supplement (Sec. I.A) uses to
store every operator.  The regularised OTOC is the F of Eq. (2) with the
Majoranas chi_a, chi_b replaced by two Pauli strings W and V, so the functions
of ``otoc`` (F_trace, F_state) apply unchanged with X = {0: W, 1: V}.

Encoding of one string by two L-bit masks (x, z): on qubit q,
  x_q = 0, z_q = 0 -> 1;   x_q = 1, z_q = 0 -> sigma_x;
  x_q = 0, z_q = 1 -> sigma_z;   x_q = 1, z_q = 1 -> sigma_y.
Conventions as in the rest of the oracle: qubit q is bit q of the basis index,
operators are Kronecker products op_{L-1} (x) ... (x) op_0, and
sigma_y = [[0, -i], [i, 0]].

Two independent constructions are given so that each checks the other:
dense Kronecker products of the 2x2 matrices, and per-basis-state maps built
from the single-qubit rules (sigma_x|b> = |1-b>, sigma_y|b> = i(-1)^b |1-b>,
sigma_z|b> = (-1)^b |b>).  Pinned by ``tests/test_oracle_spin.py``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

SIGMA = {
    "I": np.eye(2, dtype=np.complex128),
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


def letters(L: int, x: int, z: int) -> list:
    """Per-qubit letters of the string (x, z), index q = qubit q."""
    out = []
    for q in range(L):
        xb, zb = (x >> q) & 1, (z >> q) & 1
        out.append("Y" if xb and zb else "X" if xb else "Z" if zb else "I")
    return out


def pauli_dense(L: int, x: int, z: int) -> np.ndarray:
    """Dense 2^L x 2^L matrix of the string: op_{L-1} (x) ... (x) op_0."""
    M = np.ones((1, 1), dtype=np.complex128)
    for op in reversed(letters(L, x, z)):
        M = np.kron(M, SIGMA[op])
    return M


def dense_H(L: int, xs, zs, h) -> np.ndarray:
    """H = sum_t h_t P(x_t, z_t), dense."""
    H = np.zeros((1 << L, 1 << L), dtype=np.complex128)
    for x, z, c in zip(np.asarray(xs), np.asarray(zs), np.asarray(h)):
        H += float(c) * pauli_dense(L, int(x), int(z))
    return H


def apply_map(L: int, x: int, z: int, m):
    """P(x, z)|m> = ph |g> for basis states m (uint64 array), qubit by qubit.

    Returns (g, ph).  Qubit q of the state is read before that qubit's flip.
    """
    g = np.asarray(m, dtype=np.uint64).copy()
    ph = np.ones(g.shape, dtype=np.complex128)
    for q in range(L):
        xb, zb = (x >> q) & 1, (z >> q) & 1
        if not (xb or zb):
            continue
        bit = ((g >> np.uint64(q)) & np.uint64(1)).astype(np.int64)
        sgn = 1.0 - 2.0 * bit  # (-1)^b
        if xb and zb:  # sigma_y |b> = i (-1)^b |1 - b>
            ph = ph * (1j * sgn)
        elif zb:  # sigma_z |b> = (-1)^b |b>
            ph = ph * sgn
        if xb:
            g ^= np.uint64(1 << q)
    return g, ph


def csr_H(L: int, xs, zs, h) -> sp.csr_matrix:
    """H as CSR from the basis-state maps: H[g, m] += h ph for P|m> = ph|g>."""
    D = 1 << L
    cols = np.arange(D, dtype=np.uint64)
    rows, cc, vals = [], [], []
    for x, z, c in zip(np.asarray(xs), np.asarray(zs), np.asarray(h)):
        g, ph = apply_map(L, int(x), int(z), cols)
        rows.append(g.astype(np.int64))
        cc.append(cols.astype(np.int64))
        vals.append(float(c) * ph)
    if not rows:
        return sp.csr_matrix((D, D), dtype=np.complex128)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cc))), shape=(D, D))


def rows_of_Hpsi(L: int, xs, zs, h, m_rows, psi_at) -> np.ndarray:
    """Sampled rows (H psi)[m] for basis indices m_rows, from the definition.

    Each string maps |m> to ph|g>; being an involution up to a phase, it maps
    |g> back to ph'|m>, and <m|P|g> = ph'.  psi_at(g_array) returns psi at
    basis indices g.  Valid for L <= 63.
    """
    m_rows = np.asarray(m_rows, dtype=np.uint64)
    out = np.zeros(m_rows.shape, dtype=np.complex128)
    for x, z, c in zip(np.asarray(xs), np.asarray(zs), np.asarray(h)):
        g, _ = apply_map(L, int(x), int(z), m_rows)
        back, ph = apply_map(L, int(x), int(z), g)
        if not np.array_equal(back, m_rows):
            raise AssertionError("Pauli string is not an involution on basis states")
        out += float(c) * ph * psi_at(g)
    return out


def commute(x1: int, z1: int, x2: int, z2: int) -> bool:
    """Whether two Pauli strings commute: each qubit where they carry
    different non-identity letters contributes one sign flip; they commute
    when the number of such qubits is even (counted letter by letter)."""
    n = 0
    for q in range(64):
        a = ((x1 >> q) & 1, (z1 >> q) & 1)
        b = ((x2 >> q) & 1, (z2 >> q) & 1)
        if a != (0, 0) and b != (0, 0) and a != b:
            n += 1
    return n % 2 == 0
