"""The sparse SYK Hamiltonian, Eq. (1) of the main text, in the chi-normalisation.

    H = sum_t J_t chi_{i_t} chi_{j_t} chi_{k_t} chi_{l_t},  i<j<k<l,

with {chi_m, chi_n} = delta_mn (the main text's normalisation); the
supplement's gamma = sqrt(2) chi with {gamma, gamma} = 2 delta gives the same
operator with J_gamma = J_chi / 4.  H is even in the Majoranas and therefore
block diagonal in fermion parity (supplement, parity-block formulas).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import majorana as mj


def dense_H(N: int, quads, J, rep: str) -> np.ndarray:
    """Full 2^{N/2} x 2^{N/2} Hamiltonian from dense Majorana matrices."""
    X = mj.chis(N, rep)
    dim = 1 << (N // 2)
    H = np.zeros((dim, dim), dtype=np.complex128)
    for (i, j, k, l), c in zip(np.asarray(quads), np.asarray(J)):
        H += c * (X[i] @ X[j] @ X[k] @ X[l])
    return H


def blocks(H: np.ndarray, N: int, rep: str):
    """(H_UU, H_DD) ordered by the block index m."""
    iU, iD = mj.block_indices(N, rep)
    return H[np.ix_(iU, iU)], H[np.ix_(iD, iD)]


def block_of(M: np.ndarray, N: int, rep: str, to_block: int, from_block: int):
    """Sub-matrix M[to, from] of a full-space operator, in block indices."""
    idx = mj.block_indices(N, rep)
    return M[np.ix_(idx[to_block], idx[from_block])]


def csr_block(N: int, quads, J, rep: str, block: int) -> sp.csr_matrix:
    """H_PP as a CSR matrix, built term by term from the basis-state maps.

    For each term and each basis state |f> of the block, chi chi chi chi |f>
    = ph |g>; that is the matrix element H[g, f] += J ph.  Duplicated (g, f)
    entries are summed by scipy.
    """
    q = N // 2
    L = q - 1
    D = 1 << L
    idx = mj.block_indices(N, rep)[block].astype(np.uint64)
    pos = np.full(1 << q, -1, dtype=np.int64)
    pos[idx.astype(np.int64)] = np.arange(D)
    rows, cols, vals = [], [], []
    for quad, c in zip(np.asarray(quads), np.asarray(J)):
        g, ph = mj.apply_product_map(quad, N, rep, idx)
        r = pos[g.astype(np.int64)]
        if np.any(r < 0):
            raise AssertionError("term left the parity block")
        rows.append(r)
        cols.append(np.arange(D))
        vals.append(c * ph)
    if not rows:
        return sp.csr_matrix((D, D), dtype=np.complex128)
    return sp.csr_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(D, D)
    )


def rows_of_Hpsi(N: int, quads, J, rep: str, block: int, m_rows, psi_at):
    """Sampled rows (H_PP psi)[m] for block indices m_rows, from the definition.

    Row m of the block is the full-space basis state f; each term P maps f to
    a single basis state g (P^2 is a multiple of 1), and <f|P|g> is the phase
    of P|g> = ph |f>.  psi_at(block, m_array) returns psi values of the block
    at block indices m.  Valid for any N <= 64 (indices in uint64).
    """
    q = N // 2
    L = q - 1
    D = np.uint64(1 << L)
    m_rows = np.asarray(m_rows, dtype=np.uint64)
    topbit = np.uint64(1 << L)
    if rep == "paper":
        f = m_rows | (topbit if block else np.uint64(0))
    else:
        par = (np.bitwise_count(m_rows) & np.uint8(1)).astype(np.uint64)
        f = m_rows | (((par ^ np.uint64(block)) & np.uint64(1)) << np.uint64(L))
    out = np.zeros(m_rows.shape, dtype=np.complex128)
    for quad, c in zip(np.asarray(quads), np.asarray(J)):
        g, _ = mj.apply_product_map(quad, N, rep, f)
        back, ph = mj.apply_product_map(quad, N, rep, g)
        if not np.array_equal(back, f):
            raise AssertionError("term is not an involution on basis states")
        gm = g & (D - np.uint64(1))
        out += c * ph * psi_at(block, gm)
    return out
