"""Non-Hermitian sparse SYK: the other model the paper's conclusions name for
OTOC studies.

Reading (the paper gives no formula): the couplings of Eq. (1) become complex,
    H = sum_t (J_t + i M_t) chi_i chi_j chi_k chi_l,
so H^dagger = sum_t (J_t - i M_t) chi chi chi chi (a product of four distinct
Majoranas is Hermitian).  Time evolution e^{-iHt} is no longer unitary, and a
Heisenberg-picture operator is W(t) = e^{iH^dagger t} W e^{-iHt}, which is the
usual W(t) when H is Hermitian.  The OTOC is Eq. (2) at infinite temperature
(beta = 0: e^{-beta H} is not a density matrix for non-Hermitian H) with this
W(t):
    F_psi(t) = <psi| e^{iH^dag t} chi_a e^{-iHt} chi_b e^{iH^dag t} chi_a e^{-iHt} chi_b |psi>,
    F_tr(t)  = Tr[e^{iH^dag t} chi_a e^{-iHt} chi_b e^{iH^dag t} chi_a e^{-iHt} chi_b] / dim.
With M = 0 these are the beta = 0 forms of ``otoc``.

Exact evolution of a non-Hermitian matrix uses scipy.linalg.expm (Pade
approximation with scaling and squaring, Al-Mohy & Higham 2009) on the dense
matrix, or scipy.sparse.linalg.expm_multiply on the CSR form.  Pinned by
``tests/test_oracle_nonherm.py``.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from . import hamiltonian as ham


def couplings(J_re, J_im) -> np.ndarray:
    return np.asarray(J_re, dtype=np.float64) + 1j * np.asarray(J_im, dtype=np.float64)


def dense_H(N: int, quads, J_re, J_im, rep: str) -> np.ndarray:
    """Full 2^{N/2} x 2^{N/2} matrix of sum_t (J_t + i M_t) chi chi chi chi."""
    return ham.dense_H(N, quads, couplings(J_re, J_im), rep)


def csr_block(N: int, quads, J_re, J_im, rep: str, block: int):
    """H_PP of the parity block as CSR (basis-state maps, complex couplings)."""
    return ham.csr_block(N, quads, couplings(J_re, J_im), rep, block)


def evolve(H, z, x) -> np.ndarray:
    """e^{-zH} x for a dense (non-Hermitian) H."""
    return sla.expm(-complex(z) * np.asarray(H, dtype=np.complex128)) @ np.asarray(x, dtype=np.complex128)


def evolve_sparse(Hcsr, z, x) -> np.ndarray:
    return spla.expm_multiply((-complex(z)) * Hcsr.astype(np.complex128), np.asarray(x, dtype=np.complex128))


def _chain(H, Xa, Xb, t):
    U = sla.expm(-1j * t * H)                 # e^{-iHt}
    Ub = sla.expm(1j * t * H.conj().T)        # e^{iH^dag t}
    return Ub, U, Ub @ Xa @ U @ Xb @ Ub @ Xa @ U @ Xb


def F_state(H, X, a: int, b: int, ts, psi) -> np.ndarray:
    """F_psi(t) on the full space for one state (beta = 0)."""
    psi = np.asarray(psi, dtype=np.complex128)
    return np.array([np.vdot(psi, _chain(H, X[a], X[b], t)[2] @ psi) for t in np.asarray(ts, np.float64)])


def F_trace(H, X, a: int, b: int, ts) -> np.ndarray:
    """F_tr(t) = Tr[...] / dim (beta = 0)."""
    return np.array([np.trace(_chain(H, X[a], X[b], t)[2]) / H.shape[0] for t in np.asarray(ts, np.float64)])
