"""Exact time evolution e^{-zH} x for complex z = tau + i t.

The paper evolves states with a restarted Krylov method (supplement Sec. I.A);
the oracle instead computes the exact quantity the Krylov method approximates:
  * dense: H = V diag(lam) V^dagger (numpy.linalg.eigh), e^{-zH} = V e^{-z lam} V^dagger;
  * sparse: scipy.sparse.linalg.expm_multiply (Al-Mohy & Higham 2011) on -zH.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


def eig(H):
    lam, V = np.linalg.eigh(H)
    return lam, V


def expm_z(H, z, eigpair=None) -> np.ndarray:
    """Dense e^{-zH} for Hermitian H."""
    lam, V = eig(H) if eigpair is None else eigpair
    return (V * np.exp(-z * lam)) @ V.conj().T


def evolve(H, z, x, eigpair=None) -> np.ndarray:
    """e^{-zH} x (dense)."""
    lam, V = eig(H) if eigpair is None else eigpair
    return V @ (np.exp(-z * lam) * (V.conj().T @ np.asarray(x, dtype=np.complex128)))


def evolve_sparse(Hcsr, z, x) -> np.ndarray:
    """e^{-zH} x with H a scipy sparse matrix."""
    return spla.expm_multiply((-complex(z)) * Hcsr.astype(np.complex128), np.asarray(x, dtype=np.complex128))
