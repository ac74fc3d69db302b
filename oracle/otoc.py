"""Regularised OTOC of Eq. (2) (main text) and its single-state estimator.

Exact trace (Eq. (2), raw, divided by the dimension instead of Z):
    F_tr(t) = Tr[e^{itH} chi_a e^{-(it+b/4)H} chi_b e^{(it-b/4)H} chi_a
                 e^{-(it+b/4)H} chi_b e^{-bH/4}] / dim
and the normalised OTOC F_tr(t)/F_tr(0) (Z of Eq. (2) is F_tr(0) * dim).
The paper uses a = N-1, b = N-2.

Single state (supplement, OTOC paragraph, symmetric beta/8 + beta/8 split):
    F_psi(t) = <psi| e^{(it-b/8)H} chi_a e^{-(it+b/4)H} chi_b e^{(it-b/4)H}
                 chi_a e^{-(it+b/4)H} chi_b e^{-bH/8} |psi>
and in parity blocks (same paragraph) F_psi = F_U + F_D with
    F_U = <psi_U| e^{(it-b/8)H_UU} chi_a^{UD} e^{-(it+b/4)H_DD} chi_b^{DU}
          e^{(it-b/4)H_UU} chi_a^{UD} e^{-(it+b/4)H_DD} chi_b^{DU}
          e^{-bH_UU/8} |psi_U>
and F_D the same with U and D swapped.  For a normalised typical state the
mean of F_psi over states is F_tr.  The OTOC of a set of states is
Re mean F_psi(t) / Re mean F_psi(0).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import dynamics as dyn
from . import hamiltonian as ham
from . import majorana as mj


def F_trace(H, X, a: int, b: int, beta: float, ts, eigpair=None) -> np.ndarray:
    """Raw exact-trace F(t)/dim on the full space, for each t in ts."""
    lam, V = dyn.eig(H) if eigpair is None else eigpair
    Xa = V.conj().T @ X[a] @ V
    Xb = V.conj().T @ X[b] @ V
    q = beta / 4.0
    out = []
    for t in np.asarray(ts, dtype=np.float64):
        e_m = np.exp(-(1j * t + q) * lam)   # e^{-(it+b/4)H}
        e_p = np.exp(-(-1j * t + q) * lam)  # e^{(it-b/4)H}
        e_l = np.exp(1j * t * lam)          # e^{itH}
        e_r = np.exp(-q * lam)              # e^{-bH/4}
        # Tr[ E_l Xa E_m Xb E_p Xa E_m Xb E_r ] in the eigenbasis of H.
        M1 = (e_l[:, None] * Xa) * e_m[None, :]
        M2 = Xb * e_p[None, :]
        M3 = Xa * e_m[None, :]
        M4 = Xb * e_r[None, :]
        P = M1 @ M2
        Q = M3 @ M4
        out.append(np.sum(P * Q.T) / H.shape[0])
    return np.array(out)


def F_state(H, X, a: int, b: int, beta: float, ts, psi, eigpair=None) -> np.ndarray:
    """F_psi(t) on the full space for one (normalised) state."""
    lam, V = dyn.eig(H) if eigpair is None else eigpair
    Xa = V.conj().T @ X[a] @ V
    Xb = V.conj().T @ X[b] @ V
    p = V.conj().T @ np.asarray(psi, dtype=np.complex128)
    out = []
    for t in np.asarray(ts, dtype=np.float64):
        k = np.exp(-beta / 8.0 * lam) * p
        k = np.exp(-(1j * t + beta / 4.0) * lam) * (Xb @ k)
        k = np.exp(-(-1j * t + beta / 4.0) * lam) * (Xa @ k)
        k = np.exp(-(1j * t + beta / 4.0) * lam) * (Xb @ k)
        k = Xa @ k
        bra = np.exp(-(1j * t + beta / 8.0) * lam) * p  # e^{-(it+b/8)H} psi
        out.append(np.vdot(bra, k))
    return np.array(out)


def F_state_blocks(N, rep, HUU, HDD, X, a, b, beta, ts, psi_U, psi_D) -> np.ndarray:
    """F_psi(t) = F_U + F_D from the parity-block formula (dense blocks)."""
    Hs = (HUU, HDD)
    eigs = (dyn.eig(HUU), dyn.eig(HDD))
    chi = {
        (n, to, fr): ham.block_of(X[n], N, rep, to, fr)
        for n in (a, b)
        for (to, fr) in ((0, 1), (1, 0))
    }
    psis = (np.asarray(psi_U, np.complex128), np.asarray(psi_D, np.complex128))
    out = np.zeros(len(ts), dtype=np.complex128)
    for P in (0, 1):
        Q = 1 - P
        ev = lambda blk, z, v: dyn.evolve(Hs[blk], z, v, eigs[blk])
        u0 = ev(P, beta / 8.0, psis[P])
        for n, t in enumerate(np.asarray(ts, dtype=np.float64)):
            k = chi[(b, Q, P)] @ u0
            k = ev(Q, 1j * t + beta / 4.0, k)
            k = chi[(a, P, Q)] @ k
            k = ev(P, -1j * t + beta / 4.0, k)
            k = chi[(b, Q, P)] @ k
            k = ev(Q, 1j * t + beta / 4.0, k)
            k = chi[(a, P, Q)] @ k
            bra = ev(P, 1j * t + beta / 8.0, psis[P])
            out[n] += np.vdot(bra, k)
    return out


def chi_block_sparse(N: int, rep: str, n: int, from_block: int) -> sp.csr_matrix:
    """chi_n restricted to from_block -> other block, built from basis maps."""
    iB = mj.block_indices(N, rep)
    src = iB[from_block].astype(np.uint64)
    dst_pos = np.full(2 * len(src), -1, dtype=np.int64)
    dst_pos[iB[1 - from_block]] = np.arange(len(src))
    g, ph = mj.apply_majorana_map(n, N, rep, src, 1.0)
    r = dst_pos[g.astype(np.int64)]
    if np.any(r < 0):
        raise AssertionError("Majorana did not change the parity block")
    D = len(src)
    return sp.csr_matrix((ph, (r, np.arange(D))), shape=(D, D))


def F_state_sparse(N, rep, quads, J, a, b, beta, ts, psi_U, psi_D) -> np.ndarray:
    """Parity-block F_psi(t) with CSR blocks and expm_multiply (N up to ~32)."""
    Hs = (ham.csr_block(N, quads, J, rep, 0), ham.csr_block(N, quads, J, rep, 1))
    psis = (np.asarray(psi_U, np.complex128), np.asarray(psi_D, np.complex128))
    out = np.zeros(len(ts), dtype=np.complex128)
    for P in (0, 1):
        Q = 1 - P
        cb = chi_block_sparse(N, rep, b, P)
        ca = chi_block_sparse(N, rep, a, Q)
        cb2 = chi_block_sparse(N, rep, b, P)
        ev = lambda blk, z, v: dyn.evolve_sparse(Hs[blk], z, v)
        u0 = ev(P, beta / 8.0, psis[P])
        for n, t in enumerate(np.asarray(ts, dtype=np.float64)):
            k = ev(Q, 1j * t + beta / 4.0, cb @ u0)
            k = ev(P, -1j * t + beta / 4.0, ca @ k)
            k = ev(Q, 1j * t + beta / 4.0, cb2 @ k)
            k = ca @ k
            bra = ev(P, 1j * t + beta / 8.0, psis[P])
            out[n] += np.vdot(bra, k)
    return out


def normalise(F) -> np.ndarray:
    """OTOC(t) = Re F(t) / Re F(0) (F(0) = F[0])."""
    F = np.asarray(F)
    return F.real / F.real[0]


# --- Green function (supplement, G(t) paragraph) ----------------------------
#   G(t) = <psi| e^{(it - b/2)H} chi_a e^{-iHt} chi_a e^{-bH/2} |psi>,
#   G_R(t) = Re G(t) / Re G(0); the paper uses a = N-1.
#   In parity blocks G = sum_P <psi_P| e^{(it-b/2)H_PP} chi_a^{PQ}
#   e^{-iH_QQ t} chi_a^{QP} e^{-bH_PP/2} |psi_P>.
def G_state(H, X, a: int, beta: float, ts, psi, eigpair=None) -> np.ndarray:
    lam, V = dyn.eig(H) if eigpair is None else eigpair
    Xa = V.conj().T @ X[a] @ V
    p = V.conj().T @ np.asarray(psi, dtype=np.complex128)
    out = []
    for t in np.asarray(ts, dtype=np.float64):
        k = np.exp(-beta / 2.0 * lam) * p
        k = Xa @ (np.exp(-1j * t * lam) * (Xa @ k))
        bra = np.exp(-(1j * t + beta / 2.0) * lam) * p  # e^{-(it+b/2)H} psi
        out.append(np.vdot(bra, k))
    return np.array(out)


def G_state_blocks(N, rep, HUU, HDD, X, a, beta, ts, psi_U, psi_D) -> np.ndarray:
    Hs = (HUU, HDD)
    eigs = (dyn.eig(HUU), dyn.eig(HDD))
    psis = (np.asarray(psi_U, np.complex128), np.asarray(psi_D, np.complex128))
    out = np.zeros(len(ts), dtype=np.complex128)
    for P in (0, 1):
        Q = 1 - P
        ev = lambda blk, z, v: dyn.evolve(Hs[blk], z, v, eigs[blk])
        u0 = ev(P, beta / 2.0, psis[P])
        for n, t in enumerate(np.asarray(ts, dtype=np.float64)):
            k = ham.block_of(X[a], N, rep, Q, P) @ u0
            k = ev(Q, 1j * t, k)
            k = ham.block_of(X[a], N, rep, P, Q) @ k
            bra = ev(P, 1j * t + beta / 2.0, psis[P])
            out[n] += np.vdot(bra, k)
    return out
