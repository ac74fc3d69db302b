"""Majorana operators as dense matrices and as basis-state maps.

Paper reference: supplement Sec. I, Eq. (S1) and its compact form (the
sigma_{y/z}(floor((n-1)/2)) * prod sigma_x formula), gamma_{N-1} blocks
UD = -i, DU = +i, and the Pauli matrices listed after (S1).  The printed
sigma_y there is [[0, i], [-i, 0]]; this oracle uses the standard
[[0, -i], [i, 0]], which is what Algorithm 1 with coeff = lambda * i^{#sigma_y}
implements.  The choice flips the sign of every odd-index gamma in the paper
representation; that is a unitary equivalence of the Clifford algebra and does
not change traces (e.g. the OTOC).
"""
from __future__ import annotations

import math

import numpy as np

I2 = np.eye(2, dtype=np.complex128)
SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULI = {"I": I2, "X": SX, "Y": SY, "Z": SZ}


def kron_sites(ops: dict, q: int) -> np.ndarray:
    """Kronecker product over q qubits; ops maps site -> 'X'|'Y'|'Z'.

    Site s is bit s of the basis index, so the leftmost factor is site q-1.
    """
    M = np.ones((1, 1), dtype=np.complex128)
    for s in range(q - 1, -1, -1):
        M = np.kron(M, PAULI[ops.get(s, "I")])
    return M


def paper_A_ops(n: int, L: int) -> dict:
    """Single-site content of A_n = gamma_n^{UD} = gamma_n^{DU} (n <= 2L = N-2).

    Compact form: sigma_{y/z}(floor((n-1)/2)) times sigma_x on sites
    floor((n+1)/2) .. L-1; the y/z factor is absent for n = 0, sigma_y for odd
    n, sigma_z for even n >= 2.
    """
    ops = {}
    for s in range((n + 1) // 2, L):
        ops[s] = "X"
    if n > 0:
        ops[(n - 1) // 2] = "Y" if n % 2 == 1 else "Z"
    return ops


def jw_ops(n: int) -> dict:
    """gamma_{2s} = Z_0..Z_{s-1} X_s ; gamma_{2s+1} = Z_0..Z_{s-1} Y_s."""
    s = n // 2
    ops = {r: "Z" for r in range(s)}
    ops[s] = "X" if n % 2 == 0 else "Y"
    return ops


def gammas(N: int, rep: str) -> list:
    """Dense gamma_0..gamma_{N-1} on 2^{N/2}, {gamma_m, gamma_n} = 2 delta_mn."""
    if N % 2 or N < 4:
        raise ValueError("N must be even and >= 4")
    q = N // 2
    L = q - 1
    out = []
    if rep == "paper":
        for n in range(N - 1):
            ops = paper_A_ops(n, L)
            ops[L] = "X"  # block off-diagonal with UD = DU = A_n
            out.append(kron_sites(ops, q))
        out.append(kron_sites({L: "Y"}, q))  # UD = -i 1, DU = +i 1
    elif rep == "jw":
        for n in range(N):
            out.append(kron_sites(jw_ops(n), q))
    else:
        raise ValueError(rep)
    return out


def chis(N: int, rep: str) -> list:
    """chi_n = gamma_n / sqrt(2), {chi_m, chi_n} = delta_mn."""
    return [g / math.sqrt(2.0) for g in gammas(N, rep)]


def block_indices(N: int, rep: str):
    """Full-space indices of the U and D blocks, ordered by block index m."""
    q = N // 2
    L = q - 1
    D = 1 << L
    m = np.arange(D, dtype=np.int64)
    if rep == "paper":
        return m, m + D
    par = (np.bitwise_count(m) & 1).astype(np.int64)
    return m | (par << L), m | ((1 - par) << L)


def to_full(psi_U, psi_D, N: int, rep: str) -> np.ndarray:
    iU, iD = block_indices(N, rep)
    v = np.zeros(2 * len(psi_U), dtype=np.complex128)
    v[iU] = psi_U
    v[iD] = psi_D
    return v


def from_full(v, N: int, rep: str):
    iU, iD = block_indices(N, rep)
    return v[iU].copy(), v[iD].copy()


# ---------------------------------------------------------------------------
# Basis-state maps: the action of one Majorana on |f> for integer arrays f,
# built only from the single-site rules  X|b> = |1-b>,  Y|b> = i(-1)^b |1-b>,
# Z|b> = (-1)^b |b>.  These do not use the dense matrices above; the tests pin
# the two constructions against each other.
def _site_rule(op: str, f: np.ndarray, s: int):
    b = (f >> np.uint64(s)) & np.uint64(1)
    sign = 1.0 - 2.0 * b.astype(np.float64)
    if op == "X":
        return f ^ np.uint64(1 << s), np.ones(f.shape, dtype=np.complex128)
    if op == "Y":
        return f ^ np.uint64(1 << s), 1j * sign
    if op == "Z":
        return f, sign.astype(np.complex128)
    raise ValueError(op)


def majorana_site_ops(n: int, N: int, rep: str) -> dict:
    q = N // 2
    L = q - 1
    if rep == "paper":
        if n == N - 1:
            return {L: "Y"}
        ops = paper_A_ops(n, L)
        ops[L] = "X"
        return ops
    return jw_ops(n)


def apply_majorana_map(n: int, N: int, rep: str, f, phase):
    """chi_n |f> : returns (f', phase * <f'|chi_n|f>), vectorised over f."""
    f = np.asarray(f, dtype=np.uint64)
    ph = np.asarray(phase, dtype=np.complex128) / math.sqrt(2.0)
    for s, op in majorana_site_ops(n, N, rep).items():
        f, p = _site_rule(op, f, s)
        ph = ph * p
    return f, ph


def apply_product_map(idx, N: int, rep: str, f, phase=1.0):
    """chi_{idx[0]} chi_{idx[1]} ... |f>  (rightmost factor acts first)."""
    f = np.asarray(f, dtype=np.uint64)
    ph = np.broadcast_to(np.asarray(phase, dtype=np.complex128), f.shape).copy()
    for n in reversed(list(idx)):
        f, ph = apply_majorana_map(int(n), N, rep, f, ph)
    return f, ph
