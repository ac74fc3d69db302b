"""The paper's <bits, coeff> spin-operator encoding and Algorithm 1.

Supplement Sec. I.A: a Pauli string sigma_{i_{L-1}} (x) ... (x) sigma_{i_0}
with weight lambda is stored as bits = s_{i_{L-1}} ... s_{i_0} (two bits per
site, s_I = 00, s_X = 01, s_Y = 11, s_Z = 10, site k at bit positions 2k and
2k+1) and coeff = lambda * i^{#sigma_y}.  Algorithm 1 applies a list of such
tuples to a state vector.

Reading of "the i-th bit of n" (the algorithm writes it in terms of the 2L-bit
string index i): the bit that is tested is qubit floor(i/2) of n, after the
flips of that site have been applied.  With this reading sigma_y comes out as
[[0, -i], [i, 0]].
"""
from __future__ import annotations

import numpy as np

_CODE = {"I": 0b00, "X": 0b01, "Y": 0b11, "Z": 0b10}


def encode(ops: dict, lam: complex = 1.0):
    """ops: site -> 'I'|'X'|'Y'|'Z'.  Returns (bits, coeff)."""
    bits = 0
    ny = 0
    for s, op in ops.items():
        bits |= _CODE[op] << (2 * s)
        ny += op == "Y"
    return bits, complex(lam) * (1j ** ny)


def algorithm1(L: int, terms, psi) -> np.ndarray:
    """Phi = S Psi for S given as a list of (bits, coeff); plain loops.

    Outer loop over output index m, middle loop over tuples, inner loop over
    the set bits of `bits` (even position 2k: flip qubit k of n; odd position
    2k+1: if qubit k of n is set, toggle the sign).  Only for small L.
    """
    psi = np.asarray(psi, dtype=np.complex128)
    phi = np.zeros(1 << L, dtype=np.complex128)
    for m in range(1 << L):
        for bits, coeff in terms:
            n = m
            minus = False
            for i in range(2 * L):
                if not (bits >> i) & 1:
                    continue
                if i % 2 == 0:
                    n ^= 1 << (i // 2)
                elif (n >> (i // 2)) & 1:
                    minus = not minus
            phi[m] += (-coeff if minus else coeff) * psi[n]
    return phi
