"""Exact evolution and OTOC for a sparse SYK Hamiltonian whose terms commute.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Eq. (1) (main text) with a set of kept quadruples in which every two share an
even number of indices.  Two products of four distinct Majoranas then
commute, and each product P_t = chi_i chi_j chi_k chi_l squares to
(chi^2)^4 = 1/16 (reordering the eight factors takes 4*3/2 = 6 transpositions,
sign +1).  Hence, with H = sum_t J_t P_t,

    e^{-z J_t P_t} = cosh(z J_t / 4) - 4 sinh(z J_t / 4) P_t,
    e^{-zH}        = prod_t e^{-z J_t P_t}          (commuting factors),

exactly, for any complex z.  The product is applied factor by factor to a
parity-block vector with the per-basis-state maps of ``majorana`` (no matrix
is built), so the oracle reaches block sizes that the dense and CSR tiers
cannot (N = 44: 2^21 amplitudes per block).

Each term's map is composed from the maps of two Majorana pairs: a term that
is the union of the pairs (a, b) and (c, d) (a < b, c < d) satisfies
chi_a chi_b chi_c chi_d = sgn * P_sorted, sgn the sign of the permutation
that sorts (a, b, c, d), because distinct Majoranas anticommute.  A pair
product is even, so it maps each parity block to itself; its map over a
block is computed once from the single-site rules and cached.

The OTOC is the parity-block single-state formula of the supplement (OTOC
paragraph, symmetric beta/8 + beta/8 split) with these exact evolutions, in
the same order as ``otoc.F_state_sparse``.
"""
from __future__ import annotations

import numpy as np

from . import majorana as mj
from . import otoc as ot


def check_commuting(quads) -> None:
    """Raise ValueError unless every two quadruples share an even number of indices."""
    sets = [set(int(v) for v in q) for q in np.asarray(quads)]
    for i in range(len(sets)):
        for j in range(i + 1, len(sets)):
            if len(sets[i] & sets[j]) % 2:
                raise ValueError(f"terms {i} and {j} anticommute")


_BLOCK = {}
_PAIR = {}


def _block_position(N: int, rep: str, block: int):
    """Full-space indices of the block and a lookup full index -> block index."""
    key = (N, rep, block)
    if key not in _BLOCK:
        idx = mj.block_indices(N, rep)[block]
        pos = np.full(1 << (N // 2), -1, dtype=np.int64)
        pos[idx] = np.arange(len(idx))
        _BLOCK[key] = (idx.astype(np.uint64), pos)
    return _BLOCK[key]


def pair_map(N: int, rep: str, a: int, b: int, block: int):
    """(r, k): chi_a chi_b e_m = (i^k[m] / 2) e_{r[m]} inside the block (cached)."""
    key = (N, rep, a, b, block)
    if key not in _PAIR:
        idx, pos = _block_position(N, rep, block)
        g, ph = mj.apply_product_map([a, b], N, rep, idx)
        r = pos[g.astype(np.int64)]
        if np.any(r < 0):
            raise AssertionError("a Majorana pair left the parity block")
        k = np.rint(np.angle(ph * 2.0) / (np.pi / 2)).astype(np.int64) % 4
        if not np.allclose(ph, 0.5 * (1j ** k)):
            raise AssertionError("a Majorana pair phase is not a power of i over 2")
        _PAIR[key] = (r.astype(np.int32), k.astype(np.int8))
    return _PAIR[key]


def _split_pairs(quad, pairs=None):
    """The quadruple as two pairs (a, b), (c, d), a < b and c < d, with (a, b)
    one of `pairs` when one of them lies inside the quadruple (so that the
    pair maps of a matching are reused), else its two lowest indices; and the
    sign of the permutation that sorts (a, b, c, d)."""
    q = [int(v) for v in quad]
    a, b = q[0], q[1]
    for p in ([] if pairs is None else np.asarray(pairs)):
        if int(p[0]) in q and int(p[1]) in q:
            a, b = sorted((int(p[0]), int(p[1])))
            break
    c, d = sorted(v for v in q if v not in (a, b))
    s = [a, b, c, d]
    inversions = sum(1 for i in range(4) for j in range(i + 1, 4) if s[i] > s[j])
    return (a, b), (c, d), (-1) ** inversions


def term_map(N: int, rep: str, quad, block: int, pairs=None):
    """(r, ph): P e_m = ph[m] e_{r[m]} inside the block, P = chi_i chi_j chi_k chi_l."""
    (a, b), (c, d), sgn = _split_pairs(quad, pairs)
    r1, k1 = pair_map(N, rep, c, d, block)  # chi_c chi_d acts first
    r2, k2 = pair_map(N, rep, a, b, block)
    r = r2[r1]
    powers_of_i = sgn * 0.25 * np.array([1, 1j, -1, -1j])
    ph = powers_of_i[(k1 + k2[r1]) & 3]
    return r, ph


def apply_term(N: int, rep: str, quad, block: int, v, pairs=None) -> np.ndarray:
    """P v for P = chi_i chi_j chi_k chi_l acting inside parity block `block`."""
    r, ph = term_map(N, rep, quad, block, pairs)
    out = np.zeros(len(r), dtype=np.complex128)
    out[r] = ph * np.asarray(v, dtype=np.complex128)
    return out


def evolve(N: int, rep: str, quads, J, block: int, z, v, pairs=None) -> np.ndarray:
    """e^{-zH} v inside one parity block, H = sum_t J_t P_t with commuting P_t.
    pairs: optional Majorana pairs whose unions form the quadruples (only
    used to share cached pair maps)."""
    check_commuting(quads)
    out = np.array(v, dtype=np.complex128)
    z = complex(z)
    for quad, c in zip(np.asarray(quads), np.asarray(J, dtype=np.float64)):
        w = z * c / 4.0
        out = np.cosh(w) * out - 4.0 * np.sinh(w) * apply_term(N, rep, quad, block, out, pairs)
    return out


def F_state(N: int, rep: str, quads, J, a: int, b: int, beta: float, ts, psi_U, psi_D, pairs=None) -> np.ndarray:
    """Parity-block F_psi(t) = F_U + F_D with the exact commuting-term evolutions."""
    psis = (np.asarray(psi_U, np.complex128), np.asarray(psi_D, np.complex128))
    out = np.zeros(len(ts), dtype=np.complex128)
    for P in (0, 1):
        Q = 1 - P
        cb = ot.chi_block_sparse(N, rep, b, P)
        ca = ot.chi_block_sparse(N, rep, a, Q)
        ev = lambda blk, z, v: evolve(N, rep, quads, J, blk, z, v, pairs)
        u0 = ev(P, beta / 8.0, psis[P])
        for n, t in enumerate(np.asarray(ts, dtype=np.float64)):
            k = ev(Q, 1j * t + beta / 4.0, cb @ u0)
            k = ev(P, -1j * t + beta / 4.0, ca @ k)
            k = ev(Q, 1j * t + beta / 4.0, cb @ k)
            k = ca @ k
            bra = ev(P, 1j * t + beta / 8.0, psis[P])
            out[n] += np.vdot(bra, k)
    return out
