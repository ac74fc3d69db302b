"""Seeded synthetic inputs for the sparse-SYK workloads.

This module is shared by the CPU oracle, the tests and the benchmark.  It holds
only input generation: coupling draws, random states and a counter-based
generator.  It computes nothing that the method itself computes (no Majorana
algebra, no Hamiltonian action, no time evolution).

Workload recipe (the paper's ensemble, main text around Eq. (1)):
  * every quadruple 0 <= i < j < k < l < N is kept independently with
    probability p (a Bernoulli mask), with p = k_sp * N / C(N, 4) so that the
    expected number of kept terms is k_sp * N (sparsity parameter k);
  * each kept coupling J is Gaussian with mean 0 and variance 3! J0^2/(p N^3)
    in the chi-normalisation ({chi_i, chi_j} = delta_ij);
  * couplings for realisation r use numpy PCG64(1000 + r) unless a seed is
    given;
  * a typical (Haar-like) state is an i.i.d. complex Gaussian vector over the
    full 2^(N/2) space, normalised over the full space; its two parity blocks
    are returned separately and are *not* renormalised.

Spin-chain inputs (the outlook's sparse spin chains): Pauli strings given as
two L-bit masks (x, z) -- on qubit q, x only = sigma_x, z only = sigma_z,
both = sigma_y -- with real weights h.  The many-body-localisation workload
is the random-field Heisenberg chain
  H = J sum_i S_i . S_{i+1} - sum_i h_i S^z_i,  S = sigma / 2,
  h_i uniform in [-W, W] (PCG64(2000 + r)), periodic unless stated,
written as the strings X_i X_{i+1}, Y_i Y_{i+1}, Z_i Z_{i+1} (weight J/4) and
Z_i (weight -h_i/2).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

__all__ = [
    "all_quads",
    "sample_sparse_syk",
    "sample_dense_syk",
    "sample_commuting_syk",
    "random_state",
    "philox4x32_10",
    "philox_state",
    "pauli_mask",
    "heisenberg_chain",
    "random_pauli_terms",
    "served_requests",
]


def all_quads(N: int) -> np.ndarray:
    """All index quadruples i<j<k<l<N in lexicographic order, int32 [C(N,4), 4]."""
    if N < 4:
        return np.zeros((0, 4), dtype=np.int32)
    return np.array(list(itertools.combinations(range(N), 4)), dtype=np.int32)


def sample_sparse_syk(N: int, k: float, seed: int | None = None, r: int = 0, J0: float = 1.0):
    """Draw one sparse-SYK realisation.

    Returns (quads int32 [T,4], J float64 [T], p).  T is random (Bernoulli mask).
    """
    rng = np.random.Generator(np.random.PCG64(1000 + r if seed is None else seed))
    q = all_quads(N)
    C = q.shape[0]
    p = min(1.0, k * N / C)
    keep = rng.random(C) < p
    quads = q[keep]
    var = 6.0 * J0 * J0 / (p * N ** 3)
    J = rng.normal(0.0, math.sqrt(var), size=quads.shape[0])
    return quads.astype(np.int32), J.astype(np.float64), p


def sample_dense_syk(N: int, seed: int = 0, J0: float = 1.0):
    """Dense SYK (p = 1): every quadruple, J ~ N(0, 3! J0^2 / N^3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    quads = all_quads(N)
    J = rng.normal(0.0, math.sqrt(6.0 * J0 * J0 / N ** 3), size=quads.shape[0])
    return quads, J, 1.0


def sample_commuting_syk(N: int, seed: int, n_terms: int | None = None, J0: float = 0.5):
    """Quadruples that pairwise share 0 or 2 indices, so that their products
    commute (the oracle's exact commuting tier).

    The N Majorana indices are split into N/2 pairs: (N-2, N-1) (the
    Majoranas of the paper's OTOC, so that their OTOC varies with t) and a
    random perfect matching of the rest; each term is the union of two
    distinct pairs, for n_terms distinct random pairs of pairs (default N),
    written as a sorted quadruple; J ~ N(0, J0^2) (couplings of order one, so
    that a few dozen terms spread the spectrum over a few units).  Returns
    (quads int32 [T, 4], J float64 [T], pairs int32 [N/2, 2]).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    rest = np.sort(rng.permutation(N - 2).reshape(-1, 2), axis=1)
    pairs = np.concatenate([rest, [[N - 2, N - 1]]])
    edges = [(i, j) for i in range(len(pairs)) for j in range(i + 1, len(pairs))]
    T = min(len(edges), N if n_terms is None else n_terms)
    pick = rng.choice(len(edges), size=T, replace=False)
    quads = np.array([np.sort(np.concatenate([pairs[edges[e][0]], pairs[edges[e][1]]])) for e in pick])
    J = rng.normal(0.0, J0, size=T)
    return quads.astype(np.int32).reshape(-1, 4), J.astype(np.float64), pairs.astype(np.int32)


def random_state(N: int, seed: int, dtype=np.complex128):
    """Typical state over the full 2^(N/2) space: (psi_U, psi_D), each 2^(N/2-1).

    Gaussian real and imaginary parts, normalised so that
    ||psi_U||^2 + ||psi_D||^2 = 1.
    """
    D = 1 << (N // 2 - 1)
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.normal(size=(2, D)) + 1j * rng.normal(size=(2, D))
    v /= np.linalg.norm(v)
    return v[0].astype(dtype), v[1].astype(dtype)


# --- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
# easy as 1, 2, 3", SC'11).  Written from the published definition: a 4-word
# counter and 2-word key; each round multiplies words 0 and 2 by two constants
# (full 64-bit products split into hi/lo halves), XORs the high halves with the
# other counter words and the key, and permutes; the key is bumped by two
# Weyl constants between rounds.
_PM0 = np.uint64(0xD2511F53)
_PM1 = np.uint64(0xCD9E8D57)
_PW0 = np.uint64(0x9E3779B9)
_PW1 = np.uint64(0xBB67AE85)
_M32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Vectorised Philox4x32-10.  ctr: uint [...,4]; key: uint [...,2] -> uint32 [...,4]."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) & _M32 for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64) & _M32
    k1 = np.asarray(key[..., 1], dtype=np.uint64) & _M32
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _PW0) & _M32
            k1 = (k1 + _PW1) & _M32
        p0 = _PM0 * c[0]
        p1 = _PM1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _M32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _M32
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=-1).astype(np.uint32)


def philox_state(N: int, seed: int, state_id: int, idx=None):
    """Counter-based typical state: unnormalised complex Gaussian amplitudes.

    Amplitude number g in [0, 2D) (g = block * D + m, block 0 = U, 1 = D) uses
    counter (g mod 2^32, g >> 32, state_id mod 2^32, state_id >> 32) and key
    (seed mod 2^32, seed >> 32).  Output words w0..w3 give two 53-bit uniforms
    u1 = ((w1:w0 >> 11) + 1) / 2^53 in (0, 1] and u2 = (w3:w2 >> 11) / 2^53 in
    [0, 1); the amplitude is sqrt(-2 ln u1) * (cos 2 pi u2 + i sin 2 pi u2)
    (Box-Muller).  Returns complex128 values for the requested global indices
    (all 2D if idx is None).  Normalisation is left to the caller.
    """
    D = 1 << (N // 2 - 1)
    g = np.arange(2 * D, dtype=np.uint64) if idx is None else np.asarray(idx, dtype=np.uint64)
    ctr = np.zeros(g.shape + (4,), dtype=np.uint64)
    ctr[..., 0] = g & _M32
    ctr[..., 1] = g >> np.uint64(32)
    ctr[..., 2] = np.uint64(state_id & 0xFFFFFFFF)
    ctr[..., 3] = np.uint64(state_id >> 32)
    key = np.zeros(g.shape + (2,), dtype=np.uint64)
    key[..., 0] = np.uint64(seed & 0xFFFFFFFF)
    key[..., 1] = np.uint64(seed >> 32)
    w = philox4x32_10(ctr, key).astype(np.uint64)
    a = ((w[..., 1] << np.uint64(32)) | w[..., 0]) >> np.uint64(11)
    b = ((w[..., 3] << np.uint64(32)) | w[..., 2]) >> np.uint64(11)
    u1 = (a.astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = b.astype(np.float64) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2 * np.pi * u2) + 1j * r * np.sin(2 * np.pi * u2)


# ------------------------------------------------------------ spin chains --
def pauli_mask(ops: dict):
    """{qubit: 'X'|'Y'|'Z'} -> (x, z) masks of the string (identity elsewhere)."""
    x = z = 0
    for q, op in ops.items():
        if op in ("X", "Y"):
            x |= 1 << q
        if op in ("Z", "Y"):
            z |= 1 << q
    return x, z


def heisenberg_chain(L: int, W: float, r: int = 0, J: float = 1.0, periodic: bool = True, seed: int | None = None):
    """Random-field Heisenberg chain on L qubits as Pauli strings.

    Returns (x uint32 [T], z uint32 [T], h float64 [T], fields [L]).
    """
    rng = np.random.Generator(np.random.PCG64(2000 + r if seed is None else seed))
    fields = rng.uniform(-W, W, size=L)
    xs, zs, hs = [], [], []
    bonds = [(i, i + 1) for i in range(L - 1)]
    if periodic and L > 2:
        bonds.append((L - 1, 0))
    for i, j in bonds:
        for op in "XYZ":
            x, z = pauli_mask({i: op, j: op})
            xs.append(x)
            zs.append(z)
            hs.append(J / 4.0)
    for i in range(L):
        x, z = pauli_mask({i: "Z"})
        xs.append(x)
        zs.append(z)
        hs.append(-fields[i] / 2.0)
    return (np.array(xs, dtype=np.uint32), np.array(zs, dtype=np.uint32), np.array(hs, dtype=np.float64),
            fields)


def random_pauli_terms(L: int, T: int, seed: int, max_weight: int = 4):
    """T random Pauli strings of 1..max_weight non-identity letters (uniform
    letters, distinct qubits) with N(0, 1) weights; duplicates are possible.
    Returns (x uint32 [T], z uint32 [T], h float64 [T])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xs, zs = [], []
    for _ in range(T):
        w = int(rng.integers(1, min(max_weight, L) + 1))
        qs = rng.choice(L, size=w, replace=False)
        x, z = pauli_mask({int(q): "XYZ"[int(rng.integers(0, 3))] for q in qs})
        xs.append(x)
        zs.append(z)
    return np.array(xs, dtype=np.uint32), np.array(zs, dtype=np.uint32), rng.normal(size=T)


def served_requests(n: int, rate: float, seed: int = 0, n_choices=(28, 30, 32, 34, 36, 38, 40, 42, 44, 46, 48),
                    weight: float = 0.7, ks=(0.5, 1.0, 2.0, 4.0), betas=(2.0, 5.0, 10.0, 20.0), t_max: float = 20.0,
                    dt: float = 0.1):
    """The served workload: n requests with Poisson arrival times of the given
    rate (1/s), N weighted toward small sizes (P(N) ~ weight^((N - N_min)/2)),
    sparsity k and beta uniform over the listed values, t = 0..t_max step dt.
    Returns dicts with keys rid, arrival, N, quads, J, beta, t_grid, seed."""
    rng = np.random.default_rng(seed)
    Ns = np.asarray(n_choices)
    p = weight ** ((Ns - Ns[0]) / 2.0)
    p /= p.sum()
    arr = np.cumsum(np.random.default_rng(seed).exponential(1.0 / rate, size=n))
    grid = np.round(np.arange(0.0, t_max + 1e-9, dt), 10)
    out = []
    for i in range(n):
        N = int(rng.choice(Ns, p=p))
        k = float(rng.choice(ks))
        q, J, _ = sample_sparse_syk(N, k, seed=10_000 + seed * 100_000 + i)
        out.append({"rid": i, "arrival": float(arr[i]), "N": N, "quads": q, "J": J, "beta": float(rng.choice(betas)),
                    "t_grid": grid, "seed": seed * 1_000_003 + i})
    return out
