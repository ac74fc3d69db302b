"""Pins of the spin-chain oracle (oracle/spin.py) against facts that do not
come from the oracle itself: the Pauli multiplication table, textbook spectra
(free-fermion XX chain, two-site Heisenberg singlet/triplet, a single field),
a conservation law, two independent constructions against each other, and
closed forms of the OTOC chain of Eq. (2) with Pauli strings W, V."""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg as sla

import syk_inputs as si
from oracle import otoc
from oracle import spin


def _normed(v):
    return v / np.linalg.norm(v)


def test_pauli_multiplication_table():
    """XY = iZ, YZ = iX, ZX = iY and squares = 1 (fixes the sign of sigma_y
    relative to X and Z, and the letter of each mask pattern)."""
    X, Y, Z = (spin.pauli_dense(1, *si.pauli_mask({0: op})) for op in "XYZ")
    I = np.eye(2)
    assert np.allclose(X @ Y, 1j * Z) and np.allclose(Y @ Z, 1j * X) and np.allclose(Z @ X, 1j * Y)
    for P in (X, Y, Z):
        assert np.allclose(P @ P, I)
    assert np.allclose(Z, np.diag([1, -1]))  # |0> is the +1 eigenstate of Z
    assert np.allclose(X @ np.array([1, 0]), [0, 1])


def test_qubit_order_is_bit_order():
    """The letter on qubit q acts on bit q of the basis index."""
    L = 3
    for q in range(L):
        P = spin.pauli_dense(L, *si.pauli_mask({q: "X"}))
        for m in range(1 << L):
            e = np.zeros(1 << L)
            e[m] = 1
            assert np.argmax(np.abs(P @ e)) == m ^ (1 << q)
        Zq = spin.pauli_dense(L, *si.pauli_mask({q: "Z"}))
        assert np.allclose(np.diag(Zq), [1 - 2 * ((m >> q) & 1) for m in range(1 << L)])


@pytest.mark.parametrize("L", [1, 2, 4])
def test_maps_match_dense_products(L):
    """Basis-state maps (single-qubit rules) equal the Kronecker products, for
    every string on L qubits."""
    cols = np.arange(1 << L, dtype=np.uint64)
    for x in range(1 << L):
        for z in range(1 << L):
            P = spin.pauli_dense(L, x, z)
            g, ph = spin.apply_map(L, x, z, cols)
            M = np.zeros_like(P)
            M[g.astype(np.int64), cols.astype(np.int64)] = ph
            assert np.allclose(M, P), (x, z)
            assert np.allclose(P, P.conj().T)  # Hermitian
            assert np.allclose(P @ P, np.eye(1 << L))


def test_commutation_rule():
    L = 3
    for x1, z1, x2, z2 in itertools.product(range(8), repeat=4):
        A, B = spin.pauli_dense(L, x1, z1), spin.pauli_dense(L, x2, z2)
        assert np.allclose(A @ B, B @ A) == spin.commute(x1, z1, x2, z2)
        assert np.allclose(A @ B, B @ A) or np.allclose(A @ B, -B @ A)


def test_xx_chain_free_fermion_spectrum():
    """H = (J/2) sum_i (X_i X_{i+1} + Y_i Y_{i+1}), open chain, maps by
    Jordan-Wigner to free fermions hopping with amplitude J: many-body levels
    are the subset sums of eps_k = 2 J cos(pi k / (L + 1)), k = 1..L."""
    L, J = 6, 0.7
    xs, zs, hs = [], [], []
    for i in range(L - 1):
        for op in "XY":
            x, z = si.pauli_mask({i: op, i + 1: op})
            xs.append(x)
            zs.append(z)
            hs.append(J / 2)
    ev = np.linalg.eigvalsh(spin.dense_H(L, xs, zs, hs))
    eps = [2 * J * math.cos(math.pi * k / (L + 1)) for k in range(1, L + 1)]
    sums = sorted(sum(s) for r in range(L + 1) for s in itertools.combinations(eps, r))
    assert np.allclose(np.sort(ev), sums, atol=1e-12)


def test_two_site_heisenberg_singlet_triplet():
    H = spin.dense_H(2, *zip(*[si.pauli_mask({0: op, 1: op}) for op in "XYZ"]), [1.0, 1.0, 1.0])
    assert np.allclose(np.sort(np.linalg.eigvalsh(H)), [-3, 1, 1, 1], atol=1e-13)


def test_single_site_fields_spectrum():
    """h_x X + h_z Z on one qubit: eigenvalues +-sqrt(h_x^2 + h_z^2); a Y field
    adds in quadrature too."""
    hx, hy, hz = 0.3, -1.1, 0.8
    H = spin.dense_H(1, [1, 1, 0], [0, 1, 1], [hx, hy, hz])
    r = math.sqrt(hx * hx + hy * hy + hz * hz)
    assert np.allclose(np.linalg.eigvalsh(H), [-r, r], atol=1e-13)


def test_heisenberg_chain_conserves_magnetisation_and_trace_identities():
    L = 6
    x, z, h, fields = si.heisenberg_chain(L, W=2.0, r=3)
    H = spin.dense_H(L, x, z, h)
    Mz = sum(spin.pauli_dense(L, *si.pauli_mask({q: "Z"})) for q in range(L))
    assert np.allclose(H @ Mz, Mz @ H, atol=1e-12)
    # Tr H = 0 and Tr H^2 / dim = sum h^2 (orthonormal strings under Tr/dim)
    assert abs(np.trace(H)) < 1e-12
    assert np.isclose(np.trace(H @ H).real / (1 << L), np.sum(h ** 2), rtol=1e-12)
    # the field term is -sum_i h_i S^z_i: its diagonal at |0...0> is -sum h_i / 2
    Hf = spin.dense_H(L, x[-L:], z[-L:], h[-L:])
    assert np.isclose(Hf[0, 0].real, -np.sum(fields) / 2)


@pytest.mark.parametrize("L", [3, 7])
def test_csr_and_rows_match_dense(L):
    x, z, h = si.random_pauli_terms(L, 25, seed=L)
    Hd = spin.dense_H(L, x, z, h)
    Hc = spin.csr_H(L, x, z, h).toarray()
    assert np.allclose(Hc, Hd, atol=1e-13)
    rng = np.random.default_rng(1)
    psi = rng.normal(size=1 << L) + 1j * rng.normal(size=1 << L)
    rows = rng.integers(0, 1 << L, 20).astype(np.uint64)
    got = spin.rows_of_Hpsi(L, x, z, h, rows, lambda g: psi[g.astype(np.int64)])
    assert np.allclose(got, (Hd @ psi)[rows.astype(np.int64)], atol=1e-12)


def test_otoc_single_field_closed_form():
    """H = h Z_0 + g Z_1, W = V = X_0, beta = 0: W(t) = X_0 e^{-2ihtZ_0}, so
    F(t) = Tr[(W(t) V)^2] / dim = cos(4 h t)."""
    L, hh, g = 2, 0.37, 1.3
    H = spin.dense_H(L, [0, 0], [1, 2], [hh, g])
    Wm = spin.pauli_dense(L, *si.pauli_mask({0: "X"}))
    ts = np.array([0.0, 0.3, 1.0, 2.2])
    F = otoc.F_trace(H, {0: Wm, 1: Wm}, 0, 1, 0.0, ts)
    assert np.allclose(F, np.cos(4 * hh * ts), atol=1e-13)


def _anti_instance(L, seed):
    """Strings that each carry Z on qubit 0: every one anticommutes with X_0
    and with Y_0."""
    rng = np.random.default_rng(seed)
    xs, zs = [], []
    for _ in range(5):
        ops = {0: "Z"}
        for q in rng.choice(np.arange(1, L), size=2, replace=False):
            ops[int(q)] = "XYZ"[int(rng.integers(0, 3))]
        x, z = si.pauli_mask(ops)
        xs.append(x)
        zs.append(z)
    return xs, zs, rng.normal(size=5)


def test_otoc_closed_form_all_terms_anticommute():
    """W and V anticommute with every term and with each other: the chain
    collapses to F_psi(t) = -<psi| e^{4itH} |psi> for every beta."""
    L = 4
    xs, zs, hs = _anti_instance(L, 3)
    H = spin.dense_H(L, xs, zs, hs)
    Wm = spin.pauli_dense(L, *si.pauli_mask({0: "X"}))
    Vm = spin.pauli_dense(L, *si.pauli_mask({0: "Y"}))
    rng = np.random.default_rng(4)
    psi = _normed(rng.normal(size=1 << L) + 1j * rng.normal(size=1 << L))
    ts = [0.0, 0.4, 1.7]
    for beta in (0.0, 3.0):
        ref = [-np.vdot(psi, sla.expm(4j * t * H) @ psi) for t in ts]
        assert np.allclose(otoc.F_state(H, {0: Wm, 1: Vm}, 0, 1, beta, ts, psi), ref, atol=1e-12)


def test_otoc_closed_form_all_terms_commute():
    """W and V commute with every term: F_psi = s <psi| e^{-beta H} |psi> with
    s = +1 if W and V commute, -1 if they anticommute."""
    L = 4
    xs, zs, hs = [], [], []
    for q in range(1, L):
        for op in "XZ":
            x, z = si.pauli_mask({q: op, (q % (L - 1)) + 1: "Z"} if op == "X" else {q: op})
            xs.append(x)
            zs.append(z)
    hs = np.random.default_rng(8).normal(size=len(xs))
    H = spin.dense_H(L, xs, zs, hs)
    rng = np.random.default_rng(5)
    psi = _normed(rng.normal(size=1 << L) + 1j * rng.normal(size=1 << L))
    for (wo, vo, s) in (("X", "X", 1.0), ("X", "Y", -1.0)):
        Wm = spin.pauli_dense(L, *si.pauli_mask({0: wo}))
        Vm = spin.pauli_dense(L, *si.pauli_mask({0: vo}))
        for beta in (0.0, 2.0):
            ref = s * np.vdot(psi, sla.expm(-beta * H) @ psi)
            assert np.allclose(otoc.F_state(H, {0: Wm, 1: Vm}, 0, 1, beta, [0.0, 1.3], psi), ref, atol=1e-12)


def test_otoc_trace_t0_beta0_and_mean_over_basis():
    L = 5
    x, z, h, _ = si.heisenberg_chain(L, W=1.0, r=1)
    H = spin.dense_H(L, x, z, h)
    W0 = spin.pauli_dense(L, *si.pauli_mask({0: "Z"}))
    V2 = spin.pauli_dense(L, *si.pauli_mask({2: "Z"}))
    X0 = spin.pauli_dense(L, *si.pauli_mask({0: "X"}))
    assert np.isclose(otoc.F_trace(H, {0: W0, 1: V2}, 0, 1, 0.0, [0.0])[0], 1.0, atol=1e-13)
    assert np.isclose(otoc.F_trace(H, {0: W0, 1: X0}, 0, 1, 0.0, [0.0])[0], -1.0, atol=1e-13)
    ts = np.array([0.0, 0.9, 2.5])
    Ft = otoc.F_trace(H, {0: W0, 1: V2}, 0, 1, 3.0, ts)
    acc = sum(otoc.F_state(H, {0: W0, 1: V2}, 0, 1, 3.0, ts, e) for e in np.eye(1 << L))
    assert np.allclose(Ft, acc / (1 << L), atol=1e-13)
    assert np.max(np.abs(Ft.imag)) < 1e-13


def test_typical_states_estimate_the_trace():
    """The mean of F_psi over normalised complex-Gaussian states approaches
    the exact trace within the statistical error O(1 / sqrt(S dim))."""
    L = 6
    x, z, h, _ = si.heisenberg_chain(L, W=1.0, r=2)
    H = spin.dense_H(L, x, z, h)
    X = {0: spin.pauli_dense(L, *si.pauli_mask({0: "Z"})), 1: spin.pauli_dense(L, *si.pauli_mask({3: "Z"}))}
    ts = np.array([0.0, 1.0, 2.0])
    Ft = otoc.F_trace(H, X, 0, 1, 0.0, ts)
    S = 300
    rng = np.random.default_rng(12)
    acc = np.zeros(len(ts), dtype=np.complex128)
    for _ in range(S):
        acc += otoc.F_state(H, X, 0, 1, 0.0, ts, _normed(rng.normal(size=1 << L) + 1j * rng.normal(size=1 << L)))
    assert np.all(np.abs(acc / S - Ft) < 4.0 / math.sqrt(S * (1 << L)))
