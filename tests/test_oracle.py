"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these tests re-types an oracle formula: each compares the oracle with
an independent construction (closed form, algebraic identity, brute force, a
library routine on a special case) chosen so that a dropped term, wrong sign,
wrong index or transposed operand fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import syk_inputs as si
from oracle import dynamics as dyn
from oracle import hamiltonian as ham
from oracle import majorana as mj
from oracle import otoc
from oracle import pauli

REPS = ("paper", "jw")


def anticomm(A, B):
    return A @ B + B @ A


# --- Majorana algebra (supplement Eq. (S1); main text {gamma, gamma} statement)
@pytest.mark.parametrize("rep", REPS)
@pytest.mark.parametrize("N", [4, 6, 8, 10])
def test_clifford_algebra(rep, N):
    X = mj.chis(N, rep)
    dim = 1 << (N // 2)
    I = np.eye(dim)
    for m in range(N):
        assert np.allclose(X[m], X[m].conj().T)
        for n in range(N):
            assert np.allclose(anticomm(X[m], X[n]), I * (m == n), atol=1e-14)


@pytest.mark.parametrize("N", [6, 8, 10, 12])
def test_paper_special_gammas(N):
    """gamma_{N-1}: UD = -i 1, DU = +i 1; gamma_{N-2} blocks = sigma_z on the top
    site of the block (supplement, simplification paragraph); gamma_0 blocks =
    sigma_x on every site (compact form with n = 0)."""
    G = mj.gammas(N, "paper")
    L = N // 2 - 1
    D = 1 << L
    UD = lambda M: M[:D, D:]
    DU = lambda M: M[D:, :D]
    assert np.allclose(UD(G[N - 1]), -1j * np.eye(D))
    assert np.allclose(DU(G[N - 1]), 1j * np.eye(D))
    diag = np.array([1.0 - 2.0 * ((m >> (L - 1)) & 1) for m in range(D)])
    assert np.allclose(UD(G[N - 2]), np.diag(diag))
    assert np.allclose(DU(G[N - 2]), np.diag(diag))
    allx = np.zeros((D, D))
    for m in range(D):
        allx[m ^ (D - 1), m] = 1.0
    assert np.allclose(UD(G[0]), allx) and np.allclose(DU(G[0]), allx)
    for n in range(N):  # block off-diagonal
        assert np.allclose(G[n][:D, :D], 0) and np.allclose(G[n][D:, D:], 0)


@pytest.mark.parametrize("rep", REPS)
@pytest.mark.parametrize("N", [4, 6, 8, 10])
def test_basis_maps_match_dense(rep, N):
    X = mj.chis(N, rep)
    dim = 1 << (N // 2)
    f = np.arange(dim, dtype=np.uint64)
    for n in range(N):
        g, ph = mj.apply_majorana_map(n, N, rep, f, 1.0)
        M = np.zeros((dim, dim), dtype=np.complex128)
        M[g.astype(np.int64), np.arange(dim)] = ph
        assert np.allclose(M, X[n], atol=1e-15), n


# --- Algorithm 1 and the <bits, coeff> encoding (supplement Sec. I.A)
def test_algorithm1_sigma_y_is_standard():
    bits, coeff = pauli.encode({0: "Y"}, 1.0)
    assert bits == 0b11 and coeff == 1j
    M = np.column_stack([pauli.algorithm1(1, [(bits, coeff)], e) for e in np.eye(2)])
    assert np.allclose(M, [[0, -1j], [1j, 0]])


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_algorithm1_matches_kronecker(L):
    rng = np.random.default_rng(L)
    terms, Mref = [], np.zeros((1 << L, 1 << L), dtype=np.complex128)
    for _ in range(5):
        ops = {s: "IXYZ"[rng.integers(4)] for s in range(L)}
        lam = rng.normal() + 1j * rng.normal()
        terms.append(pauli.encode(ops, lam))
        Mref += lam * mj.kron_sites({s: o for s, o in ops.items() if o != "I"}, L)
    psi = rng.normal(size=1 << L) + 1j * rng.normal(size=1 << L)
    assert np.allclose(pauli.algorithm1(L, terms, psi), Mref @ psi, atol=1e-13)


# --- Hamiltonian (Eq. (1))
def _instance(N, k=4, r=0):
    q, J, _ = si.sample_sparse_syk(N, k, r=r)
    return q, J


@pytest.mark.parametrize("rep", REPS)
@pytest.mark.parametrize("N", [8, 10, 12])
def test_H_trace_identities(rep, N):
    q, J = _instance(N)
    H = ham.dense_H(N, q, J, rep)
    dim = H.shape[0]
    assert np.allclose(H, H.conj().T, atol=1e-14)
    assert abs(np.trace(H)) < 1e-12
    # distinct Majorana monomials are trace-orthogonal and each squares to 1/16
    assert np.isclose(np.trace(H @ H).real / dim, np.sum(J ** 2) / 16, rtol=1e-12)
    iU, iD = mj.block_indices(N, rep)
    assert np.allclose(H[np.ix_(iU, iD)], 0) and np.allclose(H[np.ix_(iD, iU)], 0)


@pytest.mark.parametrize("N", [6, 8, 10, 12])
def test_representation_independence_spectrum(N):
    q, J = _instance(N, r=3)
    e1 = np.linalg.eigvalsh(ham.dense_H(N, q, J, "paper"))
    e2 = np.linalg.eigvalsh(ham.dense_H(N, q, J, "jw"))
    assert np.allclose(e1, e2, atol=1e-12)


@pytest.mark.parametrize("rep", REPS)
@pytest.mark.parametrize("N", [8, 10, 12])
def test_csr_and_rows_match_dense(rep, N):
    q, J = _instance(N, r=1)
    H = ham.dense_H(N, q, J, rep)
    HU, HD = ham.blocks(H, N, rep)
    rng = np.random.default_rng(0)
    D = HU.shape[0]
    psi = [rng.normal(size=D) + 1j * rng.normal(size=D) for _ in range(2)]
    for blk, Hb in ((0, HU), (1, HD)):
        C = ham.csr_block(N, q, J, rep, blk).toarray()
        assert np.allclose(C, Hb, atol=1e-14)
        rows = rng.integers(0, D, size=17)
        got = ham.rows_of_Hpsi(N, q, J, rep, blk, rows, lambda b, m: psi[b][m.astype(np.int64)])
        assert np.allclose(got, (Hb @ psi[blk])[rows], atol=1e-13)


# --- Dynamics
def test_single_term_closed_form():
    """H = J chi_i chi_j chi_k chi_l has H^2 = (J/4)^2, so
    e^{-zH} = cosh(zJ/4) - sinh(zJ/4) H/(J/4)."""
    N = 10
    q = np.array([[1, 4, 6, 9]], dtype=np.int32)
    Jv = np.array([0.73])
    for rep in REPS:
        H = ham.dense_H(N, q, Jv, rep)
        HU, _ = ham.blocks(H, N, rep)
        w = Jv[0] / 4
        x = np.random.default_rng(1).normal(size=HU.shape[0]) + 0j
        for z in (0.3, 2.0 + 1.5j, -1j * 7.0, 5.0 - 3.0j):
            ref = np.cosh(z * w) * x - np.sinh(z * w) * (HU @ x) / w
            assert np.allclose(dyn.evolve(HU, z, x), ref, atol=1e-12)
            Hc = ham.csr_block(N, q, Jv, rep, 0)
            assert np.allclose(dyn.evolve_sparse(Hc, z, x), ref, atol=1e-10)


def test_evolve_matches_scipy_expm_and_semigroup():
    N = 10
    qd, J = _instance(N, r=2)
    HU, _ = ham.blocks(ham.dense_H(N, qd, J, "jw"), N, "jw")
    x = np.random.default_rng(2).normal(size=HU.shape[0]) + 0j
    z1, z2 = 0.7 + 1.9j, 1.3 - 0.4j
    assert np.allclose(dyn.evolve(HU, z1, x), sla.expm(-z1 * HU) @ x, atol=1e-12)
    assert np.allclose(dyn.evolve(HU, z1, dyn.evolve(HU, z2, x)), dyn.evolve(HU, z1 + z2, x), atol=1e-12)
    y = dyn.evolve(HU, 3.7j, x)  # unitary for imaginary z
    assert np.isclose(np.linalg.norm(y), np.linalg.norm(x), rtol=1e-13)
    assert np.isclose(np.vdot(y, HU @ y).real, np.vdot(x, HU @ x).real, rtol=1e-12)


# --- OTOC (Eq. (2); supplement OTOC formulas)
def _normed(v):
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("rep", REPS)
def test_otoc_t0_beta0_is_minus_quarter(rep):
    N = 10
    q, J = _instance(N, r=4)
    H = ham.dense_H(N, q, J, rep)
    X = mj.chis(N, rep)
    rng = np.random.default_rng(5)
    psi = _normed(rng.normal(size=H.shape[0]) + 1j * rng.normal(size=H.shape[0]))
    for a, b in ((N - 1, N - 2), (0, 3), (5, 2)):
        assert np.isclose(otoc.F_state(H, X, a, b, 0.0, [0.0], psi)[0], -0.25, atol=1e-13)
        assert np.isclose(otoc.F_trace(H, X, a, b, 0.0, [0.0])[0], -0.25, atol=1e-13)
    assert np.isclose(otoc.F_trace(H, X, 3, 3, 0.0, [0.0])[0], 0.25, atol=1e-13)


def _commuting_instance(N, a, b, n_terms, contain):
    """Terms that all contain both a and b (contain=True) or neither."""
    rng = np.random.default_rng(11)
    others = [i for i in range(N) if i not in (a, b)]
    quads = []
    while len(quads) < n_terms:
        if contain:
            c, d = rng.choice(others, 2, replace=False)
            quads.append(sorted([a, b, int(c), int(d)]))
        else:
            quads.append(sorted(int(v) for v in rng.choice(others, 4, replace=False)))
    return np.array(quads, dtype=np.int32), rng.normal(size=n_terms)


@pytest.mark.parametrize("rep", REPS)
def test_otoc_closed_form_terms_containing_a_and_b(rep):
    """If every term contains chi_a and chi_b, each term anticommutes with both,
    and the chain collapses to F_psi(t) = -1/4 <psi| e^{4itH} |psi> for every
    beta; F_tr(t) = -1/4 Tr e^{4itH} / dim."""
    N, a, b = 10, 9, 8
    q, J = _commuting_instance(N, a, b, 4, True)
    H = ham.dense_H(N, q, J, rep)
    X = mj.chis(N, rep)
    rng = np.random.default_rng(6)
    psi = _normed(rng.normal(size=H.shape[0]) + 1j * rng.normal(size=H.shape[0]))
    ts = [0.0, 0.4, 1.7, 3.2]
    for beta in (0.0, 2.5, 10.0):
        ref = [-0.25 * np.vdot(psi, sla.expm(4j * t * H) @ psi) for t in ts]
        assert np.allclose(otoc.F_state(H, X, a, b, beta, ts, psi), ref, atol=1e-12)
        reft = [-0.25 * np.trace(sla.expm(4j * t * H)) / H.shape[0] for t in ts]
        assert np.allclose(otoc.F_trace(H, X, a, b, beta, ts), reft, atol=1e-12)


@pytest.mark.parametrize("rep", REPS)
def test_otoc_closed_form_terms_avoiding_a_and_b(rep):
    """If no term contains a or b, chi_a and chi_b commute with H and
    F_psi(t) = -1/4 <psi| e^{-beta H} |psi>."""
    N, a, b = 10, 9, 8
    q, J = _commuting_instance(N, a, b, 6, False)
    H = ham.dense_H(N, q, J, rep)
    X = mj.chis(N, rep)
    rng = np.random.default_rng(7)
    psi = _normed(rng.normal(size=H.shape[0]) + 1j * rng.normal(size=H.shape[0]))
    for beta in (0.0, 3.0, 12.0):
        ref = -0.25 * np.vdot(psi, sla.expm(-beta * H) @ psi)
        got = otoc.F_state(H, X, a, b, beta, [0.0, 1.1, 4.0], psi)
        assert np.allclose(got, ref, atol=1e-12)


@pytest.mark.parametrize("rep", REPS)
def test_block_form_equals_full_space(rep):
    N = 10
    q, J = _instance(N, r=5)
    H = ham.dense_H(N, q, J, rep)
    HU, HD = ham.blocks(H, N, rep)
    X = mj.chis(N, rep)
    pU, pD = si.random_state(N, seed=9)
    full = mj.to_full(pU, pD, N, rep)
    ts = np.array([0.0, 0.5, 2.0, 4.5])
    for beta in (0.0, 5.0):
        a, b = N - 1, N - 2
        Ff = otoc.F_state(H, X, a, b, beta, ts, full)
        Fb = otoc.F_state_blocks(N, rep, HU, HD, X, a, b, beta, ts, pU, pD)
        assert np.allclose(Ff, Fb, atol=1e-13)
        Fs = otoc.F_state_sparse(N, rep, q, J, a, b, beta, ts, pU, pD)
        assert np.allclose(Fs, Fb, atol=1e-10)


@pytest.mark.parametrize("rep", REPS)
def test_trace_is_mean_over_basis_and_real(rep):
    N = 8
    q, J = _instance(N, r=6)
    H = ham.dense_H(N, q, J, rep)
    X = mj.chis(N, rep)
    ts = np.array([0.0, 0.8, 2.3])
    beta = 4.0
    Ft = otoc.F_trace(H, X, N - 1, N - 2, beta, ts)
    acc = sum(otoc.F_state(H, X, N - 1, N - 2, beta, ts, e) for e in np.eye(H.shape[0]))
    assert np.allclose(Ft, acc / H.shape[0], atol=1e-13)
    assert np.max(np.abs(Ft.imag)) < 1e-13


def test_trace_representation_independent():
    N = 10
    q, J = _instance(N, r=7)
    ts = np.array([0.0, 1.0, 3.0])
    F = [otoc.F_trace(ham.dense_H(N, q, J, rep), mj.chis(N, rep), N - 1, N - 2, 5.0, ts) for rep in REPS]
    assert np.allclose(F[0], F[1], atol=1e-12)


def test_typical_mean_close_to_trace():
    N = 10
    q, J = _instance(N, r=8)
    rep = "jw"
    H = ham.dense_H(N, q, J, rep)
    X = mj.chis(N, rep)
    ts = np.array([0.0, 1.0, 2.0])
    Ft = otoc.F_trace(H, X, N - 1, N - 2, 2.0, ts)
    S = 200
    acc = np.zeros(len(ts), dtype=np.complex128)
    for s in range(S):
        pU, pD = si.random_state(N, seed=100 + s)
        acc += otoc.F_state(H, X, N - 1, N - 2, 2.0, ts, mj.to_full(pU, pD, N, rep))
    # each state deviates by O(1/sqrt(dim)) relative; the mean of S by 1/sqrt(S dim)
    tol = 4.0 * 0.25 / math.sqrt(S * H.shape[0])
    assert np.all(np.abs(acc / S - Ft) < tol)


# --- seeded input generators both sides use
def test_philox_known_answers():
    """Known-answer vectors of Philox4x32-10 (Random123 distribution)."""
    kat = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        (
            [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
            [0xA4093822, 0x299F31D0],
            [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1],
        ),
    ]
    for c, k, ref in kat:
        got = si.philox4x32_10(np.array(c, dtype=np.uint64), np.array(k, dtype=np.uint64))
        assert [int(v) for v in got] == ref


def test_coupling_law():
    N, k = 32, 4
    Ts, vs = [], []
    for r in range(20):
        q, J, p = si.sample_sparse_syk(N, k, r=r)
        Ts.append(len(J))
        vs.append(np.mean(J ** 2) * p * N ** 3 / 6.0)
        assert np.all(q[:, 0] < q[:, 1]) and np.all(q[:, 2] < q[:, 3]) and np.all(q[:, 1] < q[:, 2])
    assert abs(np.mean(Ts) - k * N) < 4 * math.sqrt(k * N / 20)
    assert abs(np.mean(vs) - 1.0) < 0.1


# --- Green function (supplement, G(t) paragraph) closed forms
@pytest.mark.parametrize("rep", REPS)
def test_green_closed_forms(rep):
    N, a = 10, 9
    X = mj.chis(N, rep)
    rng = np.random.default_rng(8)
    ts = [0.0, 0.6, 2.2]
    # no term contains chi_a: chi_a commutes with H, G(t) = <psi|e^{-bH}|psi>/2 for all t
    q, J = _commuting_instance(N, a, 8, 5, False)
    H = ham.dense_H(N, q, J, rep)
    psi = _normed(rng.normal(size=H.shape[0]) + 1j * rng.normal(size=H.shape[0]))
    for beta in (0.0, 4.0):
        ref = 0.5 * np.vdot(psi, sla.expm(-beta * H) @ psi)
        assert np.allclose(otoc.G_state(H, X, a, beta, ts, psi), ref, atol=1e-12)
    # every term contains chi_a: chi_a e^{-iHt} chi_a = e^{iHt}/2, G(t) = <psi|e^{(2it-b)H}|psi>/2
    q, J = _commuting_instance(N, a, 8, 4, True)
    H = ham.dense_H(N, q, J, rep)
    for beta in (0.0, 3.0):
        ref = [0.5 * np.vdot(psi, sla.expm((2j * t - beta) * H) @ psi) for t in ts]
        assert np.allclose(otoc.G_state(H, X, a, beta, ts, psi), ref, atol=1e-12)


@pytest.mark.parametrize("rep", REPS)
def test_green_block_form_equals_full_space(rep):
    N = 10
    q, J = _instance(N, r=9)
    H = ham.dense_H(N, q, J, rep)
    HU, HD = ham.blocks(H, N, rep)
    X = mj.chis(N, rep)
    pU, pD = si.random_state(N, seed=3)
    ts = np.array([0.0, 0.7, 2.5])
    for beta in (0.0, 5.0):
        full = otoc.G_state(H, X, N - 1, beta, ts, mj.to_full(pU, pD, N, rep))
        blk = otoc.G_state_blocks(N, rep, HU, HD, X, N - 1, beta, ts, pU, pD)
        assert np.allclose(full, blk, atol=1e-13)
        # G(0) = <psi|e^{-bH}|psi>/2 for any H (chi_a^2 = 1/2)
        psi = mj.to_full(pU, pD, N, rep)
        assert np.isclose(full[0], 0.5 * np.vdot(psi, sla.expm(-beta * H) @ psi), atol=1e-13)


# --- Commuting-term tier (exact evolution by a product of single-term exponentials)
COMMUTING_QUADS = np.array([[0, 3, 5, 9], [1, 2, 6, 11], [4, 7, 8, 10], [0, 1, 2, 3]], dtype=np.int32)


def test_commuting_quads_really_commute():
    """The pin set: the fourth quadruple shares two indices with each of the
    first two and none with the third, so all dense products commute."""
    from oracle import commuting as cm

    N = 12
    X = mj.chis(N, "jw")
    P = [X[i] @ X[j] @ X[k] @ X[l] for i, j, k, l in COMMUTING_QUADS]
    for A in P:
        assert np.allclose(A @ A, np.eye(A.shape[0]) / 16.0, atol=1e-14)
        for B in P:
            assert np.allclose(A @ B, B @ A, atol=1e-14)
    cm.check_commuting(COMMUTING_QUADS)
    with pytest.raises(ValueError):
        cm.check_commuting(np.array([[0, 1, 2, 3], [0, 4, 5, 6]]))


@pytest.mark.parametrize("rep", REPS)
def test_commuting_evolve_matches_dense_eigh(rep):
    """e^{-zH} as a product of cosh - 4 sinh P factors equals the dense
    eigendecomposition e^{-zH} (a library routine) for complex z, both blocks:
    the fixed set above (terms split at their two lowest indices), and a
    matching-generated set whose terms are split along the matching's pairs
    (odd permutations included, so the reordering sign matters)."""
    from oracle import commuting as cm

    N = 12
    q2, J2, pairs = si.sample_commuting_syk(N, seed=5, n_terms=12)
    cases = [(COMMUTING_QUADS, np.array([0.9, -1.3, 0.4, 1.7]), None), (q2, J2, pairs)]
    assert any(cm._split_pairs(q, pairs)[2] < 0 for q in q2)
    v = np.random.default_rng(3).normal(size=1 << 5) + 1j * np.random.default_rng(4).normal(size=1 << 5)
    for quads, J, pr in cases:
        HU, HD = ham.blocks(ham.dense_H(N, quads, J, rep), N, rep)
        for blk, Hb in ((0, HU), (1, HD)):
            for z in (0.7, 2.5j, 1.2 - 3.0j):
                ref = dyn.evolve(Hb, z, v)
                got = cm.evolve(N, rep, quads, J, blk, z, v, pr)
                assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_commuting_otoc_matches_dense_block_formula():
    """The commuting-tier OTOC equals the dense parity-block OTOC (eigh) at
    N=12, on a matching-generated term set (F varies with t)."""
    from oracle import commuting as cm

    N = 12
    quads, J, pairs = si.sample_commuting_syk(N, seed=6, n_terms=10)
    H = ham.dense_H(N, quads, J, "jw")
    HU, HD = ham.blocks(H, N, "jw")
    X = mj.chis(N, "jw")
    pU, pD = si.random_state(N, seed=21)
    ts = [0.0, 0.8, 2.5]
    for a, b in ((N - 1, N - 2), (3, 8)):
        ref = otoc.F_state_blocks(N, "jw", HU, HD, X, a, b, 3.0, ts, pU, pD)
        got = cm.F_state(N, "jw", quads, J, a, b, 3.0, ts, pU, pD, pairs)
        assert np.max(np.abs(got - ref)) < 1e-12
        assert np.max(np.abs(ref - ref[0])) > 1e-3
