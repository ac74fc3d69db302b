"""Pins of the non-Hermitian SYK oracle (oracle/nonherm.py): the Hermitian
limit reduces to the beta = 0 OTOC of Eq. (2); the adjoint of a complex
coupling sum is the conjugate-coupling sum; a single complex term has a
closed-form exponential; when every term anticommutes with chi_a and chi_b the
OTOC chain collapses to a product of evolutions with no Majorana left; the
trace is the mean over basis states, and typical states estimate it."""
import numpy as np
import pytest
import scipy.linalg as sla

import syk_inputs as si
from oracle import dynamics as dyn
from oracle import hamiltonian as ham
from oracle import majorana as mj
from oracle import nonherm as nh
from oracle import otoc

REPS = ["jw", "paper"]


def _instance(N, k=4, r=0):
    q, J, _ = si.sample_sparse_syk(N, k, r=r)
    M = np.random.default_rng(100 + r).normal(size=len(J)) * np.std(J)
    return q, J, M


def _normed(v):
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("rep", REPS)
def test_hermitian_limit_is_beta0_otoc(rep):
    N = 10
    q, J, _ = _instance(N, r=1)
    H = nh.dense_H(N, q, J, np.zeros_like(J), rep)
    assert np.allclose(H, ham.dense_H(N, q, J, rep))
    X = mj.chis(N, rep)
    rng = np.random.default_rng(2)
    psi = _normed(rng.normal(size=H.shape[0]) + 1j * rng.normal(size=H.shape[0]))
    ts = [0.0, 0.7, 2.0]
    assert np.allclose(nh.F_state(H, X, N - 1, N - 2, ts, psi), otoc.F_state(H, X, N - 1, N - 2, 0.0, ts, psi),
                       atol=1e-12)
    assert np.allclose(nh.F_trace(H, X, N - 1, N - 2, ts), otoc.F_trace(H, X, N - 1, N - 2, 0.0, ts), atol=1e-12)


@pytest.mark.parametrize("rep", REPS)
def test_adjoint_is_conjugate_couplings(rep):
    N = 10
    q, J, M = _instance(N, r=2)
    H = nh.dense_H(N, q, J, M, rep)
    Hd = nh.dense_H(N, q, J, -M, rep)
    assert np.allclose(H.conj().T, Hd, atol=1e-14)
    assert not np.allclose(H, Hd)  # genuinely non-Hermitian
    # parity blocks survive complex couplings
    iU, iD = mj.block_indices(N, rep)
    assert np.allclose(H[np.ix_(iU, iD)], 0) and np.allclose(H[np.ix_(iD, iU)], 0)


def test_single_complex_term_closed_form():
    """H = w chi_0 chi_1 chi_2 chi_3 with P = chi chi chi chi, P^2 = 1/16:
    e^{-zH} = cosh(z w / 4) - 4 sinh(z w / 4) P for complex w."""
    N = 8
    X = mj.chis(N, "jw")
    P = X[0] @ X[1] @ X[2] @ X[3]
    assert np.allclose(P @ P, np.eye(P.shape[0]) / 16)
    w = 0.9 - 0.6j
    H = nh.dense_H(N, np.array([[0, 1, 2, 3]], np.int32), [w.real], [w.imag], "jw")
    rng = np.random.default_rng(3)
    x = rng.normal(size=H.shape[0]) + 1j * rng.normal(size=H.shape[0])
    for z in (0.5, 1.5j, 0.3 - 2.0j):
        ref = np.cosh(z * w / 4) * x - 4 * np.sinh(z * w / 4) * (P @ x)
        assert np.allclose(nh.evolve(H, z, x), ref, atol=1e-12)


def test_sparse_and_dense_evolution_agree():
    N = 14
    q, J, M = _instance(N, r=3)
    rep = "jw"
    HU = ham.blocks(nh.dense_H(N, q, J, M, rep), N, rep)[0]
    Hc = nh.csr_block(N, q, J, M, rep, 0)
    assert np.allclose(Hc.toarray(), HU, atol=1e-14)
    x = _normed(np.random.default_rng(4).normal(size=HU.shape[0]) + 0j)
    assert np.allclose(nh.evolve_sparse(Hc, 0.4 + 2.0j, x), nh.evolve(HU, 0.4 + 2.0j, x), atol=1e-11)
    # non-unitary: the norm changes under e^{-iHt}
    assert abs(np.linalg.norm(nh.evolve(HU, 2.0j, x)) - 1.0) > 1e-3


def test_otoc_closed_form_all_terms_contain_a_and_b():
    """Every term contains chi_a and chi_b, so both anticommute with H and
    H^dag; the chain collapses to
    F_psi(t) = -1/4 <psi| e^{itH^dag} e^{itH} e^{itH^dag} e^{itH} |psi>."""
    N, a, b = 10, 9, 8
    rng = np.random.default_rng(11)
    others = [i for i in range(N) if i not in (a, b)]
    quads = np.array([sorted([a, b] + [int(v) for v in rng.choice(others, 2, replace=False)]) for _ in range(4)],
                     np.int32)
    J, M = rng.normal(size=4), rng.normal(size=4)
    H = nh.dense_H(N, quads, J, M, "jw")
    X = mj.chis(N, "jw")
    psi = _normed(rng.normal(size=H.shape[0]) + 1j * rng.normal(size=H.shape[0]))
    ts = [0.0, 0.5, 1.3]
    ref = []
    for t in ts:
        A, B = sla.expm(1j * t * H.conj().T), sla.expm(1j * t * H)
        ref.append(-0.25 * np.vdot(psi, A @ B @ A @ B @ psi))
    assert np.allclose(nh.F_state(H, X, a, b, ts, psi), ref, atol=1e-12)


def test_trace_is_mean_over_basis_and_t0_value():
    N = 8
    q, J, M = _instance(N, r=5)
    H = nh.dense_H(N, q, J, M, "jw")
    X = mj.chis(N, "jw")
    ts = [0.0, 0.6, 1.8]
    Ft = nh.F_trace(H, X, N - 1, N - 2, ts)
    acc = sum(nh.F_state(H, X, N - 1, N - 2, ts, e) for e in np.eye(H.shape[0]))
    assert np.allclose(Ft, acc / H.shape[0], atol=1e-13)
    assert np.isclose(Ft[0], -0.25, atol=1e-14)  # chi_a chi_b chi_a chi_b = -1/4 at t = 0


def test_typical_states_estimate_the_trace():
    """As for the Hermitian OTOC: the mean over normalised complex-Gaussian
    states approaches the exact trace within O(|F| / sqrt(S dim))."""
    N = 10
    q, J, M = _instance(N, r=6)
    H = nh.dense_H(N, q, J, 0.3 * M, "jw")
    X = mj.chis(N, "jw")
    ts = [0.0, 0.8]
    Ft = nh.F_trace(H, X, N - 1, N - 2, ts)
    S = 200
    rng = np.random.default_rng(13)
    acc = np.zeros(len(ts), dtype=np.complex128)
    for _ in range(S):
        acc += nh.F_state(H, X, N - 1, N - 2, ts, _normed(rng.normal(size=H.shape[0]) + 1j * rng.normal(size=H.shape[0])))
    assert np.all(np.abs(acc / S - Ft) < 6.0 * np.max(np.abs(Ft)) / np.sqrt(S * H.shape[0]))
