"""The projected-exponential step of the Krylov engine (syk_tridiag_exp) on
given Lanczos matrices: c = e^{-s z T} e_1 against scipy's expm of the small
matrix (a library routine), for the lane-parallel eigensolver and for the QL
fallback, on well-separated spectra (the lane-parallel path must be taken) and
on clustered ones (the checks must hand over to QL).  The accepted fraction s
passes the a-posteriori error estimate: err <= tol * s."""
import numpy as np
import pytest
import scipy.linalg as sla

pytestmark = pytest.mark.gpu

ZS = [0.7j, 1.5 + 3.0j, 4.0 - 10.0j, 2.5]


@pytest.fixture(scope="module")
def syk():
    import paper_2311_00639_b300 as p

    return p


def lanczos(A, v, m):
    """Plain Lanczos (full reorthogonalisation) on a symmetric matrix: alpha,
    beta with beta[m-1] the residual norm."""
    V = [v / np.linalg.norm(v)]
    al, be = [], []
    for j in range(m):
        w = A @ V[j]
        a = V[j] @ w
        w = w - a * V[j] - (be[-1] * V[j - 1] if j else 0)
        for u in V:
            w = w - (u @ w) * u
        b = np.linalg.norm(w)
        al.append(a)
        be.append(b)
        V.append(w / b)
    return np.array(al), np.array(be)


def expm_first_column(al, be, z, s):
    m = len(al)
    T = np.diag(al) + np.diag(be[: m - 1], 1) + np.diag(be[: m - 1], -1)
    return sla.expm(-s * z * T)[:, 0]


def check(syk, al, be, z, tol, force_ql):
    c, s, err, used_ql = syk.tridiag_exp(al, be, z, tol, force_ql=force_ql)
    assert 0.0 < s <= 1.0
    assert err <= tol * s * (1 + 1e-12)
    ref = expm_first_column(al, be, z, s)
    # e^{-s z lam} spans e^{+-7.5} for real z here: c = sum_k f(lam_k) z_k z_k[0] cancels
    # by up to ~1e2 relative to max |c|, so 1e-12 is a few ulps of the largest term
    assert np.max(np.abs(c - ref)) < 1e-12 * np.max(np.abs(ref)), (len(al), z, force_ql, used_ql)
    return s, used_ql


@pytest.mark.parametrize("m", [5, 20, 30, 48, 64])
def test_separated_spectrum_both_paths(syk, m):
    rng = np.random.default_rng(m)
    lam = np.sort(rng.uniform(-3.0, 3.0, 2000))  # a dense spectrum: Ritz values stay apart
    al, be = lanczos(np.diag(lam), rng.normal(size=2000), m)
    # with m = 5 the estimate's rounding floor (~1e-16 / s) and its O(s^4)
    # truncation leave no fraction s that passes tol = 1e-12
    tol = 1e-12 if m >= 20 else 1e-9
    for z in ZS:
        s_fast, used = check(syk, al, be, z, tol, False)
        assert not used, "the lane-parallel path should accept a separated spectrum"
        s_ql, used_q = check(syk, al, be, z, tol, True)
        assert used_q
        assert s_fast == s_ql


@pytest.mark.parametrize("k", [4, 15, 32])
def test_clustered_spectrum_falls_back_to_ql(syk, k):
    """Two copies of one tridiagonal block joined by beta = 1e-9: the
    eigenvalues come in pairs about 1e-9 apart, so the lane-parallel checks
    must hand over to QL, and the result must still be right."""
    rng = np.random.default_rng(100 + k)
    a1 = rng.normal(size=k)
    b1 = np.abs(rng.normal(size=k)) + 0.2
    al = np.concatenate([a1, a1])
    be = np.concatenate([b1[: k - 1], [1e-9], b1[: k - 1], [0.3]])
    for z in ZS:
        _, used = check(syk, al, be, z, 1e-12, False)
        assert used, "clustered eigenvalues must take the QL path"


def test_step_time_m30(syk):
    """The projected-exponential step at m = 30 (the complex128 default) on a
    separated spectrum: lane-parallel path well under 0.1 ms per call (FP64
    on this part costs ~64 cycles of issue per warp instruction; the
    lane-replicated QL recurrence took ~1 ms)."""
    rng = np.random.default_rng(30)
    lam = np.sort(rng.uniform(-3.0, 3.0, 2000))
    al, be = lanczos(np.diag(lam), rng.normal(size=2000), 30)
    *_, used, ms = syk.tridiag_exp(al, be, 1.5 + 3.0j, 1e-12, timed=True)
    *_, used_q, ms_q = syk.tridiag_exp(al, be, 1.5 + 3.0j, 1e-12, force_ql=True, timed=True)
    print(f"m=30 step: lane-parallel {ms:.4f} ms, QL {ms_q:.4f} ms")
    assert not used and used_q
    assert ms < 0.1
