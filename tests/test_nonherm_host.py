"""CPU checks of the complex-coupling (non-Hermitian SYK) term compiler of
libsyk (syk_compile_terms_complex_host, the host code syk_build_terms_complex
uploads): its block strings reproduce the oracle's non-Hermitian blocks
exactly in both representations, reduce to the Hermitian compiler when the
imaginary couplings vanish, and obey the documented adjoint rule (conjugate
couplings = conj(value) (-1)^{popc(x & z)} per string).  No GPU is needed."""
import os

import numpy as np
import pytest

import syk_inputs as si
from oracle import hamiltonian as ham
from oracle import nonherm as nh

from .test_abi_host import dense_from_strings

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import importlib.util

    spec = importlib.util.spec_from_file_location("_syk_build", os.path.join(ROOT, "paper_2311_00639_b300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()
    import paper_2311_00639_b300 as p

    return p


def _instance(N, r):
    q, J, _ = si.sample_sparse_syk(N, 4, r=r)
    if N <= 6:
        q = si.all_quads(N)
        J = np.random.default_rng(N).normal(size=len(q))
    M = np.random.default_rng(50 + r).normal(size=len(J)) * np.sqrt(np.mean(J ** 2))
    return q, J, M


@pytest.mark.parametrize("rep", ["jw", "paper"])
@pytest.mark.parametrize("N", [4, 6, 8, 10, 12])
def test_complex_terms_match_oracle_blocks(pkg, rep, N):
    q, J, M = _instance(N, N)
    out = pkg.compile_terms_complex_host(N, q, J, M, rep)
    D = 1 << (N // 2 - 1)
    HU, HD = ham.blocks(nh.dense_H(N, q, J, M, rep), N, rep)
    assert np.allclose(dense_from_strings(D, out["x"], out["z"], out["coef_U"], out["imag"]), HU, atol=1e-14)
    assert np.allclose(dense_from_strings(D, out["x"], out["z"], out["coef_D"], out["imag"]), HD, atol=1e-14)
    assert not np.allclose(HU, HU.conj().T)


@pytest.mark.parametrize("rep", ["jw", "paper"])
def test_zero_imaginary_couplings_give_the_hermitian_table(pkg, rep):
    N = 14
    q, J, _ = _instance(N, 3)
    a = pkg.compile_terms_complex_host(N, q, J, np.zeros_like(J), rep)
    b = pkg.compile_terms_host(N, q, J, rep)
    for k in ("x", "z", "coef_U", "coef_D", "imag"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("rep", ["jw", "paper"])
def test_adjoint_rule(pkg, rep):
    """The strings of H(J - iM) are those of H(J + iM) with each value w
    replaced by conj(w) (-1)^{popc(x & z)} (the rule syk_terms_adjoint applies)."""
    N = 12
    q, J, M = _instance(N, 4)
    fwd = pkg.compile_terms_complex_host(N, q, J, M, rep)
    adj = pkg.compile_terms_complex_host(N, q, J, -M, rep)
    sg = 1.0 - 2.0 * (np.bitwise_count(fwd["x"] & fwd["z"]) & 1)
    f = np.where(fwd["imag"] == 1, -sg, sg)
    key = lambda d, cu, cd: sorted(zip(d["x"].tolist(), d["z"].tolist(), d["imag"].tolist(), np.round(cu, 15).tolist(),
                                       np.round(cd, 15).tolist()))
    assert key(fwd, fwd["coef_U"] * f, fwd["coef_D"] * f) == key(adj, adj["coef_U"], adj["coef_D"])
    D = 1 << (N // 2 - 1)
    HU = dense_from_strings(D, fwd["x"], fwd["z"], fwd["coef_U"] * f, fwd["imag"])
    HUf = dense_from_strings(D, fwd["x"], fwd["z"], fwd["coef_U"], fwd["imag"])
    assert np.allclose(HU, HUf.conj().T, atol=1e-14)
