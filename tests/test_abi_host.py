"""CPU checks of the C-ABI library: it loads, exports every declared symbol,
rejects bad input with a status and message, and its host-side term compiler
reproduces the oracle's Hamiltonian blocks and Majorana blocks exactly."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import syk_inputs as si
from oracle import hamiltonian as ham
from oracle import majorana as mj

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


def declared_functions():
    src = open(os.path.join(ROOT, "include", "syk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(syk_[A-Za-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(pkg):
    from paper_2311_00639_b300 import _lib

    lib = C.CDLL(_lib.LIB_PATH)
    names = declared_functions()
    assert len(names) == len(_lib.SIGNATURES)
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, n
    assert _lib.load().syk_version().startswith(b"libsyk")


def test_error_paths_host(pkg):
    from paper_2311_00639_b300 import _lib

    lib = _lib.load()
    n = C.c_int64(0)
    bad = np.array([[3, 2, 1, 0]], dtype=np.int32)
    J = np.array([1.0])
    rc = lib.syk_compile_terms_host(8, 1, bad.ctypes.data, J.ctypes.data, 0, 0, C.byref(n), None, None, None, None,
                                    None)
    assert rc == _lib.SYK_EINVAL
    buf = C.create_string_buffer(256)
    lib.syk_last_error(buf, 256)
    assert b"strictly increasing" in buf.value
    rc = lib.syk_compile_terms_host(7, 0, None, None, 0, 0, C.byref(n), None, None, None, None, None)
    assert rc == _lib.SYK_EINVAL
    oob = np.array([[0, 1, 2, 8]], dtype=np.int32)
    assert lib.syk_compile_terms_host(8, 1, oob.ctypes.data, J.ctypes.data, 0, 0, C.byref(n), None, None, None,
                                      None, None) == _lib.SYK_EINVAL
    nan = np.array([np.nan])
    ok = np.array([[0, 1, 2, 3]], dtype=np.int32)
    assert lib.syk_compile_terms_host(8, 1, ok.ctypes.data, nan.ctypes.data, 0, 0, C.byref(n), None, None, None,
                                      None, None) == _lib.SYK_EINVAL
    assert lib.syk_compile_terms_host(8, 1, ok.ctypes.data, J.ctypes.data, 5, 0, C.byref(n), None, None, None,
                                      None, None) == _lib.SYK_EINVAL
    # null handles are rejected, not dereferenced
    assert lib.syk_apply_H(None, 0, None, None, 1, None) == _lib.SYK_EINVAL
    assert lib.syk_terms_get_info(None, None) == _lib.SYK_EINVAL


def dense_from_strings(D, x, z, coef, imag):
    """(H psi)[m] = sum_t coef_t (i if imag) (-1)^{popc(z_t & m)} psi[m ^ x_t]."""
    H = np.zeros((D, D), dtype=np.complex128)
    m = np.arange(D)
    for xt, zt, ct, it in zip(x, z, coef, imag):
        sign = 1.0 - 2.0 * (np.bitwise_count(m & int(zt)) & 1)
        H[m, m ^ int(xt)] += ct * (1j if it else 1.0) * sign
    return H


@pytest.mark.parametrize("rep", ["jw", "paper"])
@pytest.mark.parametrize("N", [4, 6, 8, 10, 12])
def test_host_terms_match_oracle_blocks(pkg, rep, N):
    q, J, _ = si.sample_sparse_syk(N, 4, r=N)
    if N <= 6:
        q = si.all_quads(N)
        J = np.random.default_rng(N).normal(size=len(q))
    out = pkg.compile_terms_host(N, q, J, rep)
    D = 1 << (N // 2 - 1)
    HU, HD = ham.blocks(ham.dense_H(N, q, J, rep), N, rep)
    assert np.allclose(dense_from_strings(D, out["x"], out["z"], out["coef_U"], out["imag"]), HU, atol=1e-14)
    assert np.allclose(dense_from_strings(D, out["x"], out["z"], out["coef_D"], out["imag"]), HD, atol=1e-14)
    # real terms first, then imaginary ones
    assert np.all(np.diff(out["imag"].astype(int)) >= 0)


def test_dense_N8_merges_parity_partners(pkg):
    """At N=8, chi0..chi3 and chi4..chi7 differ by the parity operator and
    become the same block string; the compiler merges them per block."""
    q = si.all_quads(8)
    J = np.random.default_rng(1).normal(size=len(q))
    for rep in ("jw", "paper"):
        out = pkg.compile_terms_host(8, q, J, rep)
        assert len(out["x"]) < len(q)
        HU, HD = ham.blocks(ham.dense_H(8, q, J, rep), 8, rep)
        assert np.allclose(dense_from_strings(8, out["x"], out["z"], out["coef_U"], out["imag"]), HU, atol=1e-13)
        assert np.allclose(dense_from_strings(8, out["x"], out["z"], out["coef_D"], out["imag"]), HD, atol=1e-13)


@pytest.mark.parametrize("rep", ["jw", "paper"])
@pytest.mark.parametrize("N", [4, 8, 10])
def test_host_chi_match_oracle(pkg, rep, N):
    X = mj.chis(N, rep)
    D = 1 << (N // 2 - 1)
    for n in range(N):
        c = pkg.compile_chi_host(N, n, rep)
        for P in (0, 1):
            ref = ham.block_of(X[n], N, rep, 1 - P, P)
            got = dense_from_strings(D, [c["x"]], [c["z"]], [c["coef"][P]], [False])
            assert np.allclose(got, ref, atol=1e-15), (n, P)


def test_paper_rep_special_chis(pkg):
    """chi_{N-1}: U->D by +i/sqrt2, D->U by -i/sqrt2; chi_{N-2}: sigma_z on the
    top block qubit over sqrt2 (supplement, simplification of the OTOC)."""
    N = 16
    L = N // 2 - 1
    c1 = pkg.compile_chi_host(N, N - 1, "paper")
    assert c1["x"] == 0 and c1["z"] == 0
    assert np.allclose(c1["coef"], [1j / np.sqrt(2), -1j / np.sqrt(2)])
    c2 = pkg.compile_chi_host(N, N - 2, "paper")
    assert c2["x"] == 0 and c2["z"] == 1 << (L - 1)
    assert np.allclose(c2["coef"], [1 / np.sqrt(2), 1 / np.sqrt(2)])


def test_N64_jw_terms_flip_at_most_four_bits(pkg):
    q, J, _ = si.sample_sparse_syk(64, 4, r=0)
    out = pkg.compile_terms_host(64, q, J, "jw")
    assert len(out["x"]) == len(q)
    assert np.max(np.bitwise_count(out["x"])) <= 4
    assert np.all(out["x"] < (1 << 31)) and np.all(out["z"] < (1 << 31))
