"""CPU checks of the Pauli-string (spin-chain) term compiler of libsyk
(syk_compile_pauli_host, the same host code syk_build_pauli_terms uploads):
the compiled block form reproduces the oracle's dense Hamiltonian exactly,
equal strings merge, zero sums drop, and bad input is refused with a status
and a message.  No GPU is needed."""
import ctypes as C
import os

import numpy as np
import pytest

import syk_inputs as si
from oracle import spin

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


def dense_from_compiled(L, c):
    """H[m, m ^ x] += coef (imag ? i : 1) (-1)^{popc(z & m)} from the compiled
    block form (the matrix element every kernel applies)."""
    D = 1 << L
    H = np.zeros((D, D), dtype=np.complex128)
    m = np.arange(D)
    for x, z, cf, im in zip(c["x"].tolist(), c["z"].tolist(), c["coef"].tolist(), c["imag"].tolist()):
        sgn = 1.0 - 2.0 * (np.bitwise_count(np.uint32(z) & m.astype(np.uint32)) & 1)
        H[m, m ^ x] += cf * (1j if im else 1.0) * sgn
    return H


@pytest.mark.parametrize("L,T,seed", [(1, 6, 0), (3, 30, 1), (6, 80, 2), (8, 40, 3)])
def test_compiled_form_equals_oracle_dense(pkg, L, T, seed):
    x, z, h = si.random_pauli_terms(L, T, seed=seed, max_weight=L)
    c = pkg.compile_pauli_host(L, x, z, h)
    assert np.allclose(dense_from_compiled(L, c), spin.dense_H(L, x, z, h), atol=1e-13)
    # imag flag = odd number of sigma_y
    for xi, zi, im in zip(c["x"].tolist(), c["z"].tolist(), c["imag"].tolist()):
        assert im == (bin(xi & zi).count("1") & 1)


def test_heisenberg_chain_compiles_exactly(pkg):
    L = 7
    x, z, h, _ = si.heisenberg_chain(L, W=3.0, r=2)
    c = pkg.compile_pauli_host(L, x, z, h)
    assert len(c["x"]) == 3 * L + L  # periodic: L bonds x (XX, YY, ZZ) + L fields
    assert not c["imag"].any()  # Y_i Y_j carries i^2: real
    assert np.allclose(dense_from_compiled(L, c), spin.dense_H(L, x, z, h), atol=1e-13)
    # XX and YY of a bond share a flip mask; every ZZ and field has x = 0
    assert len(set(c["x"].tolist())) == L + 1


def test_duplicates_merge_and_zero_sums_drop(pkg):
    L = 4
    x, z, h = si.random_pauli_terms(L, 10, seed=5)
    c1 = pkg.compile_pauli_host(L, x, z, h)
    c2 = pkg.compile_pauli_host(L, np.concatenate([x, x]), np.concatenate([z, z]), np.concatenate([h, h]))
    assert np.array_equal(c1["x"], c2["x"]) and np.array_equal(c1["z"], c2["z"])
    assert np.allclose(c2["coef"], 2 * c1["coef"])
    c0 = pkg.compile_pauli_host(L, np.concatenate([x, x]), np.concatenate([z, z]), np.concatenate([h, -h]))
    assert len(c0["x"]) == 0
    ce = pkg.compile_pauli_host(L, [], [], [])
    assert len(ce["x"]) == 0


def test_identity_string_is_a_shift(pkg):
    c = pkg.compile_pauli_host(3, [0], [0], [0.75])
    assert np.allclose(dense_from_compiled(3, c), 0.75 * np.eye(8))


def test_error_paths(pkg):
    from paper_2311_00639_b300 import _lib

    lib = _lib.load()
    n = C.c_int64(0)
    buf = C.create_string_buffer(256)

    def rc_of(L, x, z, h):
        xa, za, ha = (np.ascontiguousarray(a) for a in (np.asarray(x, np.uint32), np.asarray(z, np.uint32),
                                                         np.asarray(h, np.float64)))
        return lib.syk_compile_pauli_host(L, len(ha), xa.ctypes.data, za.ctypes.data, ha.ctypes.data, 0,
                                          C.byref(n), None, None, None, None)

    assert rc_of(3, [8], [0], [1.0]) == _lib.SYK_EINVAL  # X on qubit 3 of a 3-qubit chain
    lib.syk_last_error(buf, 256)
    assert b"n_qubits" in buf.value
    assert rc_of(3, [0], [16], [1.0]) == _lib.SYK_EINVAL
    assert rc_of(3, [1], [0], [np.nan]) == _lib.SYK_EINVAL
    assert rc_of(0, [0], [0], [1.0]) == _lib.SYK_EINVAL
    assert rc_of(32, [0], [0], [1.0]) == _lib.SYK_EINVAL
    assert rc_of(31, [1 << 30], [1 << 30], [1.0]) == _lib.SYK_OK
    # building or applying needs a device; without one the handle is not created
    h = C.c_void_p()
    xa = np.array([1], np.uint32)
    ha = np.array([1.0])
    rc = lib.syk_build_pauli_terms(3, 1, xa.ctypes.data, xa.ctypes.data, ha.ctypes.data, 7, C.byref(h))
    assert rc == _lib.SYK_EINVAL and not h.value  # bad dtype
