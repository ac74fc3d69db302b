"""GPU parity of the Pauli-string (spin-chain) path against the CPU oracle.

Every call goes through the C-ABI (syk_build_pauli_terms, syk_apply_H,
syk_apply_pauli, syk_krylov_evolve, syk_pauli_otoc).  Workload: the
random-field Heisenberg chain of many-body-localisation studies (the paper's
outlook) and random Pauli strings carrying sigma_y on many qubits.  Sizes span
the small-vector kernels (D < 2048), the tiled complex64 / complex128 kernels
with forced multi-pass plans, and the 2^31-amplitude chain the benchmark times
(sampled rows).  Tolerances as for the SYK path: complex128 H psi 1e-12 of the
largest entry, complex64 2e-5; Krylov results 1e-10 / 5e-5; OTOC 1e-10 /
1e-4 absolute on F (|F| <= 1).
"""
import numpy as np
import pytest

import syk_inputs as si
from oracle import dynamics as dyn
from oracle import otoc as ot
from oracle import spin

pytestmark = pytest.mark.gpu

TOL_H = {"c128": 1e-12, "c64": 2e-5}


def _dev(a, dtype):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.complex128 if dtype == "c128" else
                                                         torch.complex64)


def _state(D, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=D) + 1j * rng.normal(size=D)
    return v / np.linalg.norm(v)


def _rel(got, ref):
    return np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("L,kind", [(1, "rand"), (5, "rand"), (10, "rand"), (9, "heis"), (12, "heis"),
                                    (13, "rand"), (12, "many")])
def test_apply_H_matches_oracle(dtype, L, kind):
    """Small vectors (dense oracle), a few tiles (CSR oracle), and 300 strings
    on 4096 amplitudes (complex64 splits the pass across CTAs by chunks)."""
    import paper_2311_00639_b300 as syk

    if kind == "heis":
        x, z, h, _ = si.heisenberg_chain(L, W=4.0, r=L)
    elif kind == "many":
        x, z, h = si.random_pauli_terms(L, 300, seed=200 + L, max_weight=6)
    else:
        x, z, h = si.random_pauli_terms(L, 3 * L + 4, seed=100 + L, max_weight=min(L, 5))
    H = spin.dense_H(L, x, z, h) if L <= 10 else spin.csr_H(L, x, z, h)
    psi = np.stack([_state(1 << L, 1), _state(1 << L, 2)])
    with syk.PauliTerms(L, x, z, h, dtype=dtype) as t:
        assert t.D == 1 << L and t.info["rep"] == 2 and t.info["N"] == 0
        got = t.apply_H(_dev(psi, dtype), 0).cpu().numpy()
        ref = np.stack([H @ psi[0], H @ psi[1]])
        assert _rel(got, ref) < TOL_H[dtype], (L, kind, dtype, _rel(got, ref))
        assert t.device_error() == 0


@pytest.mark.parametrize("dtype,budget", [("c64", 1 << 14), ("c64", 1 << 15), ("c128", 1 << 15)])
def test_apply_H_multi_pass_plans(dtype, budget):
    """L = 16 (D = 65536) with small L2 budgets: several passes, stragglers,
    super-tiles; against the oracle's CSR matrix (basis-state maps)."""
    import paper_2311_00639_b300 as syk

    L = 16
    x, z, h, _ = si.heisenberg_chain(L, W=2.0, r=7)
    x2, z2, h2 = si.random_pauli_terms(L, 40, seed=9, max_weight=4)
    x, z, h = np.concatenate([x, x2]), np.concatenate([z, z2]), np.concatenate([h, h2])
    Hc = spin.csr_H(L, x, z, h)
    psi = _state(1 << L, 3)
    ref = Hc @ psi
    with syk.PauliTerms(L, x, z, h, dtype=dtype) as t:
        assert t.replan(budget, 0.0) >= 2  # no stragglers: the high-bit bonds need their own pass
        got = t.apply_H(_dev(psi, dtype), 0).cpu().numpy()
        assert _rel(got, ref) < TOL_H[dtype]
        for ratio in (3.0, 1.5):  # light passes dissolved into heavier ones as stragglers
            t.replan(budget, ratio)
            got = t.apply_H(_dev(psi, dtype), 0).cpu().numpy()
            assert _rel(got, ref) < TOL_H[dtype]
        t.replan(0, 0)
        got = t.apply_H(_dev(psi, dtype), 0).cpu().numpy()
        assert _rel(got, ref) < TOL_H[dtype]


@pytest.mark.parametrize("L,dtype", [(24, "c128"), (31, "c64")])
def test_apply_H_sampled_rows_large(L, dtype):
    """The benchmark's chain (L = 31, D = 2^31, complex64, default plan) and a
    complex128 L = 24 chain: sampled rows against the definition."""
    import torch

    import paper_2311_00639_b300 as syk

    x, z, h, _ = si.heisenberg_chain(L, W=5.0, r=0)
    with syk.PauliTerms(L, x, z, h, dtype=dtype) as t:
        seed = 31
        psi, _ = t.random_state(seed, 0, blocks=(0,))
        out = t.apply_H(psi, 0)
        torch.cuda.synchronize()
        rng = np.random.default_rng(4)
        rows = np.concatenate([[0, (1 << L) - 1], rng.integers(0, 1 << L, 2000)]).astype(np.uint64)
        got = out[torch.from_numpy(rows.astype(np.int64)).to("cuda")].cpu().numpy().astype(np.complex128)
        N = 2 * L + 2  # the Philox counter of block 0 is the basis index
        ref = spin.rows_of_Hpsi(L, x, z, h, rows, lambda g: si.philox_state(N, seed, 0, g))
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(got - ref)) / scale < (1e-12 if dtype == "c128" else 2e-5)
        assert t.device_error() == 0
        del psi, out


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("L", [4, 12])
def test_apply_pauli_matches_basis_maps(dtype, L):
    import paper_2311_00639_b300 as syk

    x, z, h, _ = si.heisenberg_chain(L, W=1.0, r=1)
    psi = _state(1 << L, 5)
    cols = np.arange(1 << L, dtype=np.uint64)
    strings = [si.pauli_mask({0: "X"}), si.pauli_mask({1: "Y", L - 1: "Z"}), si.pauli_mask({0: "Z", 2: "Z"}),
               si.pauli_mask({q: "Y" for q in range(L)}), (0, 0)]

    def ref_of(px, pz, v):
        g, ph = spin.apply_map(L, px, pz, cols)  # P|m> = ph |g>
        r = np.zeros_like(v)
        r[g.astype(np.int64)] = ph * v
        return r

    with syk.PauliTerms(L, x, z, h, dtype=dtype) as t:
        for (px, pz) in strings:
            got = t.apply_pauli(px, pz, _dev(psi, dtype)).cpu().numpy()
            assert np.max(np.abs(got - ref_of(px, pz, psi))) < (1e-14 if dtype == "c128" else 1e-6), (px, pz)
        d = _dev(psi, dtype)  # diagonal string in place
        t.apply_pauli(0, 5, d, out=d)
        assert np.max(np.abs(d.cpu().numpy() - ref_of(0, 5, psi))) < 1e-6


def test_krylov_evolve_matches_eigh_and_expm_multiply():
    import paper_2311_00639_b300 as syk

    L = 10
    x, z, h = si.random_pauli_terms(L, 40, seed=12, max_weight=4)
    Hd = spin.dense_H(L, x, z, h)
    psi = _state(1 << L, 6)
    with syk.PauliTerms(L, x, z, h, dtype="c128") as t:
        for tau, tt in ((0.0, 2.0), (0.4, -1.5), (1.0, 0.0)):
            y, st = t.krylov_evolve(_dev(psi, "c128"), 0, tau, tt)
            ref = dyn.evolve(Hd, tau + 1j * tt, psi)
            assert _rel(y.cpu().numpy(), ref) < 1e-10
            assert st.matvecs > 0
    L = 15
    x, z, h, _ = si.heisenberg_chain(L, W=3.0, r=2)
    psi = _state(1 << L, 7)
    ref = dyn.evolve_sparse(spin.csr_H(L, x, z, h), 0.5 + 3.0j, psi)
    with syk.PauliTerms(L, x, z, h, dtype="c64") as t:
        y, _ = t.krylov_evolve(_dev(psi, "c64"), 0, 0.5, 3.0)
        assert _rel(y.cpu().numpy(), ref) < 5e-5


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("L", [2, 3, 4])
def test_krylov_tiny_chains(dtype, L):
    """Vectors of fewer than 256 bytes: the stored Lanczos basis is indexed at
    j * D amplitudes."""
    import paper_2311_00639_b300 as syk

    x, z, h = si.random_pauli_terms(L, 3 * L, seed=300 + L, max_weight=L)
    Hd = spin.dense_H(L, x, z, h)
    psi = _state(1 << L, 11)
    with syk.PauliTerms(L, x, z, h, dtype=dtype) as t:
        y, _ = t.krylov_evolve(_dev(psi, dtype), 0, 0.3, 2.0)
        assert _rel(y.cpu().numpy(), dyn.evolve(Hd, 0.3 + 2.0j, psi)) < (1e-10 if dtype == "c128" else 5e-5)


def test_pauli_otoc_same_state_and_philox_state_complex128():
    import paper_2311_00639_b300 as syk

    L = 9
    x, z, h, _ = si.heisenberg_chain(L, W=2.0, r=3)
    Hd = spin.dense_H(L, x, z, h)
    eig = dyn.eig(Hd)
    W = si.pauli_mask({0: "Z"})
    V = si.pauli_mask({4: "Z"})
    X = {0: spin.pauli_dense(L, *W), 1: spin.pauli_dense(L, *V)}
    ts = [0.0, 0.5, 1.5, 3.0]
    beta = 2.0
    psi = np.stack([_state(1 << L, 8), _state(1 << L, 9)])
    with syk.PauliTerms(L, x, z, h, dtype="c128") as t:
        F, o, st = t.pauli_otoc(W, V, beta, ts, psi=_dev(psi, "c128"))
        for s in range(2):
            ref = ot.F_state(Hd, X, 0, 1, beta, ts, psi[s], eigpair=eig)
            assert np.max(np.abs(F[s] - ref)) < 1e-10
        mean = F.mean(axis=0)
        assert np.allclose(o, mean.real / mean.real[0], atol=1e-12)
        # Philox typical states: block-0 counters, normalised over the D amplitudes
        F2, _, _ = t.pauli_otoc(W, V, beta, ts, n_states=2, seed=77)
        for s in range(2):
            v = si.philox_state(2 * L + 2, 77, s)[: 1 << L]
            ref = ot.F_state(Hd, X, 0, 1, beta, ts, v / np.linalg.norm(v), eigpair=eig)
            assert np.max(np.abs(F2[s] - ref)) < 1e-10


def test_pauli_otoc_exact_trace_and_closed_form():
    import paper_2311_00639_b300 as syk

    L = 6
    x, z, h, _ = si.heisenberg_chain(L, W=1.5, r=4)
    Hd = spin.dense_H(L, x, z, h)
    W = si.pauli_mask({0: "Z"})
    V = si.pauli_mask({3: "X"})
    X = {0: spin.pauli_dense(L, *W), 1: spin.pauli_dense(L, *V)}
    ts = [0.0, 0.7, 2.0]
    with syk.PauliTerms(L, x, z, h, dtype="c128") as t:
        F, o, _ = t.pauli_otoc(W, V, 3.0, ts, mode="exact")
        ref = ot.F_trace(Hd, X, 0, 1, 3.0, ts)
        assert np.max(np.abs(F[0] - ref)) < 1e-10
        assert np.allclose(o, ref.real / ref.real[0], atol=1e-10)
    # H = h Z_0 + g Z_1, W = V = X_0, beta = 0: F(t) = cos(4 h t)
    hh = 0.37
    tg = np.array([0.0, 0.3, 1.0, 2.2])
    with syk.PauliTerms(2, [0, 0], [1, 2], [hh, 1.3], dtype="c128") as t:
        F, _, _ = t.pauli_otoc((1, 0), (1, 0), 0.0, tg, mode="exact")
        assert np.allclose(F[0], np.cos(4 * hh * tg), atol=1e-12)


def test_pauli_otoc_complex64_against_oracle_and_shift():
    """complex64 states against the oracle (relative to the largest |F|: the
    raw F of a spin chain grows like e^{beta |E_min|}), and the identity-string
    shift H -> H + c that keeps complex64 weights in range: F -> e^{-beta c} F
    exactly, the OTOC ratio unchanged."""
    import paper_2311_00639_b300 as syk

    L = 12
    x, z, h, _ = si.heisenberg_chain(L, W=3.0, r=5)
    Hd = spin.dense_H(L, x, z, h)
    W = si.pauli_mask({0: "Z"})
    V = si.pauli_mask({6: "Z"})
    X = {0: spin.pauli_dense(L, *W), 1: spin.pauli_dense(L, *V)}
    ts = [0.0, 1.0, 2.5]
    beta, c = 4.0, 9.0
    psi = _state(1 << L, 10)
    ref = ot.F_state(Hd, X, 0, 1, beta, ts, psi)
    with syk.PauliTerms(L, x, z, h, dtype="c64") as t:
        F, o, _ = t.pauli_otoc(W, V, beta, ts, psi=_dev(psi[None, :], "c64"))
        assert _rel(F[0], ref) < 1e-4
        assert np.allclose(o, ref.real / ref.real[0], atol=1e-4)
    xs, zs, hs = np.append(x, 0), np.append(z, 0), np.append(h, c)
    for dtype, lim in (("c64", 1e-4), ("c128", 1e-10)):
        with syk.PauliTerms(L, xs, zs, hs, dtype=dtype) as t:
            F, o, _ = t.pauli_otoc(W, V, beta, ts, psi=_dev(psi[None, :], dtype))
            assert _rel(F[0], np.exp(-beta * c) * ref) < lim, dtype
            assert np.allclose(o, ref.real / ref.real[0], atol=lim)


def test_majorana_calls_refuse_a_pauli_handle():
    import paper_2311_00639_b300 as syk
    from paper_2311_00639_b300 import _lib as L

    x, z, h, _ = si.heisenberg_chain(6, W=1.0)
    with syk.PauliTerms(6, x, z, h, dtype="c128") as t:
        psi = _dev(_state(64, 1), "c128")
        with pytest.raises(L.SykError):
            t.apply_chi(0, psi, 0)
        with pytest.raises(L.SykError):
            t.otoc(1, 0, 1.0, [0.0])
        with syk.Batch(dtype="c128", max_slots=1, max_bytes=16 << 20) as b:
            with pytest.raises(L.SykError):
                b.submit(t, 1, 0, 1.0, [0.0], 0, 0, 0)
        with pytest.raises(L.SykError):
            t.apply_pauli(1 << 6, 0, psi)  # qubit 6 of a 6-qubit chain
    import ctypes as C

    import torch

    q, J, _ = si.sample_sparse_syk(12, 4)
    with syk.Terms(12, q, J, dtype="c128") as ts:  # syk_apply_pauli takes Pauli handles only
        v = _dev(_state(32, 2), "c128")
        o = torch.empty_like(v)
        rc = L.load().syk_apply_pauli(ts._h, 1, 0, C.c_void_p(v.data_ptr()), C.c_void_p(o.data_ptr()), 1,
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == L.SYK_EINVAL


def _diagonal_strings(L, n, seed):
    """n distinct Z-only strings (x = 0) avoiding qubit 0 (z & 1 = 0): one
    class, so one stretch of equal flip mask, longer than a merge group."""
    rng = np.random.default_rng(seed)
    z = rng.choice(np.arange(2, 1 << L, 2), size=n, replace=False).astype(np.uint32)
    return np.zeros(n, np.uint32), z, rng.normal(size=n)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_long_merge_groups_H_and_krylov(dtype):
    """600 diagonal strings on L = 12 (two 2048-amplitude tiles): one stretch
    of equal flip mask and class, which the records split into merge groups
    of 256, 256 and 88 (complex64: summed in the consumer's group loop, over a
    pass split into chunks).  H psi against the oracle's CSR matrix, and the
    Krylov propagator of this diagonal H against its closed form
    e^{-iHt} x = exp(-i t d) x, with d the diagonal."""
    import paper_2311_00639_b300 as syk

    L, n = 12, 600
    x, z, h = _diagonal_strings(L, n, 7)
    H = spin.csr_H(L, x, z, h)
    psi = _state(1 << L, 3)
    with syk.PauliTerms(L, x, z, h, dtype=dtype) as t:
        if dtype == "c64":
            assert 2 * t.info["n_merged"] >= t.n_terms
        got = t.apply_H(_dev(psi, dtype), 0).cpu().numpy()
        assert _rel(got, H @ psi) < TOL_H[dtype]
        d = H.diagonal()
        xv = psi / np.linalg.norm(psi)
        y, st = t.krylov_evolve(_dev(xv, dtype), 0, 0.0, 0.3, **({"tol": 1e-12} if dtype == "c128" else {}))
        ref = np.exp(-1j * 0.3 * d) * xv
        assert _rel(y.cpu().numpy(), ref) < (1e-10 if dtype == "c128" else 5e-5)
        assert st.matvecs > 0 and t.device_error() == 0
