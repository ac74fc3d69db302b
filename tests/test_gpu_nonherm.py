"""GPU parity of the non-Hermitian SYK path (complex couplings) against the
CPU oracle, through the C-ABI: H psi and H^dag psi, Arnoldi propagation
(syk_krylov_evolve on a non-Hermitian handle) against scipy's expm /
expm_multiply, and the infinite-temperature OTOC with
W(t) = e^{iH^dag t} W e^{-iHt} (syk_otoc_nonhermitian) against the oracle's
chain, its Hermitian limit against syk_otoc at beta = 0, and the refusals.
Tolerances: complex128 H psi 1e-12 of the largest entry, Arnoldi results and
OTOC 1e-10 relative; complex64 2e-5 / 5e-5 / 1e-4."""
import numpy as np
import pytest

import syk_inputs as si
from oracle import hamiltonian as ham
from oracle import majorana as mj
from oracle import nonherm as nh

pytestmark = pytest.mark.gpu


def _dev(a, dtype):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.complex128 if dtype == "c128" else
                                                         torch.complex64)


def _instance(N, k=4, r=0, scale=1.0):
    q, J, _ = si.sample_sparse_syk(N, k, r=r)
    M = np.random.default_rng(500 + r).normal(size=len(J)) * np.sqrt(np.mean(J ** 2)) * scale
    return q, J, M


def _state(D, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=D) + 1j * rng.normal(size=D)
    return v / np.linalg.norm(v)


def _rel(got, ref):
    return np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("N,rep", [(10, "jw"), (10, "paper"), (14, "jw"), (26, "jw")])
def test_apply_H_and_adjoint(dtype, N, rep):
    import paper_2311_00639_b300 as syk

    q, J, M = _instance(N, r=N)
    D = 1 << (N // 2 - 1)
    lim = 1e-12 if dtype == "c128" else 2e-5
    with syk.Terms.complex(N, q, J, M, dtype=dtype, rep=rep) as h:
        assert not h.hermitian
        with h.adjoint() as hd:
            for blk in (0, 1):
                psi = _state(D, blk + 1)
                if N <= 14:
                    Hb = ham.blocks(nh.dense_H(N, q, J, M, rep), N, rep)[blk]
                    ref, refd = Hb @ psi, Hb.conj().T @ psi
                else:
                    Hc = nh.csr_block(N, q, J, M, rep, blk)
                    ref, refd = Hc @ psi, Hc.conj().T @ psi
                got = h.apply_H(_dev(psi, dtype), blk).cpu().numpy()
                assert _rel(got, ref) < lim
                gotd = hd.apply_H(_dev(psi, dtype), blk).cpu().numpy()
                assert _rel(gotd, refd) < lim


@pytest.mark.parametrize("N", [6, 12, 16])
def test_arnoldi_matches_expm_complex128(N):
    import paper_2311_00639_b300 as syk

    q, J, M = _instance(N, r=20 + N)
    rep = "jw"
    Hs = ham.blocks(nh.dense_H(N, q, J, M, rep), N, rep)
    with syk.Terms.complex(N, q, J, M, dtype="c128") as h:
        for blk in (0, 1):
            x = _state(Hs[blk].shape[0], 10 + blk)
            for z in (2.0j, 0.5 + 1.5j, -1.5j, 1.0, 6.0j):
                y, st = h.krylov_evolve(_dev(x, "c128"), blk, z.real, z.imag)
                ref = nh.evolve(Hs[blk], z, x)
                assert _rel(y.cpu().numpy(), ref) < 1e-10, (N, blk, z)
                assert st.matvecs > 0
            # a Krylov dimension below D forces several substeps (D <= m: one exact step)
            y, st = h.krylov_evolve(_dev(x, "c128"), blk, 0.0, 6.0, m=12)
            assert (st.substeps > 1) == (x.shape[0] > 12)
            assert _rel(y.cpu().numpy(), nh.evolve(Hs[blk], 6.0j, x)) < 1e-10


def test_arnoldi_tiled_blocks_and_complex64():
    """N = 24 (2048 amplitudes: the tiled matvec kernels) against
    expm_multiply in complex128 and complex64; in-place evolution."""
    import paper_2311_00639_b300 as syk

    N = 24
    q, J, M = _instance(N, r=7)
    Hc = nh.csr_block(N, q, J, M, "jw", 0)
    x = _state(1 << (N // 2 - 1), 3)
    ref = nh.evolve_sparse(Hc, 0.25 + 2.0j, x)
    for dtype, lim in (("c128", 1e-10), ("c64", 5e-5)):
        with syk.Terms.complex(N, q, J, M, dtype=dtype) as h:
            d = _dev(x, dtype)
            h.krylov_evolve(d, 0, 0.25, 2.0, y=d)
            assert _rel(d.cpu().numpy(), ref) < lim, dtype
            assert h.device_error() == 0


def test_otoc_nonhermitian_same_state_and_trace():
    import paper_2311_00639_b300 as syk

    N = 10
    q, J, M = _instance(N, r=30)
    H = nh.dense_H(N, q, J, M, "jw")
    X = mj.chis(N, "jw")
    ts = [0.0, 0.5, 1.5, 3.0]
    pU, pD = si.random_state(N, seed=31)
    pU2, pD2 = si.random_state(N, seed=32)
    psi = np.stack([np.stack([pU, pD]), np.stack([pU2, pD2])])
    with syk.Terms.complex(N, q, J, M, dtype="c128") as h:
        F, o, st = h.otoc_nonhermitian(N - 1, N - 2, ts, psi=_dev(psi, "c128"))
        for s, (u, d) in enumerate(((pU, pD), (pU2, pD2))):
            ref = nh.F_state(H, X, N - 1, N - 2, ts, mj.to_full(u, d, N, "jw"))
            assert _rel(F[s], ref) < 1e-10
        mean = F.mean(axis=0)
        assert np.allclose(o, mean.real / mean.real[0], atol=1e-12)
    N = 8
    q, J, M = _instance(N, r=33)
    H = nh.dense_H(N, q, J, M, "jw")
    with syk.Terms.complex(N, q, J, M, dtype="c128") as h:
        F, _, _ = h.otoc_nonhermitian(N - 1, N - 2, ts, mode="exact")
        ref = nh.F_trace(H, mj.chis(N, "jw"), N - 1, N - 2, ts)
        assert _rel(F[0], ref) < 1e-10


def test_otoc_nonhermitian_hermitian_limit_and_complex64():
    import paper_2311_00639_b300 as syk

    N = 12
    q, J, M = _instance(N, r=40)
    ts = [0.0, 1.0, 2.5]
    with syk.Terms(N, q, J, dtype="c128") as h:
        F0, _, _ = h.otoc(N - 1, N - 2, 0.0, ts, n_states=2, seed=9)
        F1, _, _ = h.otoc_nonhermitian(N - 1, N - 2, ts, n_states=2, seed=9)
        assert _rel(F1, F0) < 1e-10
    H = nh.dense_H(N, q, J, M, "jw")
    pU, pD = si.random_state(N, seed=41)
    ref = nh.F_state(H, mj.chis(N, "jw"), N - 1, N - 2, ts, mj.to_full(pU, pD, N, "jw"))
    with syk.Terms.complex(N, q, J, M, dtype="c64") as h:
        F, _, _ = h.otoc_nonhermitian(N - 1, N - 2, ts, psi=_dev(np.stack([np.stack([pU, pD])]), "c64"))
        assert _rel(F[0], ref) < 1e-4


def test_refusals():
    import paper_2311_00639_b300 as syk
    from paper_2311_00639_b300 import _lib as L

    N = 10
    q, J, M = _instance(N, r=50)
    with syk.Terms.complex(N, q, J, M, dtype="c128") as h:
        x = _dev(_state(16, 1), "c128")
        with pytest.raises(L.SykError):
            h.otoc(N - 1, N - 2, 1.0, [0.0])
        with pytest.raises(L.SykError):
            h.krylov_evolve(x, 0, 0.0, 1.0, two_pass=True)
        with syk.Batch(dtype="c128", max_slots=1, max_bytes=16 << 20) as b:
            with pytest.raises(L.SykError):
                b.submit(h, N - 1, N - 2, 1.0, [0.0], 0, 0, 0)
    with syk.Terms.complex(N, q, J, np.zeros_like(J), dtype="c128") as h:
        assert h.hermitian  # no imaginary couplings: Lanczos, syk_otoc accepted
        h.otoc(N - 1, N - 2, 1.0, [0.0])
