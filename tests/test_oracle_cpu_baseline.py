"""The C++/OpenMP CPU baseline (oracle/cpu_baseline.cpp) against the Python
oracle: H psi against the dense blocks and the CSR form, sampled rows against
the full product, Lanczos propagation against the eigendecomposition.  The
baseline is what the benchmark times on the host cores, so these tests make
its rate a rate of the right computation."""
import numpy as np
import pytest

import syk_inputs as si
from oracle import cpu_baseline as cb
from oracle import dynamics as dyn
from oracle import hamiltonian as ham


def rand_vec(D, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=D) + 1j * rng.normal(size=D)


@pytest.mark.parametrize("N", [8, 12, 16])
def test_cpu_hpsi_matches_dense_blocks(N):
    q, J, _ = si.sample_sparse_syk(N, 4, r=N)
    HU, HD = ham.blocks(ham.dense_H(N, q, J, "jw"), N, "jw")
    psi = rand_vec(HU.shape[0], 1)
    for blk, Hb in ((0, HU), (1, HD)):
        ref = Hb @ psi
        assert np.max(np.abs(cb.hpsi(N, q, J, blk, psi) - ref)) < 1e-13 * np.max(np.abs(ref))


def test_cpu_hpsi_matches_csr_N24_and_rows():
    N = 24
    q, J, _ = si.sample_sparse_syk(N, 4, r=3)
    psi = rand_vec(1 << 11, 2)
    for blk in (0, 1):
        ref = ham.csr_block(N, q, J, "jw", blk) @ psi
        full = cb.hpsi(N, q, J, blk, psi)
        assert np.max(np.abs(full - ref)) < 1e-13 * np.max(np.abs(ref))
        log2R = 6
        for row0 in (0, 1 << 6, 25 << 6):
            starts = cb.row_sample_starts(N, q, J, blk, row0, log2R)
            blocks = [psi[int(s): int(s) + (1 << log2R)] for s in starts]
            got = cb.hpsi_rows(N, q, J, blk, row0, log2R, blocks)
            assert np.max(np.abs(got - full[row0: row0 + (1 << log2R)])) < 1e-13 * np.max(np.abs(ref))


def test_cpu_krylov_matches_eigh_N16():
    N = 16
    q, J, _ = si.sample_sparse_syk(N, 4, r=4)
    HU, HD = ham.blocks(ham.dense_H(N, q, J, "jw"), N, "jw")
    x = rand_vec(HU.shape[0], 9)
    for blk, Hb in ((0, HU), (1, HD)):
        for z in (0.7j, 1.25, 2.5 + 3.0j, -7.5j + 0.625):
            y, mv = cb.krylov_evolve(N, q, J, blk, z, x, m=30, tol=1e-13)
            ref = dyn.evolve(Hb, z, x)
            assert mv > 0
            assert np.max(np.abs(y - ref)) < 1e-10 * np.max(np.abs(ref)), (blk, z)


def test_cpu_baseline_uses_threads():
    assert cb.threads() >= 1
