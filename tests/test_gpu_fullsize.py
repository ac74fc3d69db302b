"""GPU parity on the full-size tiled paths: the single-realisation OTOC chain
and the Lanczos epilogues of the tiled H psi kernels against the oracle.

* N = 32 (blocks of 32768 amplitudes, sparse SYK k = 4): syk_otoc on the
  Philox typical states against stored oracle values (expm_multiply on CSR
  blocks, tests/golden/otoc_N32_k4_r0_typical.txt), beta in {0, 5, 10},
  t up to 15, both dtypes.  complex64 runs the tiled TMA-staged kernel.
* N = 44 (blocks of 2^21 amplitudes, 1024 tiles) with commuting terms, where
  the oracle evolves exactly (a product of single-term exponentials,
  oracle.commuting): Krylov propagation element by element, with the basis
  stored (Lanczos epilogue of the matvec) and regenerated (two-pass
  recurrence epilogue), on the default plan and a many-pass plan with
  straggler terms; and syk_otoc against stored oracle values
  (tests/golden/otoc_N44_commuting.txt).  complex128 runs the TMA kernel of
  large blocks, complex64 the tiled complex64 kernel.

Tolerances (relative to the largest |entry| of the reference).  complex128:
1e-10 (Krylov tol 1e-13 per evolve).  complex64 Krylov vectors: 5e-5.
complex64 F(t): every evolve on the path of one F(t) value (the bra is
advanced once per grid point, the ket chain has four evolves) contributes at
most the Krylov tolerance (1e-6 relative), and binary32 rounding of a sum of
T products contributes about sqrt(T) 2^-24 ~ 1e-6 per matvec, growing like
the square root of the matvec count along the chain; the bound used is
(n_t + 4) * 1e-6 + 1e-5, with n_t the number of grid points.
"""
import os

import numpy as np
import pytest

import syk_inputs as si

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(__file__)
GOLD32 = os.path.join(HERE, "golden", "otoc_N32_k4_r0_typical.txt")
GOLD44 = os.path.join(HERE, "golden", "otoc_N44_commuting.txt")
STATE_SEED = 7
N44_SEED = 3


def c64_F_tolerance(n_t: int) -> float:
    return (n_t + 4) * 1e-6 + 1e-5


@pytest.fixture(scope="module")
def syk():
    import paper_2311_00639_b300 as p

    return p


def torch():
    import torch as t

    return t


def load_typical(path):
    rows = np.loadtxt(path, comments="#")
    out = {}
    for beta in sorted(set(rows[:, 0])):
        r = rows[rows[:, 0] == beta]
        ts = r[r[:, 1] == 0][:, 2]
        F = np.stack([r[r[:, 1] == s][:, 3] + 1j * r[r[:, 1] == s][:, 4] for s in (0, 1)])
        out[beta] = (ts, F)
    return out


def curve_err(got, ref):
    return np.max(np.abs(got - ref)) / np.max(np.abs(ref))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_otoc_N32_typical_vs_golden(syk, dtype):
    """syk_otoc (typical states from its own Philox generator) at N = 32 against
    the oracle's expm_multiply values, per state and t, for beta in {0, 5, 10}."""
    N = 32
    q, J, _ = si.sample_sparse_syk(N, 4, r=0)
    gold = load_typical(GOLD32)
    kp = {"m": 30, "tol": 1e-13} if dtype == "c128" else {"m": 30}
    with syk.Terms(N, q, J, dtype=dtype) as h:
        for beta, (ts, Fg) in gold.items():
            F, o, st = h.otoc(N - 1, N - 2, beta, ts, n_states=2, seed=STATE_SEED, **kp)
            lim = 1e-10 if dtype == "c128" else c64_F_tolerance(len(ts))
            for s in (0, 1):
                err = curve_err(F[s], Fg[s])
                print(f"N=32 {dtype} beta={beta} state={s}: max |dF| / max |F| = {err:.3e}")
                assert err < lim, (beta, s, err)
            ref_o = Fg.mean(axis=0).real / Fg.mean(axis=0).real[0]
            assert np.max(np.abs(o - ref_o)) < (1e-9 if dtype == "c128" else 10 * lim)
            assert st.matvecs > 0
        assert h.device_error() == 0


@pytest.fixture(scope="module")
def commuting44():
    """N = 44 commuting-term Hamiltonian, a Philox state of each block, and
    the oracle's exact e^{-zH} x for the z values of the Krylov test."""
    from oracle import commuting as cm

    N = 44
    q, J, pairs = si.sample_commuting_syk(N, N44_SEED)
    v = si.philox_state(N, STATE_SEED, 3)
    v = v / np.linalg.norm(v)
    D = len(v) // 2
    xs = (v[:D].copy(), v[D:].copy())
    refs = {}
    for blk, (tau, t) in ((0, (0.0, 2.0)), (1, (0.5, -3.0)), (0, (1.25, 6.0))):
        refs[(blk, tau, t)] = cm.evolve(N, "jw", q, J, blk, complex(tau, t), xs[blk], pairs)
    return N, q, J, xs, refs


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("two_pass", [False, True])
@pytest.mark.parametrize("plan", ["default", "many-pass"])
def test_krylov_N44_commuting_vs_exact(syk, commuting44, dtype, two_pass, plan):
    t = torch()
    N, q, J, xs, refs = commuting44
    tdt = t.complex64 if dtype == "c64" else t.complex128
    kp = {"tol": 1e-13} if dtype == "c128" else {}
    lim = 1e-10 if dtype == "c128" else 5e-5
    with syk.Terms(N, q, J, dtype=dtype) as h:
        if plan == "many-pass":
            assert h.replan(1 << 16, 3.0) >= 2
        for (blk, tau, tt), ref in refs.items():
            x = t.from_numpy(xs[blk]).to("cuda", tdt)
            y, st = h.krylov_evolve(x, blk, tau, tt, two_pass=two_pass, **kp)
            err = np.max(np.abs(y.cpu().numpy() - ref)) / np.max(np.abs(ref))
            print(f"N=44 {dtype} two_pass={two_pass} {plan} z=({tau},{tt}) block {blk}: {err:.3e} ({st})")
            assert err < lim, (blk, tau, tt, err)
            if tau == 0.0:  # e^{-iHt} keeps the norm
                nx = float(np.linalg.norm(xs[blk]))
                assert abs(t.linalg.vector_norm(y).item() / nx - 1.0) < (1e-12 if dtype == "c128" else 1e-5)
        assert h.device_error() == 0


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_otoc_N44_commuting_vs_golden(syk, dtype):
    """syk_otoc on the tiled large-block kernels against the exact commuting
    oracle (stored), per state and t, beta in {0, 5}."""
    N = 44
    q, J, _ = si.sample_commuting_syk(N, N44_SEED)
    gold = load_typical(GOLD44)
    kp = {"tol": 1e-13} if dtype == "c128" else {}
    with syk.Terms(N, q, J, dtype=dtype) as h:
        for beta, (ts, Fg) in gold.items():
            F, o, _ = h.otoc(N - 1, N - 2, beta, ts, n_states=2, seed=STATE_SEED, **kp)
            lim = 1e-10 if dtype == "c128" else c64_F_tolerance(len(ts))
            for s in (0, 1):
                err = curve_err(F[s], Fg[s])
                print(f"N=44 {dtype} beta={beta} state={s}: {err:.3e}")
                assert err < lim, (beta, s, err)
        assert h.device_error() == 0
