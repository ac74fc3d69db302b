"""Finite-size analysis (main text: t* at F0, Eq. (glob)) on curves the GPU
computed: exact-trace OTOC curves of the batched engine at N = 10..16 give
the same t*(N), by analysis.t_star, as the oracle's exact-trace curves
(dense eigendecomposition), and the same Eq. (glob) fit parameters."""
import numpy as np
import pytest

import syk_inputs as si
from oracle import dynamics as dyn
from oracle import hamiltonian as ham
from oracle import majorana as mj
from oracle import otoc as ot
from paper_2311_00639_b300 import analysis as an

pytestmark = pytest.mark.gpu


def test_t_star_and_glob_fit_from_gpu_curves_match_oracle():
    import paper_2311_00639_b300 as syk

    ts = np.linspace(0.0, 6.0, 49)
    beta, F0 = 0.0, 0.8
    Ns = [10, 12, 14, 16]
    t_gpu, t_ref = [], []
    for N in Ns:
        q, J, _ = si.sample_sparse_syk(N, 4, r=20 + N)
        with syk.Terms(N, q, J, dtype="c128") as h:
            res = syk.exact_trace_otoc(h, [(N - 1, N - 2)], beta, ts, tol=1e-13)
        o_gpu = res[(N - 1, N - 2)][1]
        H = ham.dense_H(N, q, J, "jw")
        F = ot.F_trace(H, mj.chis(N, "jw"), N - 1, N - 2, beta, ts, dyn.eig(H))
        o_ref = ot.normalise(F)
        assert np.max(np.abs(o_gpu - o_ref)) < 1e-10
        t_gpu.append(an.t_star(ts, o_gpu, F0))
        t_ref.append(an.t_star(ts, o_ref, F0))
    assert np.all(np.isfinite(t_ref))
    assert np.max(np.abs(np.array(t_gpu) - np.array(t_ref))) < 1e-8
    fg, fr = an.fit_glob(Ns, t_gpu, high_temperature=True), an.fit_glob(Ns, t_ref, high_temperature=True)
    for k in ("lambda_L", "gamma0", "gamma2"):
        assert abs(fg[k] - fr[k]) <= 1e-6 * max(1.0, abs(fr[k])), k
