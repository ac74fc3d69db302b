"""Post-processing (main text, finite-size analysis) on synthetic curves with
known parameters."""
import numpy as np

from paper_2311_00639_b300 import analysis as an


def test_t_star_on_exponential_curve():
    lam, c, F0 = 0.7, 0.3, 0.8
    ts = np.linspace(0, 10, 20001)
    for N in (20, 40, 60):
        otoc = 1.0 - c * np.exp(lam * ts) / N
        exact = np.log((1.0 - F0) * N / c) / lam
        assert abs(an.t_star(ts, otoc, F0) - exact) < 1e-6
    assert np.isnan(an.t_star(ts, np.ones_like(ts), 0.8))
    assert an.t_star([0, 1, 2], [1.0, 0.5, 0.2], 0.75) == 0.5


def test_fit_glob_recovers_parameters():
    Ns = np.array([14, 22, 30, 38, 46, 54])
    lam, g0, g1, g2 = 0.55, 0.8, -3.0, 12.0
    t = g0 + np.log(Ns) / lam * (1 + g1 / Ns)
    r = an.fit_glob(Ns, t)
    assert abs(r["lambda_L"] - lam) < 1e-10 and abs(r["gamma1"] - g1) < 1e-8 and abs(r["gamma0"] - g0) < 1e-10
    t2 = g0 + np.log(Ns) / lam * (1 + g2 / Ns ** 2)
    r2 = an.fit_glob(Ns, t2, high_temperature=True)
    assert abs(r2["lambda_L"] - lam) < 1e-10 and abs(r2["gamma2"] - g2) < 1e-7


def test_inverse_slope_and_lamexpan():
    # t*(N) = log(N)/lam exactly: 1/(N dt*/dN) = lam in the continuum; the
    # finite difference over 8 gives lam + O(1/N^2)
    lam = 0.6
    Ns = np.arange(14, 63, 8)
    t = np.log(Ns) / lam
    pts = an.inverse_slope(Ns, t, step=8)
    assert len(pts) == len(Ns) - 1
    Nm = pts[:, 0]
    exact = 1.0 / (Nm * (np.log(Nm + 4) - np.log(Nm - 4)) / (8 * lam))
    assert np.allclose(pts[:, 1], exact, rtol=1e-12)
    fit = an.fit_lamexpan(pts[:, 0], pts[:, 1], quadratic=True)
    assert abs(fit["lambda_L"] - lam) < 1e-3
    # a pure lam + al1/N law is recovered exactly
    y = 0.5 + 2.0 / Nm
    f2 = an.fit_lamexpan(Nm, y)
    assert abs(f2["lambda_L"] - 0.5) < 1e-12 and abs(f2["alpha1"] - 2.0) < 1e-10
