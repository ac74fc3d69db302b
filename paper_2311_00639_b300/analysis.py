"""Post-processing of OTOC curves (main text, finite-size scaling analysis).

* t_star: the time t*(N) at which a normalised OTOC first drops to F0
  (0.75 <= F0 <= 0.85 in the paper), by linear interpolation on the grid.
* fit_glob: Eq. (glob), t*(N) = g0 + (log N / lam) (1 + g1/N) for beta >= 5
  (g2 = 0), or (1 + g2/N^2) at high temperature (g1 = 0).  With a0 = g0,
  a1 = 1/lam, a2 = g/lam the model is linear in (a0, a1, a2).
* inverse_slope: 1/(N dt*/dN) from the difference t*(N + step) - t*(N)
  (the paper uses step 8), at the midpoint N + step/2.
* fit_lamexpan: Eq. (lamexpan), 1/(N dt*/dN) = lam + al1/N (+ al2/N^2), least
  squares; lam is the 1/N -> 0 extrapolation.
Host-side numpy; no GPU work.
"""
from __future__ import annotations

import numpy as np


def t_star(ts, otoc, F0: float) -> float:
    ts = np.asarray(ts, dtype=np.float64)
    o = np.asarray(otoc, dtype=np.float64)
    below = np.nonzero(o <= F0)[0]
    if len(below) == 0:
        return float("nan")
    i = int(below[0])
    if i == 0:
        return float(ts[0])
    t0, t1, f0, f1 = ts[i - 1], ts[i], o[i - 1], o[i]
    return float(t0 + (F0 - f0) * (t1 - t0) / (f1 - f0))


def fit_glob(Ns, tstar, high_temperature: bool = False) -> dict:
    N = np.asarray(Ns, dtype=np.float64)
    y = np.asarray(tstar, dtype=np.float64)
    corr = np.log(N) / (N ** 2 if high_temperature else N)
    A = np.column_stack([np.ones_like(N), np.log(N), corr])
    (a0, a1, a2), *_ = np.linalg.lstsq(A, y, rcond=None)
    lam = 1.0 / a1
    key = "gamma2" if high_temperature else "gamma1"
    return {"lambda_L": float(lam), "gamma0": float(a0), key: float(a2 / a1),
            "residual": float(np.linalg.norm(A @ np.array([a0, a1, a2]) - y))}


def inverse_slope(Ns, tstar, step: int = 8):
    """Pairs (N_mid, 1/(N_mid dt*/dN)) for every N with N + step also present."""
    d = dict(zip([int(n) for n in Ns], np.asarray(tstar, dtype=np.float64)))
    out = []
    for n in sorted(d):
        if n + step in d:
            slope = (d[n + step] - d[n]) / step
            nm = n + step / 2.0
            out.append((nm, 1.0 / (nm * slope)))
    return np.array(out)


def fit_lamexpan(N_mid, inv_slopes, quadratic: bool = False, linear: bool = True) -> dict:
    N = np.asarray(N_mid, dtype=np.float64)
    y = np.asarray(inv_slopes, dtype=np.float64)
    cols = [np.ones_like(N)]
    names = ["lambda_L"]
    if linear:
        cols.append(1.0 / N)
        names.append("alpha1")
    if quadratic:
        cols.append(1.0 / N ** 2)
        names.append("alpha2")
    coef, *_ = np.linalg.lstsq(np.column_stack(cols), y, rcond=None)
    return {k: float(v) for k, v in zip(names, coef)}
