"""Write the stored expected values under tests/golden/ (calls only oracle/).

otoc_N16_k4_r0.txt — the "plain method" configuration: N = 16 Majoranas,
sparse SYK with k = 4 (realisation r = 0 of syk_inputs.sample_sparse_syk),
the regularised OTOC of Eq. (2) as an exact trace (raw F(t) = Tr[...]/dim and
OTOC = F(t)/F(0)), averaged over all N(N-1) = 240 ordered pairs (a, b),
a != b, for beta in {0, 5} and t = 0, 0.5, ..., 10.  Jordan-Wigner
representation (the trace does not depend on it).

Usage: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import syk_inputs as si  # noqa: E402
from oracle import dynamics as dyn  # noqa: E402
from oracle import hamiltonian as ham  # noqa: E402
from oracle import majorana as mj  # noqa: E402
from oracle import otoc as ot  # noqa: E402


def main():
    N, k, r = 16, 4, 0
    q, J, _ = si.sample_sparse_syk(N, k, r=r)
    H = ham.dense_H(N, q, J, "jw")
    X = mj.chis(N, "jw")
    eig = dyn.eig(H)
    ts = np.round(np.arange(0.0, 10.0 + 1e-9, 0.5), 10)
    pairs = [(a, b) for a in range(N) for b in range(N) if a != b]
    lines = [
        "# Regularised OTOC, Eq. (2) (main text), exact trace, N=16, k=4, realisation r=0",
        "# couplings: syk_inputs.sample_sparse_syk(16, 4, r=0); Jordan-Wigner representation",
        f"# averaged over all {len(pairs)} ordered pairs (a, b), a != b; written by tests/golden/make_golden.py",
        "# columns: beta t Re<F>/dim Im<F>/dim <OTOC>   (<.> = mean over pairs; OTOC = F(t)/F(0) per pair)",
    ]
    for beta in (0.0, 5.0):
        Fs = np.array([ot.F_trace(H, X, a, b, beta, ts, eig) for a, b in pairs])
        Fm = Fs.mean(axis=0)
        Om = (Fs.real / Fs.real[:, :1]).mean(axis=0)
        for t, f, o in zip(ts, Fm, Om):
            lines.append(f"{beta:.1f} {t:.2f} {f.real:.16e} {f.imag:.16e} {o:.16e}")
    with open(os.path.join(HERE, "otoc_N16_k4_r0.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
