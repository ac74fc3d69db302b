"""Write the stored expected values under tests/golden/ (calls only oracle/).

otoc_N16_k4_r0.txt — the "plain method" configuration: N = 16 Majoranas,
sparse SYK with k = 4 (realisation r = 0 of syk_inputs.sample_sparse_syk),
the regularised OTOC of Eq. (2) as an exact trace (raw F(t) = Tr[...]/dim and
OTOC = F(t)/F(0)), averaged over all N(N-1) = 240 ordered pairs (a, b),
a != b, for beta in {0, 5} and t = 0, 0.5, ..., 10.  Jordan-Wigner
representation (the trace does not depend on it).

otoc_N32_k4_r0_typical.txt — the N = 32 configuration (16 qubits, parity
blocks of 32768 amplitudes, k = 4, realisation r = 0): the single-state F(t)
of the parity-block formula (supplement, OTOC paragraph) for the Philox
typical states (seed 7, state ids 0 and 1, syk_inputs.philox_state,
normalised over both blocks), a = N-1, b = N-2, beta in {0, 5, 10} and
t in {0, 0.1, 1, 2.5, 5, 10, 15} (a subset of the 0..15 grid, step 0.1),
by oracle.otoc.F_state_sparse (CSR blocks, expm_multiply).

otoc_N44_commuting.txt — N = 44 (blocks of 2^21 amplitudes) with commuting
terms (syk_inputs.sample_commuting_syk(44, seed=3), 44 terms): the same
single-state F(t) by the exact commuting tier oracle.commuting.F_state, Philox
states (seed 7, ids 0 and 1), a = N-1, b = N-2, beta in {0, 5},
t in {0, 0.5, 2, 6}.

Usage: python tests/golden/make_golden.py [n16|n32|n44 ...]   (default: all)
"""
import multiprocessing as mp
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


N32_TS = [0.0, 0.1, 1.0, 2.5, 5.0, 10.0, 15.0]
N32_BETAS = [0.0, 5.0, 10.0]
N44_TS = [0.0, 0.5, 2.0, 6.0]
N44_BETAS = [0.0, 5.0]
STATE_SEED = 7
N44_SEED = 3


def _n32_item(args):
    beta, sid = args
    N = 32
    q, J, _ = si.sample_sparse_syk(N, 4, r=0)
    v = si.philox_state(N, STATE_SEED, sid)
    v = v / np.linalg.norm(v)
    D = len(v) // 2
    return beta, sid, ot.F_state_sparse(N, "jw", q, J, N - 1, N - 2, beta, N32_TS, v[:D], v[D:])


def _n44_item(args):
    from oracle import commuting as cm

    beta, sid = args
    N = 44
    q, J, pairs = si.sample_commuting_syk(N, N44_SEED)
    v = si.philox_state(N, STATE_SEED, sid)
    v = v / np.linalg.norm(v)
    D = len(v) // 2
    return beta, sid, cm.F_state(N, "jw", q, J, N - 1, N - 2, beta, N44_TS, v[:D], v[D:], pairs)


def _write_typical(name, header, ts, results):
    lines = header + ["# columns: beta state t Re F Im F"]
    for beta, sid, F in sorted(results, key=lambda r: (r[0], r[1])):
        for t, f in zip(ts, F):
            lines.append(f"{beta:.1f} {sid} {t:.2f} {f.real:.16e} {f.imag:.16e}")
    with open(os.path.join(HERE, name), "w") as fh:
        fh.write("\n".join(lines) + "\n")


def main_n32(pool):
    res = pool.map(_n32_item, [(b, s) for b in N32_BETAS for s in (0, 1)])
    _write_typical("otoc_N32_k4_r0_typical.txt", [
        "# Single-state OTOC F(t), parity-block formula (supplement, OTOC paragraph), N=32, k=4, realisation r=0",
        "# couplings: syk_inputs.sample_sparse_syk(32, 4, r=0); Jordan-Wigner; a = 31, b = 30",
        f"# states: syk_inputs.philox_state(32, {STATE_SEED}, id) / norm, ids 0 and 1; "
        "oracle.otoc.F_state_sparse (expm_multiply)",
        "# written by tests/golden/make_golden.py"], N32_TS, res)


def main_n44(pool):
    res = pool.map(_n44_item, [(b, s) for b in N44_BETAS for s in (0, 1)])
    _write_typical("otoc_N44_commuting.txt", [
        "# Single-state OTOC F(t), parity-block formula (supplement, OTOC paragraph), N=44, commuting terms",
        f"# couplings: syk_inputs.sample_commuting_syk(44, seed={N44_SEED}) (44 terms); Jordan-Wigner; a = 43, b = 42",
        f"# states: syk_inputs.philox_state(44, {STATE_SEED}, id) / norm, ids 0 and 1; "
        "oracle.commuting.F_state (exact product of single-term exponentials)",
        "# written by tests/golden/make_golden.py"], N44_TS, res)


if __name__ == "__main__":
    which = sys.argv[1:] or ["n16", "n32", "n44"]
    if "n16" in which:
        main()
    if "n32" in which or "n44" in which:
        with mp.get_context("spawn").Pool(min(6, os.cpu_count() or 1)) as pool:
            if "n32" in which:
                main_n32(pool)
            if "n44" in which:
                main_n44(pool)
