"""The "plain method" configuration on the GPU: exact-trace OTOC of Eq. (2)
at N = 16, k = 4, beta in {0, 5}, averaged over all 240 ordered Majorana
pairs, by the batched engine summed over all 256 basis states, against the
stored oracle values in tests/golden/otoc_N16_k4_r0.txt (and three single
pairs against the live oracle)."""
import os

import numpy as np
import pytest

import syk_inputs as si
from oracle import dynamics as dyn
from oracle import hamiltonian as ham
from oracle import majorana as mj
from oracle import otoc as ot

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "otoc_N16_k4_r0.txt")


def load_golden():
    rows = np.loadtxt(GOLDEN, comments="#")
    out = {}
    for beta in (0.0, 5.0):
        r = rows[rows[:, 0] == beta]
        out[beta] = (r[:, 1], r[:, 2] + 1j * r[:, 3], r[:, 4])
    return out


def test_all_pairs_exact_trace_matches_golden():
    import paper_2311_00639_b300 as syk

    N = 16
    q, J, _ = si.sample_sparse_syk(N, 4, r=0)
    gold = load_golden()
    pairs = [(a, b) for a in range(N) for b in range(N) if a != b]
    with syk.Terms(N, q, J, dtype="c128") as h:
        for beta in (0.0, 5.0):
            ts, Fg, Og = gold[beta]
            res = syk.exact_trace_otoc(h, pairs, beta, ts, tol=1e-13)
            Fm = np.mean([res[p][0] for p in pairs], axis=0)
            Om = np.mean([res[p][1] for p in pairs], axis=0)
            assert np.max(np.abs(Fm - Fg)) < 1e-11
            assert np.max(np.abs(Om - Og)) < 1e-9
            if beta == 5.0:
                H = ham.dense_H(N, q, J, "jw")
                X = mj.chis(N, "jw")
                eig = dyn.eig(H)
                for a, b in [(15, 14), (0, 7), (9, 2)]:
                    ref = ot.F_trace(H, X, a, b, beta, ts, eig)
                    assert np.max(np.abs(res[(a, b)][0] - ref)) < 1e-11
