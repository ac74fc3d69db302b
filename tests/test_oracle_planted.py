"""Planted mistakes: each plausible error in the oracle must make at least one
of its pins fail.

A mistake is planted on the CPU only, in the oracle: either a module constant
is changed, or one line of an oracle function's source is rewritten and the
function is rebuilt from that text in its module's namespace and swapped in
for the duration of one test (pytest's monkeypatch restores it).  The pins
are the unchanged test functions of test_oracle.py, test_oracle_spin.py and
test_oracle_nonherm.py, called directly; a mistake counts as caught when one
of them raises AssertionError.  Without a mistake the same pins pass (they are
part of the CPU suite).
"""
import inspect
import textwrap

import numpy as np
import pytest

from oracle import commuting as cm
from oracle import majorana as mj
from oracle import nonherm as nh
from oracle import otoc
from oracle import spin

from . import test_oracle as T0
from . import test_oracle_nonherm as TN
from . import test_oracle_spin as TS


def mutant(module, fname, old, new):
    """The function `fname` of `module` rebuilt from its source with `old`
    (which must occur) replaced by `new`."""
    src = textwrap.dedent(inspect.getsource(getattr(module, fname)))
    assert old in src, (fname, old)
    ns = dict(vars(module))
    exec(compile(src.replace(old, new, 1), f"<planted {module.__name__}.{fname}>", "exec"), ns)
    return ns[fname]


def caught(pins) -> list:
    """Names of the pins that fail (AssertionError) under the planted mistake."""
    failed = []
    for fn, kw in pins:
        try:
            fn(**kw)
        except AssertionError:
            failed.append(fn.__name__)
    return failed


OTOC_PINS = [(T0.test_otoc_t0_beta0_is_minus_quarter, {"rep": "jw"}),
             (T0.test_otoc_closed_form_terms_containing_a_and_b, {"rep": "jw"}),
             (T0.test_otoc_closed_form_terms_avoiding_a_and_b, {"rep": "jw"}),
             (T0.test_block_form_equals_full_space, {"rep": "jw"})]

SOURCE_MUTATIONS = [
    # (id, module, function, old text, new text, pins)
    ("otoc exponent sign", otoc, "F_state", "k = np.exp(-(1j * t + beta / 4.0) * lam) * (Xb @ k)",
     "k = np.exp(-(-1j * t + beta / 4.0) * lam) * (Xb @ k)", OTOC_PINS),
    ("otoc beta split", otoc, "F_state", "k = np.exp(-beta / 8.0 * lam) * p", "k = np.exp(-beta / 4.0 * lam) * p",
     OTOC_PINS),
    ("otoc wrong Majorana operand", otoc, "F_state", "k = Xa @ k", "k = Xb @ k", OTOC_PINS),
    ("JW sigma_y replaced by sigma_z", mj, "jw_ops", 'ops[s] = "X" if n % 2 == 0 else "Y"',
     'ops[s] = "X" if n % 2 == 0 else "Z"', [(T0.test_clifford_algebra, {"rep": "jw", "N": 6}),
                                             (T0.test_basis_maps_match_dense, {"rep": "jw", "N": 6})]),
    ("JW parity blocks swapped", mj, "block_indices", "return m | (par << L), m | ((1 - par) << L)",
     "return m | ((1 - par) << L), m | (par << L)", [(T0.test_csr_and_rows_match_dense, {"rep": "jw", "N": 8})]),
    ("spin qubit order reversed", spin, "pauli_dense", "for op in reversed(letters(L, x, z)):",
     "for op in letters(L, x, z):", [(TS.test_qubit_order_is_bit_order, {}),
                                      (TS.test_maps_match_dense_products, {"L": 2})]),
    ("spin sigma_y phase in the basis map", spin, "apply_map", "ph = ph * (1j * sgn)", "ph = ph * (-1j * sgn)",
     [(TS.test_maps_match_dense_products, {"L": 2})]),
    ("spin Hamiltonian drops its last string", spin, "dense_H",
     "for x, z, c in zip(np.asarray(xs), np.asarray(zs), np.asarray(h)):",
     "for x, z, c in zip(np.asarray(xs)[:-1], np.asarray(zs), np.asarray(h)):",
     [(TS.test_xx_chain_free_fermion_spectrum, {}), (TS.test_two_site_heisenberg_singlet_triplet, {})]),
    ("non-Hermitian chain without the adjoint", nh, "_chain", "Ub = sla.expm(1j * t * H.conj().T)",
     "Ub = sla.expm(1j * t * H)", [(TN.test_otoc_closed_form_all_terms_contain_a_and_b, {})]),
    ("commuting factor sinh sign", cm, "evolve", "np.cosh(w) * out - 4.0 * np.sinh(w)",
     "np.cosh(w) * out + 4.0 * np.sinh(w)", [(T0.test_commuting_evolve_matches_dense_eigh, {"rep": "jw"})]),
    ("commuting factor with J/2", cm, "evolve", "w = z * c / 4.0", "w = z * c / 2.0",
     [(T0.test_commuting_evolve_matches_dense_eigh, {"rep": "jw"})]),
    ("commuting pair reordering sign dropped", cm, "_split_pairs", "return (a, b), (c, d), (-1) ** inversions",
     "return (a, b), (c, d), 1", [(T0.test_commuting_evolve_matches_dense_eigh, {"rep": "jw"})]),
    ("commuting OTOC ket without its last Majorana", cm, "F_state", "k = ca @ k", "k = k",
     [(T0.test_commuting_otoc_matches_dense_block_formula, {})]),
    ("non-Hermitian couplings conjugated", nh, "couplings",
     "np.asarray(J_re, dtype=np.float64) + 1j * np.asarray(J_im, dtype=np.float64)",
     "np.asarray(J_re, dtype=np.float64) - 1j * np.asarray(J_im, dtype=np.float64)",
     [(TN.test_single_complex_term_closed_form, {})]),
]


@pytest.mark.parametrize("case", SOURCE_MUTATIONS, ids=[c[0] for c in SOURCE_MUTATIONS])
def test_source_mutation_is_caught(monkeypatch, case):
    _, module, fname, old, new, pins = case
    monkeypatch.setattr(module, fname, mutant(module, fname, old, new))
    assert caught(pins), f"no pin caught the planted mistake in {module.__name__}.{fname}"


def test_sigma_y_sign_is_caught(monkeypatch):
    """sigma_y = [[0, i], [-i, 0]] (the sign the supplement prints) in the
    Majorana oracle, and separately in the spin oracle."""
    monkeypatch.setitem(mj.PAULI, "Y", -mj.SY)
    assert caught([(T0.test_paper_special_gammas, {"N": 6}), (T0.test_algorithm1_matches_kronecker, {"L": 2})])
    monkeypatch.undo()
    monkeypatch.setitem(spin.SIGMA, "Y", -spin.SIGMA["Y"])
    assert caught([(TS.test_pauli_multiplication_table, {})])


def test_pins_pass_without_a_mistake():
    """The same pins, unchanged oracle: nothing fails."""
    pins = {(fn, tuple(sorted(kw.items()))) for *_, ps in SOURCE_MUTATIONS for fn, kw in ps}
    assert caught([(fn, dict(kw)) for fn, kw in pins]) == []
    assert np.isfinite(otoc.F_state(np.eye(2), {0: np.eye(2), 1: np.eye(2)}, 0, 1, 0.0, [0.0], [1.0, 0.0])[0])
