"""Failure detection on the GPU without a fault: a bounded device wait on an
mbarrier that nothing completes expires, the call reports SYK_ETIMEOUT, and
the context keeps computing correct results afterwards."""
import time

import numpy as np
import pytest

import syk_inputs as si
from oracle import hamiltonian as ham

pytestmark = pytest.mark.gpu


def test_bounded_wait_expires_and_context_survives():
    import torch

    import paper_2311_00639_b300 as syk
    from paper_2311_00639_b300 import _lib as L

    t0 = time.perf_counter()
    status = syk.bounded_wait_selftest()
    waited = time.perf_counter() - t0
    assert status == L.SYK_ETIMEOUT
    assert 0.5 < waited < 30.0  # the 1 s limit of the bounded wait, not an endless spin
    # the context is still usable: an H psi against the oracle
    N = 12
    q, J, _ = si.sample_sparse_syk(N, 4, r=2)
    HU, _ = ham.blocks(ham.dense_H(N, q, J, "jw"), N, "jw")
    psi = si.random_state(N, seed=3)[0]
    with syk.Terms(N, q, J, dtype="c128") as h:
        out = h.apply_H(torch.from_numpy(psi).cuda(), 0).cpu().numpy()
        assert h.device_error() == 0
    ref = HU @ psi
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(ref))
