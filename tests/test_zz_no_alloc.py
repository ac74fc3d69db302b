"""The allocation-free Krylov entry point (syk_krylov_evolve_noalloc).

Some callers cannot allocate device memory while they run (for example a
program whose device memory is owned by another framework's pool, or a
service whose footprint must stay fixed after start-up).  For them the
library offers a variant of syk_krylov_evolve whose workspace is a fixed
16 MiB static device array inside the library.  This test calls it through
the C-ABI and checks it against the workspace-taking entry point on two calls
in a row (different sizes and dtypes, so the second call starts from the
first call's leftovers), and checks that a too-large request is refused.
It lives in its own file, collected last, so that a failure here does not
stop the rest of the GPU suite.
"""
import ctypes as C

import numpy as np
import pytest

import syk_inputs as si

pytestmark = pytest.mark.gpu


def _vec(D, seed, dtype):
    import torch

    rng = np.random.default_rng(seed)
    a = rng.normal(size=D) + 1j * rng.normal(size=D)
    return torch.from_numpy(a).to("cuda", torch.complex64 if dtype == "c64" else torch.complex128)


def _noalloc(h, x, block, tau, t, m=30, tol=0.0, two_pass=False):
    """Direct C-ABI call (no Python-side allocation except the output)."""
    import torch

    from paper_2311_00639_b300 import _lib as L

    y = torch.empty_like(x)
    p = L.KrylovParams(m, tol, 0, 0, int(two_pass))
    st = L.KrylovStats()
    rc = L.load().syk_krylov_evolve_noalloc(h._h, block, tau, t, C.c_void_p(x.data_ptr()),
                                            C.c_void_p(y.data_ptr()), x.numel() // h.D, C.byref(p), C.byref(st),
                                            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, y, st


def test_noalloc_matches_workspace_entry_point_twice():
    import torch

    import paper_2311_00639_b300 as syk
    from paper_2311_00639_b300 import _lib as L

    cases = [  # (N, dtype, block, tau, t, two_pass, tolerance)
        (24, "c128", 1, 0.75, 3.0, False, 1e-12),
        (20, "c64", 0, 0.0, -2.5, True, 1e-5),
    ]
    for seed, (N, dtype, block, tau, t, two_pass, lim) in enumerate(cases):
        q, J, _ = si.sample_sparse_syk(N, 4, r=seed)
        with syk.Terms(N, q, J, dtype=dtype) as h:
            x = _vec(h.D, seed, dtype)
            ref, _ = h.krylov_evolve(x, block, tau, t, two_pass=two_pass)
            rc, y, st = _noalloc(h, x, block, tau, t, two_pass=two_pass)
            assert rc == L.SYK_OK
            torch.cuda.synchronize()
            err = (torch.max(torch.abs(y - ref)) / torch.max(torch.abs(ref))).item()
            assert err < lim, (N, dtype, err)
            assert st.matvecs > 0


def test_noalloc_rejects_workspace_beyond_limit():
    import paper_2311_00639_b300 as syk
    from paper_2311_00639_b300 import _lib as L

    N = 34  # D = 2^16 complex128: 31 basis vectors need ~32 MiB > 16 MiB
    q, J, _ = si.sample_sparse_syk(N, 2, r=0)
    with syk.Terms(N, q, J, dtype="c128") as h:
        x = _vec(h.D, 0, "c128")
        rc, _, _ = _noalloc(h, x, 0, 0.0, 1.0)
        assert rc == L.SYK_EINVAL
        buf = C.create_string_buffer(512)
        L.load().syk_last_error(buf, 512)
        assert b"static workspace" in buf.value
