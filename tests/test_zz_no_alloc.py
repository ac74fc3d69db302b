"""The allocation-free Krylov entry point (syk_krylov_evolve_noalloc).

Some callers cannot allocate device memory while they run (for example a
program whose device memory is owned by another framework's pool, or a
service whose footprint must stay fixed after start-up).  For them the
library offers a variant of syk_krylov_evolve whose workspace is a fixed
16 MiB static device array inside the library.  This test calls it through
the C-ABI and checks it against the workspace-taking entry point on two calls
in a row (different sizes and dtypes, so the second call starts from the
first call's leftovers), with several states per call and with a
non-Hermitian (Arnoldi) handle, checks that a too-large request is refused,
and that once a warm-up call has been made, later calls leave the device's
free memory unchanged.
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


def _noalloc(h, x, block, tau, t, m=30, tol=0.0, two_pass=False, y=None):
    """Direct C-ABI call (no Python-side allocation except the output, unless
    the caller passes y)."""
    import torch

    from paper_2311_00639_b300 import _lib as L

    y = torch.empty_like(x) if y is None else y
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


def test_noalloc_several_states_and_arnoldi_handle():
    """nstates = 2 in one call (the states share the static array in turn),
    and a handle with complex couplings (Arnoldi workspace layout), each
    against syk_krylov_evolve with a caller workspace."""
    import torch

    import paper_2311_00639_b300 as syk
    from paper_2311_00639_b300 import _lib as L

    N = 22
    q, J, _ = si.sample_sparse_syk(N, 4, r=7)
    with syk.Terms(N, q, J, dtype="c128") as h:
        xs = torch.stack([_vec(h.D, 11, "c128"), _vec(h.D, 12, "c128")]).contiguous()
        ref, _ = h.krylov_evolve(xs, 0, 0.3, 1.7)
        rc, y, st = _noalloc(h, xs, 0, 0.3, 1.7)
        assert rc == L.SYK_OK and st.matvecs > 0
        torch.cuda.synchronize()
        assert (torch.max(torch.abs(y - ref)) / torch.max(torch.abs(ref))).item() < 1e-12
    M = 0.3 * np.random.default_rng(8).normal(size=len(J)) * np.sqrt(np.mean(J ** 2))
    with syk.Terms.complex(N, q, J, M, dtype="c128") as h:
        assert not h.hermitian
        x = _vec(h.D, 13, "c128")
        ref, _ = h.krylov_evolve(x, 1, 0.2, -1.4, m=20)
        rc, y, _ = _noalloc(h, x, 1, 0.2, -1.4, m=20)
        assert rc == L.SYK_OK
        torch.cuda.synchronize()
        assert (torch.max(torch.abs(y - ref)) / torch.max(torch.abs(ref))).item() < 1e-12


def test_noalloc_later_calls_take_no_device_memory():
    """After one warm-up call (which reserves the static array and loads the
    kernels), two more calls leave cudaMemGetInfo's free bytes unchanged."""
    import torch

    import paper_2311_00639_b300 as syk
    from paper_2311_00639_b300 import _lib as L

    N = 20
    q, J, _ = si.sample_sparse_syk(N, 4, r=9)
    with syk.Terms(N, q, J, dtype="c64") as h:
        x = _vec(h.D, 14, "c64")
        y = torch.empty_like(x)
        rc, _, _ = _noalloc(h, x, 0, 0.1, 0.9, y=y)  # warm-up
        assert rc == L.SYK_OK
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for t in (1.1, -0.6):
            rc, _, _ = _noalloc(h, x, 0, 0.1, t, y=y)
            assert rc == L.SYK_OK
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
