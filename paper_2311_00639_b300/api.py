"""Python binding of libsyk: torch tensors in, C-ABI calls out.

Argument marshalling only — every step of the path runs in the CUDA library.
Torch provides device memory and streams.  Names follow include/syk.h.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L

_DT = {"c64": L.SYK_C64, "c128": L.SYK_C128}
_REP = {"jw": L.SYK_REP_JW, "paper": L.SYK_REP_PAPER}


def _torch():
    import torch

    return torch


def _tdtype(dtype: str):
    torch = _torch()
    return torch.complex64 if dtype == "c64" else torch.complex128


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _host_arrays(quads, J):
    q = np.ascontiguousarray(np.asarray(quads, dtype=np.int32).reshape(-1, 4))
    j = np.ascontiguousarray(np.asarray(J, dtype=np.float64).reshape(-1))
    if q.shape[0] != j.shape[0]:
        raise ValueError("quads and J lengths differ")
    return q, j


def bounded_wait_selftest(stream=None) -> int:
    """Status of syk_bounded_wait_selftest: SYK_ETIMEOUT (-4) when the bounded
    device wait expired as intended (the failure path, without a fault)."""
    return int(L.load().syk_bounded_wait_selftest(_stream(stream)))


def probe_staging(buf, reads: int, jobs_per_cta: int = 4096, stream=None) -> float:
    """Bytes/s of the matvec's bulk-copy pipeline shape over the CUDA tensor
    `buf` (syk_probe_staging; reads = -1, 0, 1 or 2)."""
    v = C.c_double(0.0)
    L.check(L.load().syk_probe_staging(_ptr(buf), buf.numel() * buf.element_size(), int(reads), int(jobs_per_cta),
                                       C.byref(v), _stream(stream)))
    return v.value


def _relabel_once(N, q, j, iterations, seed, tile_bits):
    perm = np.zeros(N, np.int32)
    qo = np.zeros_like(q)
    jo = np.zeros_like(j)
    b, a = C.c_int64(0), C.c_int64(0)
    L.check(L.load().syk_relabel_majoranas(N, q.shape[0], q.ctypes.data, j.ctypes.data, int(tile_bits),
                                           int(iterations), C.c_uint64(seed), perm.ctypes.data, qo.ctypes.data,
                                           jo.ctypes.data, C.byref(b), C.byref(a)))
    return {"perm": perm, "quads": qo, "J": jo, "patterns_before": b.value, "patterns_after": a.value,
            "seed": int(seed)}


def relabel_for_locality(N: int, quads, J, iterations: int = 200000, seed: int = 1, tile_bits: int = 11,
                         restarts: int = 1, dtype: str = "c64", M=None):
    """A Jordan-Wigner ordering of the Majoranas with fewer distinct flip
    patterns above the matvec tile (syk_relabel_majoranas).  Returns
    {"perm", "quads", "J", "patterns_before", "patterns_after", "seed"}:
    physical Majorana i is Jordan-Wigner Majorana perm[i]; quads / J are the
    same Hamiltonian in the new labels (for Terms(N, quads, J)); perm[N-2] =
    N-2 and perm[N-1] = N-1.

    restarts > 1 runs the search from seeds seed, seed + 1, ... (in parallel
    threads; the library call releases the GIL) and keeps the labels whose
    default pass plan (syk_plan_host) stages the fewest tiles, counting each
    pass after the first as one more staged tile and each straggler term,
    read from HBM, as a third of one (the planner's default HBM/L2 cost
    ratio); the result then also carries "plan_costs" [(seed, cost)].

    M (optional): imaginary parts of complex couplings J + iM.  Terms keep
    their order and each is the original times (-1)^(inversions of its
    reordered indices), so the result's "M" is M with J's sign flips (the
    search itself looks at the flip patterns only)."""
    q, j = _host_arrays(quads, J)
    if restarts <= 1:
        res = _relabel_once(N, q, j, iterations, seed, tile_bits)
    else:
        res = _relabel_multistart(N, q, j, iterations, seed, tile_bits, restarts, dtype)
    if M is not None:  # the sign of each reordered product, from the permutation (J may be 0)
        v = res["perm"][q]
        inv = sum((v[:, a] > v[:, b]).astype(np.int64) for a in range(4) for b in range(a + 1, 4))
        res["M"] = np.asarray(M, dtype=np.float64) * np.where(inv & 1, -1.0, 1.0)
    return res


def _relabel_multistart(N, q, j, iterations, seed, tile_bits, restarts, dtype):
    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(max_workers=int(restarts)) as ex:
        cands = list(ex.map(lambda sd: _relabel_once(N, q, j, iterations, sd, tile_bits),
                            range(int(seed), int(seed) + int(restarts))))

    def cost(r):
        p = plan_host(N, r["quads"], r["J"], dtype=dtype)
        return p["n_runs"] + len(p["passes"]) - 1 + int(np.sum(p["straggler"])) / 3.0

    costs = [(r["seed"], cost(r)) for r in cands]
    best = min(range(len(cands)), key=lambda i: (costs[i][1], i))
    return dict(cands[best], plan_costs=costs)


def tridiag_exp(alpha, beta, z: complex, tol: float, force_ql: bool = False, timed: bool = False):
    """The Krylov engine's projected-exponential step on a given Lanczos matrix
    (syk_tridiag_exp): returns (c complex [m], s_acc, err, used_ql), plus the
    kernel time in ms (median of 5 launches) when timed."""
    a = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(beta, dtype=np.float64))
    if a.shape != b.shape:
        raise ValueError("alpha and beta lengths differ")
    c = np.zeros((len(a), 2))
    s, e, q, ms = C.c_double(0.0), C.c_double(0.0), C.c_int(0), C.c_double(0.0)
    L.check(L.load().syk_tridiag_exp(len(a), a.ctypes.data, b.ctypes.data, float(np.real(z)), float(np.imag(z)),
                                     float(tol), int(bool(force_ql)), c.ctypes.data, C.byref(s), C.byref(e),
                                     C.byref(q), C.byref(ms) if timed else None))
    out = (c[:, 0] + 1j * c[:, 1], s.value, e.value, bool(q.value))
    return out + (ms.value,) if timed else out


def probe_smem(stream=None) -> float:
    """Bytes per second of 16-byte shared-memory loads of the GPU (syk_probe_smem)."""
    v = C.c_double(0.0)
    L.check(L.load().syk_probe_smem(C.byref(v), _stream(stream)))
    return v.value


def probe_fp64(stream=None) -> float:
    """FP64 fused multiply-adds per second of the GPU (syk_probe_fp64)."""
    v = C.c_double(0.0)
    L.check(L.load().syk_probe_fp64(C.byref(v), _stream(stream)))
    return v.value


def compile_terms_host(N: int, quads, J, rep: str = "jw") -> dict:
    """Host-only term compilation (no GPU): x, z, coef_U, coef_D, imag arrays."""
    lib = L.load()
    q, j = _host_arrays(quads, J)
    n = C.c_int64(0)
    L.check(lib.syk_compile_terms_host(N, q.shape[0], q.ctypes.data, j.ctypes.data, _REP[rep], 0, C.byref(n),
                                       None, None, None, None, None))
    cnt = n.value
    out = {"x": np.zeros(cnt, np.uint32), "z": np.zeros(cnt, np.uint32), "coef_U": np.zeros(cnt),
           "coef_D": np.zeros(cnt), "imag": np.zeros(cnt, np.uint8)}
    L.check(lib.syk_compile_terms_host(N, q.shape[0], q.ctypes.data, j.ctypes.data, _REP[rep], cnt, C.byref(n),
                                       out["x"].ctypes.data, out["z"].ctypes.data, out["coef_U"].ctypes.data,
                                       out["coef_D"].ctypes.data, out["imag"].ctypes.data))
    return out


def _plan_outputs(call) -> dict:
    """Run a syk_plan_*_host call twice (sizes, then arrays) and unpack it."""
    o = L.PlanHostOut()
    L.check(call(C.byref(o)))
    n, P = o.n_terms, o.n_passes
    passes = (L.PassInfo * max(P, 1))()
    out = {"x": np.zeros(n, np.uint32), "z": np.zeros(n, np.uint32), "coef_U": np.zeros(n), "coef_D": np.zeros(n),
           "imag": np.zeros(n, np.uint8), "straggler": np.zeros(n, np.uint8),
           "records": np.zeros((2, n + 1, 4), np.uint32)}
    o = L.PlanHostOut(term_capacity=n, pass_capacity=P, passes=C.cast(passes, C.c_void_p),
                      **{k: v.ctypes.data for k, v in out.items()})
    L.check(call(C.byref(o)))
    out["n_runs"] = o.n_runs
    out["n_merges"] = o.n_merges
    out["passes"] = [{"t0": p.t0, "ti": p.ti, "t1": p.t1, "emask": p.emask, "cls": list(p.cls),
                      "split_chunks": p.split_chunks, "split_terms": p.split_terms,
                      "dep": np.array([list(p.dep[b]) for b in range(3)], np.uint32)} for p in passes[:P]]
    return out


def plan_host(N: int, quads, J, dtype: str = "c64", rep: str = "jw", l2_budget_bytes: int = 0,
              straggler_ratio: float = 0.0, n_sm: int = 148) -> dict:
    """Host-only (no GPU): the matvec pass plan and complex64 record layout that
    Terms(...) followed by replan(l2_budget_bytes, straggler_ratio) would use."""
    lib = L.load()
    q, j = _host_arrays(quads, J)
    return _plan_outputs(lambda o: lib.syk_plan_host(N, q.shape[0], q.ctypes.data, j.ctypes.data, _DT[dtype],
                                                     _REP[rep], l2_budget_bytes, float(straggler_ratio), n_sm, o))


def plan_strings_host(L_bits: int, strings: dict, dtype: str = "c64", l2_budget_bytes: int = 0,
                      straggler_ratio: float = 0.0, n_sm: int = 148) -> dict:
    """Host-only (no GPU): the plan and records for compiled strings on L_bits
    index bits, e.g. compile_pauli_host(...) (coef used for both blocks) or
    compile_terms_complex_host(...)."""
    lib = L.load()
    x = np.ascontiguousarray(strings["x"], dtype=np.uint32)
    z = np.ascontiguousarray(strings["z"], dtype=np.uint32)
    cu = np.ascontiguousarray(strings.get("coef_U", strings.get("coef")), dtype=np.float64)
    cd = np.ascontiguousarray(strings.get("coef_D", strings.get("coef")), dtype=np.float64)
    im = np.ascontiguousarray(strings["imag"], dtype=np.uint8)
    return _plan_outputs(lambda o: lib.syk_plan_strings_host(L_bits, len(x), x.ctypes.data, z.ctypes.data,
                                                             cu.ctypes.data, cd.ctypes.data, im.ctypes.data,
                                                             _DT[dtype], l2_budget_bytes, float(straggler_ratio),
                                                             n_sm, o))


def _pauli_arrays(x, z, h):
    xa = np.ascontiguousarray(np.asarray(x, dtype=np.uint32).reshape(-1))
    za = np.ascontiguousarray(np.asarray(z, dtype=np.uint32).reshape(-1))
    ha = np.ascontiguousarray(np.asarray(h, dtype=np.float64).reshape(-1))
    if not (xa.shape == za.shape == ha.shape):
        raise ValueError("x, z and h lengths differ")
    return xa, za, ha


def compile_pauli_host(n_qubits: int, x, z, h) -> dict:
    """Host-only compilation of a Pauli-string Hamiltonian (no GPU): x, z,
    coef, imag arrays with (H psi)[m] = sum coef (imag ? i : 1)
    (-1)^{popc(z & m)} psi[m ^ x]."""
    lib = L.load()
    xa, za, ha = _pauli_arrays(x, z, h)
    n = C.c_int64(0)
    L.check(lib.syk_compile_pauli_host(n_qubits, len(ha), xa.ctypes.data, za.ctypes.data, ha.ctypes.data, 0,
                                       C.byref(n), None, None, None, None))
    cnt = n.value
    out = {"x": np.zeros(cnt, np.uint32), "z": np.zeros(cnt, np.uint32), "coef": np.zeros(cnt),
           "imag": np.zeros(cnt, np.uint8)}
    L.check(lib.syk_compile_pauli_host(n_qubits, len(ha), xa.ctypes.data, za.ctypes.data, ha.ctypes.data, cnt,
                                       C.byref(n), out["x"].ctypes.data, out["z"].ctypes.data,
                                       out["coef"].ctypes.data, out["imag"].ctypes.data))
    return out


def compile_terms_complex_host(N: int, quads, J_re, J_im, rep: str = "jw") -> dict:
    """Host-only compilation with complex couplings J_re + i J_im (no GPU)."""
    lib = L.load()
    q, jr = _host_arrays(quads, J_re)
    ji = np.ascontiguousarray(np.asarray(J_im, dtype=np.float64).reshape(-1))
    if ji.shape != jr.shape:
        raise ValueError("J_re and J_im lengths differ")
    n = C.c_int64(0)
    args = (N, q.shape[0], q.ctypes.data, jr.ctypes.data, ji.ctypes.data, _REP[rep])
    L.check(lib.syk_compile_terms_complex_host(*args, 0, C.byref(n), None, None, None, None, None))
    cnt = n.value
    out = {"x": np.zeros(cnt, np.uint32), "z": np.zeros(cnt, np.uint32), "coef_U": np.zeros(cnt),
           "coef_D": np.zeros(cnt), "imag": np.zeros(cnt, np.uint8)}
    L.check(lib.syk_compile_terms_complex_host(*args, cnt, C.byref(n), out["x"].ctypes.data, out["z"].ctypes.data,
                                               out["coef_U"].ctypes.data, out["coef_D"].ctypes.data,
                                               out["imag"].ctypes.data))
    return out


def compile_chi_host(N: int, n: int, rep: str = "jw") -> dict:
    lib = L.load()
    x, z = C.c_uint32(0), C.c_uint32(0)
    re, im = (C.c_double * 2)(), (C.c_double * 2)()
    L.check(lib.syk_compile_chi_host(N, _REP[rep], n, C.byref(x), C.byref(z), re, im))
    return {"x": x.value, "z": z.value, "coef": [complex(re[0], im[0]), complex(re[1], im[1])]}


class KrylovStats:
    def __init__(self, s: L.KrylovStats):
        self.matvecs, self.substeps, self.err_est = s.matvecs, s.substeps, s.err_est

    def __repr__(self):
        return f"KrylovStats(matvecs={self.matvecs}, substeps={self.substeps}, err_est={self.err_est:.3g})"


def _params(m=0, tol=None, max_substeps=0, reorth=False, two_pass=False):
    """syk_krylov_params; zero fields take the library's defaults (m: 20 for
    complex64, 30 for complex128)."""
    return L.KrylovParams(int(m), float(tol or 0.0), int(max_substeps), int(bool(reorth)), int(bool(two_pass)))


class Terms:
    """A compiled sparse-SYK Hamiltonian resident on the current CUDA device."""

    def __init__(self, N: int, quads, J, dtype: str = "c64", rep: str = "jw"):
        self._lib = L.load()
        q, j = _host_arrays(quads, J)
        h = C.c_void_p()
        L.check(self._lib.syk_build_terms(N, q.shape[0], q.ctypes.data, j.ctypes.data, _DT[dtype], _REP[rep],
                                          C.byref(h)))
        self._h = h
        self.N, self.dtype, self.rep = N, dtype, rep
        info = L.TermsInfo()
        L.check(self._lib.syk_terms_get_info(h, C.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in L.TermsInfo._fields_}
        self.D = info.D
        self.n_terms = info.n_terms

    @classmethod
    def _from_handle(cls, h, N: int, dtype: str, rep: str):
        self = cls.__new__(cls)
        self._lib = L.load()
        self._h = h
        self.N, self.dtype, self.rep = N, dtype, rep
        info = L.TermsInfo()
        L.check(self._lib.syk_terms_get_info(h, C.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in L.TermsInfo._fields_}
        self.D = info.D
        self.n_terms = info.n_terms
        return self

    @classmethod
    def complex(cls, N: int, quads, J_re, J_im, dtype: str = "c64", rep: str = "jw") -> "Terms":
        """Non-Hermitian sparse SYK: couplings J_re + i J_im (syk_build_terms_complex).
        krylov_evolve uses Arnoldi when any J_im is non-zero; the OTOC is
        otoc_nonhermitian."""
        lib = L.load()
        q, jr = _host_arrays(quads, J_re)
        ji = np.ascontiguousarray(np.asarray(J_im, dtype=np.float64).reshape(-1))
        if ji.shape != jr.shape:
            raise ValueError("J_re and J_im lengths differ")
        h = C.c_void_p()
        L.check(lib.syk_build_terms_complex(N, q.shape[0], q.ctypes.data, jr.ctypes.data, ji.ctypes.data, _DT[dtype],
                                            _REP[rep], C.byref(h)))
        return cls._from_handle(h, N, dtype, rep)

    @property
    def hermitian(self) -> bool:
        v = C.c_int(0)
        L.check(self._lib.syk_terms_is_hermitian(self._h, C.byref(v)))
        return bool(v.value)

    def adjoint(self) -> "Terms":
        """A new handle for H^dagger (syk_terms_adjoint)."""
        h = C.c_void_p()
        L.check(self._lib.syk_terms_adjoint(self._h, C.byref(h)))
        out = type(self)._from_handle(h, self.N, self.dtype, self.rep)
        if hasattr(self, "n_qubits"):
            out.n_qubits = self.n_qubits
        return out

    def otoc_nonhermitian(self, a: int, b: int, t_grid, mode: str = "typical", n_states: int = 1, seed: int = 0,
                          psi=None, stream=None, **kp):
        """Infinite-temperature OTOC with W(t) = e^{iH^dag t} W e^{-iHt}
        (syk_otoc_nonhermitian).  Returns (F_raw complex [rows, n_t], otoc [n_t], KrylovStats).

        psi: optional CUDA tensor [n_states, 2, D] (U then D block per state).
        """
        tg = np.ascontiguousarray(np.asarray(t_grid, dtype=np.float64))
        md = L.SYK_OTOC_EXACT_TRACE if mode == "exact" else L.SYK_OTOC_TYPICAL
        if psi is not None:
            self._check_vec(psi)
            n_states = psi.numel() // (2 * self.D)
        rows = 1 if md == L.SYK_OTOC_EXACT_TRACE else n_states
        F = np.zeros((rows, len(tg), 2))
        o = np.zeros(len(tg))
        p = _params(**kp)
        st = L.KrylovStats()
        L.check(self._lib.syk_otoc_nonhermitian(self._h, a, b, tg.ctypes.data, len(tg), md, int(n_states),
                                                C.c_uint64(seed), None if psi is None else _ptr(psi), C.byref(p),
                                                F.ctypes.data, o.ctypes.data, C.byref(st), _stream(stream)))
        return F[..., 0] + 1j * F[..., 1], o, KrylovStats(st)

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._lib.syk_terms_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- helpers
    def empty(self, nstates: int = 1):
        torch = _torch()
        shape = (self.D,) if nstates == 1 else (nstates, self.D)
        return torch.empty(shape, dtype=_tdtype(self.dtype), device="cuda")

    def _check_vec(self, t, nstates=None):
        torch = _torch()
        if not t.is_cuda or t.dtype != _tdtype(self.dtype) or not t.is_contiguous():
            raise ValueError(f"expected a contiguous CUDA tensor of {_tdtype(self.dtype)}")
        if t.numel() % self.D:
            raise ValueError("tensor size is not a multiple of D")
        return t.numel() // self.D

    def device_error(self) -> int:
        """1 if a kernel on this handle hit its bounded-wait limit (synchronises)."""
        info = L.TermsInfo()
        L.check(self._lib.syk_terms_get_info(self._h, C.byref(info)))
        return int(info.device_error)

    def autotune(self, budgets_mb=(2.0, 8.0, 32.0, 64.0), ratios=(0.0, 1.5, 3.0), reps: int = 2, block: int = 0,
                 cache_path=None) -> dict:
        """Pick the matvec pass plan (L2 budget, straggler ratio) by timing
        syk_apply_H on this Hamiltonian; keeps the fastest plan.  With
        cache_path, the choice is stored per (term table, dtype, GPU) and reused."""
        import hashlib
        import json
        import os

        torch = _torch()
        ex = self.export()
        key = hashlib.sha256(b"".join([ex["x"].tobytes(), ex["z"].tobytes(), self.dtype.encode(),
                                      torch.cuda.get_device_name().encode()])).hexdigest()
        cache = {}
        if cache_path and os.path.exists(cache_path):
            try:
                cache = json.load(open(cache_path))
            except Exception:
                cache = {}
        if key in cache:
            c = cache[key]
            self.replan(int(c["budget"]), float(c["ratio"]))
            return dict(c, cached=True)
        psi = self.empty()
        psi.normal_()
        out = self.empty()
        trials = []
        for r in ratios:
            for bmb in budgets_mb:
                budget = int(bmb * (1 << 20))
                npass = self.replan(budget, r)
                self.apply_H(psi, block, out=out)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    self.apply_H(psi, block, out=out)
                e1.record()
                torch.cuda.synchronize()
                trials.append({"budget": budget, "ratio": r, "passes": npass, "ms": e0.elapsed_time(e1) / reps})
        best = min(trials, key=lambda t: t["ms"])
        self.replan(best["budget"], best["ratio"])
        res = dict(best, trials=trials, cached=False)
        if cache_path:
            cache[key] = {k: best[k] for k in ("budget", "ratio", "passes", "ms")}
            os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
            json.dump(cache, open(cache_path, "w"), indent=1)
        return res

    def replan(self, l2_budget_bytes: int = 0, straggler_ratio: float = 0.0):
        """Regroup the matvec passes (L2 budget in bytes, straggler cost ratio);
        l2_budget_bytes = 0 restores the dtype's default plan."""
        L.check(self._lib.syk_terms_replan(self._h, int(l2_budget_bytes), float(straggler_ratio)))
        info = L.TermsInfo()
        L.check(self._lib.syk_terms_get_info(self._h, C.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in L.TermsInfo._fields_}
        return self.info["n_passes"]

    def export(self) -> dict:
        n = self.n_terms
        out = {"x": np.zeros(n, np.uint32), "z": np.zeros(n, np.uint32), "coef_U": np.zeros(n),
               "coef_D": np.zeros(n), "imag": np.zeros(n, np.uint8)}
        L.check(self._lib.syk_terms_export(self._h, out["x"].ctypes.data, out["z"].ctypes.data,
                                           out["coef_U"].ctypes.data, out["coef_D"].ctypes.data,
                                           out["imag"].ctypes.data))
        return out

    # -- hot path
    def apply_H(self, psi, block: int, out=None, stream=None):
        ns = self._check_vec(psi)
        out = _torch().empty_like(psi) if out is None else out
        self._check_vec(out)
        L.check(self._lib.syk_apply_H(self._h, block, _ptr(psi), _ptr(out), ns, _stream(stream)))
        return out

    def apply_chi(self, i: int, psi, from_block: int, out=None, stream=None):
        ns = self._check_vec(psi)
        out = _torch().empty_like(psi) if out is None else out
        self._check_vec(out)
        L.check(self._lib.syk_apply_chi(self._h, i, from_block, _ptr(psi), _ptr(out), ns, _stream(stream)))
        return out

    def random_state(self, seed: int, state_id: int, stream=None, blocks=(0, 1)):
        """Unnormalised Philox/Box-Muller amplitudes (psi_U, psi_D); a block
        not listed in `blocks` is returned as None and not generated."""
        u = self.empty() if 0 in blocks else None
        d = self.empty() if 1 in blocks else None
        L.check(self._lib.syk_random_state(self._h, C.c_uint64(seed), C.c_uint64(state_id),
                                           None if u is None else _ptr(u), None if d is None else _ptr(d),
                                           _stream(stream)))
        return u, d

    def workspace_bytes(self, **kp) -> int:
        p = _params(**kp)
        return int(self._lib.syk_krylov_workspace_bytes(self._h, C.byref(p)))

    def krylov_evolve(self, x, block: int, tau: float, t: float, y=None, workspace=None, stream=None, **kp):
        """y = exp(-(tau + i t) H_block) x.  Returns (y, KrylovStats)."""
        torch = _torch()
        ns = self._check_vec(x)
        y = torch.empty_like(x) if y is None else y
        self._check_vec(y)
        p = _params(**kp)
        nb = int(self._lib.syk_krylov_workspace_bytes(self._h, C.byref(p)))
        if nb == 0:
            L.check(L.SYK_EINVAL)
        if workspace is None:
            workspace = torch.empty(nb, dtype=torch.uint8, device="cuda")
        st = L.KrylovStats()
        L.check(self._lib.syk_krylov_evolve(self._h, block, float(tau), float(t), _ptr(x), _ptr(y), ns,
                                            C.byref(p), _ptr(workspace), workspace.numel(), C.byref(st),
                                            _stream(stream)))
        return y, KrylovStats(st)

    def krylov_evolve_noalloc(self, x, block: int, tau: float, t: float, y=None, stream=None, **kp):
        """Same as krylov_evolve, but the library takes the workspace from its
        fixed static device array instead of a caller buffer (for callers that
        cannot allocate device memory while they run; 16 MiB limit, calls on a
        device must not overlap).  Returns (y, KrylovStats)."""
        ns = self._check_vec(x)
        y = _torch().empty_like(x) if y is None else y
        self._check_vec(y)
        p = _params(**kp)
        st = L.KrylovStats()
        L.check(self._lib.syk_krylov_evolve_noalloc(self._h, block, float(tau), float(t), _ptr(x), _ptr(y), ns,
                                                    C.byref(p), C.byref(st), _stream(stream)))
        return y, KrylovStats(st)

    def otoc(self, a: int, b: int, beta: float, t_grid, mode: str = "typical", n_states: int = 1, seed: int = 0,
             psi=None, stream=None, **kp):
        """Regularised OTOC.  Returns (F_raw complex [rows, n_t], otoc [n_t], KrylovStats).

        psi: optional CUDA tensor [n_states, 2, D] (U then D block per state).
        """
        tg = np.ascontiguousarray(np.asarray(t_grid, dtype=np.float64))
        md = L.SYK_OTOC_EXACT_TRACE if mode == "exact" else L.SYK_OTOC_TYPICAL
        if psi is not None:
            self._check_vec(psi)
            n_states = psi.numel() // (2 * self.D)
        rows = 1 if md == L.SYK_OTOC_EXACT_TRACE else n_states
        F = np.zeros((rows, len(tg), 2))
        o = np.zeros(len(tg))
        p = _params(**kp)
        st = L.KrylovStats()
        L.check(self._lib.syk_otoc(self._h, a, b, float(beta), tg.ctypes.data, len(tg), md, int(n_states),
                                   C.c_uint64(seed), None if psi is None else _ptr(psi), C.byref(p),
                                   F.ctypes.data, o.ctypes.data, C.byref(st), _stream(stream)))
        return F[..., 0] + 1j * F[..., 1], o, KrylovStats(st)


class PauliTerms(Terms):
    """A Pauli-string (spin-chain) Hamiltonian H = sum_t h_t P(x_t, z_t) on
    n_qubits qubits, resident on the current CUDA device
    (syk_build_pauli_terms).  A string is two masks: on qubit q, x alone =
    sigma_x, z alone = sigma_z, both = sigma_y.  States have D = 2^n_qubits
    amplitudes; apply_H / krylov_evolve take block 0.  The Majorana calls
    (apply_chi, otoc, Batch.submit) refuse this handle."""

    def __init__(self, n_qubits: int, x, z, h, dtype: str = "c64"):
        self._lib = L.load()
        xa, za, ha = _pauli_arrays(x, z, h)
        hd = C.c_void_p()
        L.check(self._lib.syk_build_pauli_terms(int(n_qubits), len(ha), xa.ctypes.data, za.ctypes.data,
                                                ha.ctypes.data, _DT[dtype], C.byref(hd)))
        self._h = hd
        self.N, self.dtype, self.rep, self.n_qubits = 0, dtype, "pauli", int(n_qubits)
        info = L.TermsInfo()
        L.check(self._lib.syk_terms_get_info(hd, C.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in L.TermsInfo._fields_}
        self.D = info.D
        self.n_terms = info.n_terms

    def apply_pauli(self, x: int, z: int, psi, out=None, stream=None):
        """out = P(x, z) psi (coefficient 1)."""
        ns = self._check_vec(psi)
        out = _torch().empty_like(psi) if out is None else out
        self._check_vec(out)
        L.check(self._lib.syk_apply_pauli(self._h, int(x), int(z), _ptr(psi), _ptr(out), ns, _stream(stream)))
        return out

    def pauli_otoc(self, W, V, beta: float, t_grid, mode: str = "typical", n_states: int = 1, seed: int = 0,
                   psi=None, stream=None, **kp):
        """Regularised OTOC of Eq. (2) with Pauli strings W = (x, z) and
        V = (x, z).  Returns (F_raw complex [rows, n_t], otoc [n_t], KrylovStats).

        psi: optional CUDA tensor [n_states, D] of states, used as given.
        """
        tg = np.ascontiguousarray(np.asarray(t_grid, dtype=np.float64))
        md = L.SYK_OTOC_EXACT_TRACE if mode == "exact" else L.SYK_OTOC_TYPICAL
        if psi is not None:
            n_states = self._check_vec(psi)
        rows = 1 if md == L.SYK_OTOC_EXACT_TRACE else n_states
        F = np.zeros((rows, len(tg), 2))
        o = np.zeros(len(tg))
        p = _params(**kp)
        st = L.KrylovStats()
        L.check(self._lib.syk_pauli_otoc(self._h, int(W[0]), int(W[1]), int(V[0]), int(V[1]), float(beta),
                                         tg.ctypes.data, len(tg), md, int(n_states), C.c_uint64(seed),
                                         None if psi is None else _ptr(psi), C.byref(p), F.ctypes.data,
                                         o.ctypes.data, C.byref(st), _stream(stream)))
        return F[..., 0] + 1j * F[..., 1], o, KrylovStats(st)


class Batch:
    """Batched OTOC engine (syk_batch_*): many typical-state OTOC curves at once.

    submit() admits a job if a slot and arena memory are free (returns False
    otherwise); run() advances all live jobs and returns the finished ones as
    dicts {tag, F (complex [n_t]), otoc (normalised), matvecs, substeps, status}.
    """

    def __init__(self, dtype: str = "c64", max_slots: int = 64, max_bytes: int = 1 << 30, m: int = 0, tol=None):
        self._lib = L.load()
        h = C.c_void_p()
        p = _params(m=m, tol=tol)
        L.check(self._lib.syk_batch_create(_DT[dtype], int(max_slots), int(max_bytes), C.byref(p), C.byref(h)))
        self._h = h
        self.dtype = dtype
        self._pending = {}  # tag -> (F buffer, stats, status, t_grid, terms)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.syk_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def job_bytes(self, terms: "Terms", n_t: int) -> int:
        return int(self._lib.syk_batch_job_bytes(self._h, terms._h, int(n_t)))

    def submit(self, terms: "Terms", a: int, b: int, beta: float, t_grid, seed: int, state_id: int, tag: int,
               basis_index: int = -1, kind: str = "otoc") -> bool:
        """kind: "otoc" (Eq. (2), F(t)) or "green" (G(t) with Majorana a; b unused)."""
        if terms.dtype != self.dtype:
            raise ValueError("terms dtype differs from the batch dtype")
        tg = np.ascontiguousarray(np.asarray(t_grid, dtype=np.float64))
        F = np.zeros((len(tg), 2))
        o = np.zeros(len(tg))
        st = L.KrylovStats()
        status = C.c_int(0)
        job = L.OtocJob(terms._h, int(a), int(b), float(beta), tg.ctypes.data, len(tg), C.c_uint64(seed),
                        C.c_uint64(state_id), int(tag), F.ctypes.data, C.addressof(st), C.addressof(status),
                        int(basis_index), 1 if kind == "green" else 0, o.ctypes.data)
        rc = self._lib.syk_batch_submit(self._h, C.byref(job))
        if rc == L.SYK_EAGAIN:
            return False
        L.check(rc)
        self._pending[int(tag)] = (F, o, st, status, tg, terms)
        return True

    def run(self, max_ticks: int = 1 << 20, ticks_per_sync: int = 8):
        n = C.c_int(0)
        cap = max(1, len(self._pending))
        tags = (C.c_int64 * cap)()
        L.check(self._lib.syk_batch_run(self._h, int(max_ticks), int(ticks_per_sync), C.byref(n), tags, cap))
        out = []
        for i in range(min(n.value, cap)):
            F, o, st, status, tg, _ = self._pending.pop(int(tags[i]))
            out.append({"tag": int(tags[i]), "F": F[:, 0] + 1j * F[:, 1], "otoc": o, "matvecs": st.matvecs,
                        "substeps": st.substeps, "status": status.value})
        return out

    def info(self) -> dict:
        live, used, free = C.c_int(0), C.c_size_t(0), C.c_size_t(0)
        L.check(self._lib.syk_batch_info(self._h, C.byref(live), C.byref(used), C.byref(free)))
        return {"live": live.value, "bytes_in_use": used.value, "largest_free": free.value}

    @property
    def pending(self) -> int:
        return len(self._pending)

    def drain(self, max_ticks: int = 1 << 20, ticks_per_sync: int = 8):
        """Run until every admitted job has finished; returns all results."""
        out = []
        while self._pending:
            out += self.run(max_ticks, ticks_per_sync)
        return out


def autotune_batch(jobs, dtype: str = "c64", ms=(16, 20, 24, 30), ticks=(8, 16, 32), max_slots: int = 0,
                   max_bytes: int = 8 << 30, tol=None) -> dict:
    """Pick the batched engine's Krylov dimension m and host sync period
    (ticks between collections of finished jobs) by timing a sample of the
    workload through syk_batch_*.

    jobs: (terms, a, b, beta, t_grid, seed, state_id) tuples, e.g. a random
    sample of the jobs of a batched run.  Each (m, ticks) pair runs the whole
    sample in a fresh batch, after one untimed run; a pair with a failed job
    is not chosen unless every pair has one.  Returns {"m", "ticks_per_sync",
    "trials": [{"m", "ticks_per_sync", "s", "failed"}, ...]}."""
    import time

    torch = _torch()

    def run(m, tps):
        with Batch(dtype=dtype, max_slots=max_slots or len(jobs), max_bytes=max_bytes, m=m, tol=tol) as b:
            queue = list(enumerate(jobs))
            failed = 0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            while queue or b.pending:
                while queue and b.submit(*queue[0][1], tag=queue[0][0]):
                    queue.pop(0)
                for res in b.run(ticks_per_sync=tps):
                    failed += int(res["status"] != 0)
            return time.perf_counter() - t0, failed

    run(ms[0], ticks[0])  # first use: graph capture, module loading
    trials = []
    for m in ms:
        for tps in ticks:
            wall, failed = run(m, tps)
            trials.append({"m": int(m), "ticks_per_sync": int(tps), "s": wall, "failed": failed})
    ok = [t for t in trials if t["failed"] == 0] or trials
    best = min(ok, key=lambda t: t["s"])
    return {"m": best["m"], "ticks_per_sync": best["ticks_per_sync"], "trials": trials}


def exact_trace_otoc(terms: "Terms", pairs, beta: float, t_grid, max_slots: int = 4096, max_bytes: int = 8 << 30,
                     m: int = 30, tol=None):
    """Exact-trace OTOC of Eq. (2) for each (a, b) in pairs, by the batched
    engine over all 2D basis states (syk_otoc_exact_trace_batched:
    F_tr(t) = sum_g F_{e_g}(t) / 2D and OTOC = Re F_tr / Re F_tr(0), summed in
    the library).  Returns {(a, b): (F complex [n_t], otoc [n_t])}."""
    tg = np.ascontiguousarray(np.asarray(t_grid, dtype=np.float64))
    pr = np.ascontiguousarray(np.asarray([tuple(p) for p in pairs], dtype=np.int32).reshape(-1, 2))
    F = np.zeros((len(pr), len(tg), 2))
    o = np.zeros((len(pr), len(tg)))
    p = _params(m=m, tol=tol)
    jobs = len(pr) * 2 * terms.D
    L.check(terms._lib.syk_otoc_exact_trace_batched(terms._h, len(pr), pr.ctypes.data, float(beta), tg.ctypes.data,
                                                    len(tg), int(min(max_slots, jobs)), int(max_bytes), C.byref(p),
                                                    F.ctypes.data, o.ctypes.data, None))
    return {(int(a), int(b)): (F[i, :, 0] + 1j * F[i, :, 1], o[i]) for i, (a, b) in enumerate(pr)}
