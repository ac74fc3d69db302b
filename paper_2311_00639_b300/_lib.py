"""ctypes declarations of libsyk (include/syk.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsyk.so")

SYK_OK, SYK_EINVAL, SYK_ENOMEM, SYK_ENOCONV, SYK_ETIMEOUT, SYK_ECUDA, SYK_EAGAIN = 0, -1, -2, -3, -4, -5, -6
SYK_C64, SYK_C128 = 0, 1
SYK_REP_JW, SYK_REP_PAPER, SYK_REP_PAULI = 0, 1, 2
SYK_OTOC_TYPICAL, SYK_OTOC_EXACT_TRACE = 0, 1


class TermsInfo(C.Structure):
    _fields_ = [("N", C.c_int), ("L", C.c_int), ("dtype", C.c_int), ("rep", C.c_int), ("D", C.c_int64),
                ("n_input", C.c_int64), ("n_terms", C.c_int64), ("n_real", C.c_int64),
                ("n_xgroups", C.c_int64), ("sum_abs_coef", C.c_double), ("n_passes", C.c_int64),
                ("device_error", C.c_int64), ("n_tile_reads", C.c_int64), ("n_merged", C.c_int64)]


class KrylovParams(C.Structure):
    _fields_ = [("m", C.c_int), ("tol", C.c_double), ("max_substeps", C.c_int), ("reorth", C.c_int),
                ("two_pass", C.c_int)]


class KrylovStats(C.Structure):
    _fields_ = [("matvecs", C.c_int64), ("substeps", C.c_int64), ("err_est", C.c_double)]


class OtocJob(C.Structure):
    _fields_ = [("h", C.c_void_p), ("a", C.c_int), ("b", C.c_int), ("beta", C.c_double), ("t_grid", C.c_void_p),
                ("n_t", C.c_int), ("seed", C.c_uint64), ("state_id", C.c_uint64), ("tag", C.c_int64),
                ("F_out", C.c_void_p), ("stats", C.c_void_p), ("status_out", C.c_void_p),
                ("basis_index", C.c_int64), ("kind", C.c_int), ("otoc_out", C.c_void_p)]


class PassInfo(C.Structure):
    _fields_ = [("t0", C.c_int32), ("ti", C.c_int32), ("t1", C.c_int32), ("emask", C.c_uint32),
                ("cls", C.c_int32 * 9), ("split_chunks", C.c_int32), ("split_terms", C.c_int32),
                ("dep", (C.c_uint32 * 256) * 3)]


class PlanHostOut(C.Structure):
    _fields_ = [("term_capacity", C.c_int64), ("pass_capacity", C.c_int64), ("passes", C.c_void_p),
                ("x", C.c_void_p), ("z", C.c_void_p), ("coef_U", C.c_void_p), ("coef_D", C.c_void_p),
                ("imag", C.c_void_p), ("straggler", C.c_void_p), ("records", C.c_void_p),
                ("n_terms", C.c_int64), ("n_passes", C.c_int64), ("n_runs", C.c_int64), ("n_merges", C.c_int64)]


# name -> (restype, argtypes); every symbol include/syk.h declares.
_P = C.c_void_p
_I, _I64, _U64, _D, _SZ = C.c_int, C.c_int64, C.c_uint64, C.c_double, C.c_size_t
SIGNATURES = {
    "syk_build_terms": (_I, [_I, _I64, _P, _P, _I, _I, C.POINTER(_P)]),
    "syk_terms_destroy": (_I, [_P]),
    "syk_terms_get_info": (_I, [_P, C.POINTER(TermsInfo)]),
    "syk_terms_replan": (_I, [_P, _SZ, _D]),
    "syk_terms_export": (_I, [_P, _P, _P, _P, _P, _P]),
    "syk_compile_terms_host": (_I, [_I, _I64, _P, _P, _I, _I64, C.POINTER(_I64), _P, _P, _P, _P, _P]),
    "syk_compile_chi_host": (_I, [_I, _I, _I, _P, _P, _P, _P]),
    "syk_plan_host": (_I, [_I, _I64, _P, _P, _I, _I, _SZ, _D, _I, C.POINTER(PlanHostOut)]),
    "syk_plan_strings_host": (_I, [_I, _I64, _P, _P, _P, _P, _P, _I, _SZ, _D, _I, C.POINTER(PlanHostOut)]),
    "syk_apply_H": (_I, [_P, _I, _P, _P, _I64, _P]),
    "syk_apply_chi": (_I, [_P, _I, _I, _P, _P, _I64, _P]),
    "syk_random_state": (_I, [_P, _U64, _U64, _P, _P, _P]),
    "syk_krylov_workspace_bytes": (_SZ, [_P, C.POINTER(KrylovParams)]),
    "syk_krylov_evolve": (_I, [_P, _I, _D, _D, _P, _P, _I64, C.POINTER(KrylovParams), _P, _SZ,
                               C.POINTER(KrylovStats), _P]),
    "syk_krylov_evolve_noalloc": (_I, [_P, _I, _D, _D, _P, _P, _I64, C.POINTER(KrylovParams),
                                       C.POINTER(KrylovStats), _P]),
    "syk_otoc": (_I, [_P, _I, _I, _D, _P, _I, _I, _I, _U64, _P, C.POINTER(KrylovParams), _P, _P,
                      C.POINTER(KrylovStats), _P]),
    "syk_build_pauli_terms": (_I, [_I, _I64, _P, _P, _P, _I, C.POINTER(_P)]),
    "syk_compile_pauli_host": (_I, [_I, _I64, _P, _P, _P, _I64, C.POINTER(_I64), _P, _P, _P, _P]),
    "syk_apply_pauli": (_I, [_P, C.c_uint32, C.c_uint32, _P, _P, _I64, _P]),
    "syk_pauli_otoc": (_I, [_P, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, _D, _P, _I, _I, _I, _U64, _P,
                            C.POINTER(KrylovParams), _P, _P, C.POINTER(KrylovStats), _P]),
    "syk_build_terms_complex": (_I, [_I, _I64, _P, _P, _P, _I, _I, C.POINTER(_P)]),
    "syk_compile_terms_complex_host": (_I, [_I, _I64, _P, _P, _P, _I, _I64, C.POINTER(_I64), _P, _P, _P, _P, _P]),
    "syk_terms_is_hermitian": (_I, [_P, C.POINTER(_I)]),
    "syk_terms_adjoint": (_I, [_P, C.POINTER(_P)]),
    "syk_otoc_nonhermitian": (_I, [_P, _I, _I, _P, _I, _I, _I, _U64, _P, C.POINTER(KrylovParams), _P, _P,
                                   C.POINTER(KrylovStats), _P]),
    "syk_batch_create": (_I, [_I, _I, _SZ, C.POINTER(KrylovParams), C.POINTER(_P)]),
    "syk_batch_destroy": (_I, [_P]),
    "syk_batch_submit": (_I, [_P, C.POINTER(OtocJob)]),
    "syk_batch_run": (_I, [_P, _I, _I, C.POINTER(_I), _P, _I]),
    "syk_batch_info": (_I, [_P, C.POINTER(_I), C.POINTER(_SZ), C.POINTER(_SZ)]),
    "syk_batch_job_bytes": (_SZ, [_P, _P, _I]),
    "syk_otoc_exact_trace_batched": (_I, [_P, _I, _P, _D, _P, _I, _I, _SZ, C.POINTER(KrylovParams), _P, _P,
                                          C.POINTER(KrylovStats)]),
    "syk_bounded_wait_selftest": (_I, [_P]),
    "syk_probe_staging": (_I, [_P, _SZ, _I, _I, C.POINTER(_D), _P]),
    "syk_probe_fp64": (_I, [C.POINTER(_D), _P]),
    "syk_probe_smem": (_I, [C.POINTER(_D), _P]),
    "syk_relabel_majoranas": (_I, [_I, _I64, _P, _P, _I, _I64, _U64, _P, _P, _P, C.POINTER(_I64), C.POINTER(_I64)]),
    "syk_tridiag_exp": (_I, [_I, _P, _P, _D, _D, _D, _I, _P, C.POINTER(_D), C.POINTER(_D), C.POINTER(_I), _P]),
    "syk_last_error": (_I, [C.c_char_p, _SZ]),
    "syk_version": (C.c_char_p, []),
}

_lib = None


def load():
    """Load libsyk.so from the package directory; fail loudly if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libsyk.so not found at {LIB_PATH}; build it with `python paper_2311_00639_b300/build.py`")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SykError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def check(rc: int):
    if rc != SYK_OK:
        buf = C.create_string_buffer(1024)
        load().syk_last_error(buf, 1024)
        raise SykError(rc, buf.value.decode(errors="replace"))
