"""Sparse-SYK OTOC hot path on B300 (sm_103a): a thin binding of libsyk.

The compute path is the CUDA library ``libsyk.so`` (sources in ``csrc/``,
C-ABI in ``include/syk.h``); importing this package loads it and fails loudly
if it has not been built (``python paper_2311_00639_b300/build.py``).  There
is no CPU fallback.
"""
from ._lib import LIB_PATH, SykError, load
from .api import (Batch, KrylovStats, autotune_batch, PauliTerms, Terms, bounded_wait_selftest, compile_chi_host, compile_pauli_host,
                  compile_terms_complex_host, compile_terms_host, exact_trace_otoc, plan_host, plan_strings_host,
                  probe_fp64, probe_smem, probe_staging, relabel_for_locality, tridiag_exp)

load()

__all__ = ["Terms", "PauliTerms", "compile_pauli_host", "compile_terms_complex_host", "Batch", "autotune_batch", "exact_trace_otoc", "bounded_wait_selftest", "KrylovStats", "SykError", "compile_terms_host", "compile_chi_host", "plan_host", "plan_strings_host", "probe_staging", "probe_smem", "probe_fp64", "tridiag_exp", "relabel_for_locality", "LIB_PATH", "load"]
