"""ctypes binding of the plain C++/OpenMP CPU baseline (cpu_baseline.cpp).

TEST INFRASTRUCTURE ONLY (see the package docstring): the benchmark's timed
CPU baseline and a cross-check of the Python oracle.  build() compiles the
shared library next to its source with g++ -O3 -fopenmp (no CUDA).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_baseline.cpp")
LIB = os.path.join(HERE, "libsyk_cpu.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cxx = os.environ.get("CXX", "g++")
        subprocess.run([cxx, "-O3", "-fopenmp", "-std=c++17", "-shared", "-fPIC", SRC, "-o", LIB + ".tmp"],
                       check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.c_void_p
        lib.cpu_threads.restype = C.c_int
        lib.cpu_hpsi.argtypes = [C.c_int, C.c_int64, P, P, C.c_int, P, P]
        lib.cpu_hpsi_rows.argtypes = [C.c_int, C.c_int64, P, P, C.c_int, C.c_uint64, C.c_int, P, P, P]
        lib.cpu_krylov_evolve.argtypes = [C.c_int, C.c_int64, P, P, C.c_int, C.c_double, C.c_double, C.c_int,
                                          C.c_double, P, P]
        lib.cpu_krylov_evolve.restype = C.c_int64
        _lib = lib
    return _lib


def _terms(quads, J):
    q = np.ascontiguousarray(np.asarray(quads, dtype=np.int32).reshape(-1, 4))
    j = np.ascontiguousarray(np.asarray(J, dtype=np.float64).reshape(-1))
    return q, j


def threads() -> int:
    return int(load().cpu_threads())


def hpsi(N: int, quads, J, block: int, psi) -> np.ndarray:
    """H_BB psi on the whole block (complex128)."""
    q, j = _terms(quads, J)
    x = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(x)
    rc = load().cpu_hpsi(N, len(j), q.ctypes.data, j.ctypes.data, block, x.ctypes.data, out.ctypes.data)
    if rc:
        raise ValueError(f"cpu_hpsi failed ({rc})")
    return out


def row_sample_starts(N: int, quads, J, block: int, row0: int, log2R: int) -> np.ndarray:
    """Start of the aligned input range of 2^log2R amplitudes each term reads
    for the output rows [row0, row0 + 2^log2R)."""
    q, j = _terms(quads, J)
    starts = np.zeros(len(j), dtype=np.uint64)
    rc = load().cpu_hpsi_rows(N, len(j), q.ctypes.data, j.ctypes.data, block, row0, log2R, None,
                              starts.ctypes.data, None)
    if rc:
        raise ValueError(f"cpu_hpsi_rows failed ({rc})")
    return starts


def hpsi_rows(N: int, quads, J, block: int, row0: int, log2R: int, in_blocks) -> np.ndarray:
    """Rows [row0, row0 + 2^log2R) of H_BB psi; in_blocks[t] = psi on the
    range row_sample_starts(...)[t] (complex128 arrays of 2^log2R)."""
    q, j = _terms(quads, J)
    arrs = [np.ascontiguousarray(b, dtype=np.complex128) for b in in_blocks]
    ptrs = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    out = np.empty(1 << log2R, dtype=np.complex128)
    rc = load().cpu_hpsi_rows(N, len(j), q.ctypes.data, j.ctypes.data, block, row0, log2R, ptrs, None,
                              out.ctypes.data)
    if rc:
        raise ValueError(f"cpu_hpsi_rows failed ({rc})")
    return out


def krylov_evolve(N: int, quads, J, block: int, z, x, m: int = 30, tol: float = 1e-12):
    """(e^{-zH_BB} x, matvecs) by the CPU Lanczos baseline."""
    q, j = _terms(quads, J)
    xi = np.ascontiguousarray(x, dtype=np.complex128)
    y = np.empty_like(xi)
    z = complex(z)
    mv = load().cpu_krylov_evolve(N, len(j), q.ctypes.data, j.ctypes.data, block, z.real, z.imag, m, tol,
                                  xi.ctypes.data, y.ctypes.data)
    if mv < 0:
        raise ValueError(f"cpu_krylov_evolve failed ({mv})")
    return y, int(mv)
