"""CPU node baseline for bench.py: the paper's OpenMP row-parallel CRS loop
(Sec. 2) on all host cores.  Not part of the library (which has no CPU path)
and not the oracle."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "crs_omp.c")
_LIB = os.path.join(_HERE, "_build", "libcrs_omp.so")
_lib = None


def build(force: bool = False) -> str | None:
    """Compile with gcc -fopenmp; returns None where OpenMP is not available."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        try:
            subprocess.check_call(["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                                   "-fno-fast-math", "-o", tmp, _SRC])
        except (OSError, subprocess.CalledProcessError):
            return None
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        path = build()
        if path is None:
            return None
        lib = ctypes.CDLL(path)
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        lib.crs_omp_spmv.argtypes = [i64, vp, vp, vp, vp, vp]
        lib.crs_omp_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def available() -> bool:
    return _load() is not None


def threads() -> int:
    return _load().crs_omp_threads()


def spmv(A, B) -> np.ndarray:
    lib = _load()
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
    va = np.ascontiguousarray(A.val, dtype=np.float64)
    Bc = np.ascontiguousarray(B, dtype=np.float64)
    C = np.empty(A.n_rows, dtype=np.float64)
    lib.crs_omp_spmv(A.n_rows, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, Bc.ctypes.data, C.ctypes.data)
    return C
