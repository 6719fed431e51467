"""ORACLE — test infrastructure only.

A plain, slow, obviously correct CPU reference for everything the GPU path
computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the library in ``paper_1101_0091_gb300`` never
does, and it shares no code with that library.

* ``oracle.c`` (FP64, single thread, -ffp-contract=off): the CRS loop of
  Sec. 1.2, its k-RHS and FP32-value forms, the tolerance scale sum |a*b|, the
  SELL-C-sigma builder and product, the local/halo split builder and
  product of Sec. 3.1, and the symmetric-CRS test, upper-triangle builder and
  product of Sec. 1.3.1.
* ``features.py`` (numpy): matrix features that feed the cost model.
* ``mlp.py`` (numpy FP64): the cost model's forward, backward and Adam step.

Pins (what ties each function to something other than itself) are in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c: plain gcc, -O2, no FMA contraction, no fast-math."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, vp = ctypes.c_int64, ctypes.c_void_p
            lib.oracle_crs_spmv.argtypes = [i64, vp, vp, vp, vp, vp]
            lib.oracle_crs_spmm.argtypes = [i64, i64, vp, vp, vp, vp, i64, vp, i64]
            lib.oracle_crs_spmm_f32val.argtypes = [i64, i64, vp, vp, vp, vp, i64, vp, i64]
            lib.oracle_abs_scale.argtypes = [i64, i64, vp, vp, vp, vp, i64, vp, i64]
            lib.oracle_crs_spmm_dot2.argtypes = [i64, i64, vp, vp, vp, vp, i64, vp, i64]
            lib.oracle_sell_perm.argtypes = [i64, vp, i64, i64, vp, ctypes.POINTER(i64)]
            lib.oracle_sell_perm.restype = i64
            lib.oracle_sell_fill.argtypes = [i64, vp, vp, vp, i64, vp, i64, vp, vp, vp, vp]
            lib.oracle_sell_spmv.argtypes = [i64, i64, vp, i64, vp, vp, vp, vp, vp, vp]
            lib.oracle_split_count.argtypes = [i64, vp, vp, i64, ctypes.POINTER(i64)]
            lib.oracle_split_count.restype = i64
            lib.oracle_split_fill.argtypes = [i64, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp]
            lib.oracle_split_spmv.argtypes = [i64, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp]
            lib.oracle_is_symmetric.argtypes = [i64, i64, vp, vp, vp]
            lib.oracle_is_symmetric.restype = ctypes.c_int
            lib.oracle_sym_count.argtypes = [i64, vp, vp]
            lib.oracle_sym_count.restype = i64
            lib.oracle_sym_fill.argtypes = [i64, vp, vp, vp, vp, vp, vp]
            lib.oracle_sym_spmv.argtypes = [i64, vp, vp, vp, vp, vp]
            _lib = lib
    return _lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def _csr(A):
    rp, p_rp = _c(A.row_ptr, np.int32)
    ci, p_ci = _c(A.col_idx, np.int32)
    va, p_va = _c(A.val, np.float64)
    return (rp, ci, va), (p_rp, p_ci, p_va)


def spmv(A, B) -> np.ndarray:
    """C = A*B by the CRS loop (Sec. 1.2), FP64, rows in order, j ascending."""
    keep, (rp, ci, va) = _csr(A)
    Bc, pB = _c(B, np.float64)
    assert Bc.shape[0] >= A.n_cols
    C = np.empty(A.n_rows, dtype=np.float64)
    _load().oracle_crs_spmv(A.n_rows, rp, ci, va, pB, C.ctypes.data)
    return C


def spmm(A, B, f32val: bool = False) -> np.ndarray:
    """C = A*B for a row-major block B (n_cols x k); f32val rounds val to float first."""
    keep, (rp, ci, va) = _csr(A)
    Bc, pB = _c(B, np.float64)
    if Bc.ndim == 1:
        Bc = Bc.reshape(-1, 1)
    n_cols, k = Bc.shape
    assert n_cols >= A.n_cols
    C = np.empty((A.n_rows, k), dtype=np.float64)
    fn = _load().oracle_crs_spmm_f32val if f32val else _load().oracle_crs_spmm
    fn(A.n_rows, k, rp, ci, va, pB, k, C.ctypes.data, k)
    return C


def spmm_dot2(A, B) -> np.ndarray:
    """Row sums of A*B as if computed in twice the working precision (compensated
    dot product, Ogita-Rump-Oishi Dot2); for attributing a failed parity check,
    not a reference of the checks themselves."""
    keep, (rp, ci, va) = _csr(A)
    Bc, pB = _c(B, np.float64)
    Bc2 = Bc.reshape(Bc.shape[0], -1)
    k = Bc2.shape[1]
    C = np.empty((A.n_rows, k), dtype=np.float64)
    _load().oracle_crs_spmm_dot2(A.n_rows, k, rp, ci, va, pB, k, C.ctypes.data, k)
    return C if Bc.ndim > 1 else C[:, 0]


def abs_scale(A, B) -> np.ndarray:
    """S[i, c] = sum_j |a_ij * b_jc| (the per-row error scale of the tolerance)."""
    keep, (rp, ci, va) = _csr(A)
    Bc, pB = _c(B, np.float64)
    Bc2 = Bc.reshape(Bc.shape[0], -1)
    k = Bc2.shape[1]
    S = np.empty((A.n_rows, k), dtype=np.float64)
    _load().oracle_abs_scale(A.n_rows, k, rp, ci, va, pB, k, S.ctypes.data, k)
    return S if Bc.ndim > 1 else S[:, 0]


class Sell:
    """SELL-C-sigma arrays: perm[n_rows], chunk_ptr[n_chunks+1] (int64),
    chunk_len[n_chunks], sell_col / sell_val [chunk_ptr[-1]]."""

    def __init__(self, n_rows, C, sigma, perm, chunk_ptr, chunk_len, sell_col, sell_val, nnz):
        self.n_rows, self.C, self.sigma = n_rows, C, sigma
        self.perm, self.chunk_ptr, self.chunk_len = perm, chunk_ptr, chunk_len
        self.sell_col, self.sell_val = sell_col, sell_val
        self.nnz = nnz

    @property
    def n_chunks(self) -> int:
        return len(self.chunk_len)

    @property
    def beta(self) -> float:
        """Fill efficiency: nonzeros / stored slots (1.0 when nothing is stored)."""
        stored = int(self.chunk_ptr[-1])
        return self.nnz / stored if stored else 1.0


def sell_build(A, C: int = 32, sigma: int = 1) -> Sell:
    """Build SELL-C-sigma from CRS (stable descending sort per sigma-window)."""
    lib = _load()
    keep, (rp, ci, va) = _csr(A)
    perm = np.empty(A.n_rows, dtype=np.int32)
    nch = ctypes.c_int64(0)
    total = lib.oracle_sell_perm(A.n_rows, rp, C, sigma, perm.ctypes.data, ctypes.byref(nch))
    nc = nch.value
    chunk_ptr = np.empty(nc + 1, dtype=np.int64)
    chunk_len = np.empty(nc, dtype=np.int32)
    scol = np.empty(total, dtype=np.int32)
    sval = np.empty(total, dtype=np.float64)
    lib.oracle_sell_fill(A.n_rows, rp, ci, va, C, perm.ctypes.data, nc, chunk_ptr.ctypes.data,
                         chunk_len.ctypes.data, scol.ctypes.data, sval.ctypes.data)
    return Sell(A.n_rows, C, sigma, perm, chunk_ptr, chunk_len, scol, sval, A.nnz)


def sell_spmv(S: Sell, B) -> np.ndarray:
    """SELL product by the definition of the format (padding included)."""
    Bc, pB = _c(B, np.float64)
    out = np.zeros(S.n_rows, dtype=np.float64)
    _load().oracle_sell_spmv(S.n_rows, S.C, S.perm.ctypes.data, S.n_chunks, S.chunk_ptr.ctypes.data,
                             S.chunk_len.ctypes.data, S.sell_col.ctypes.data, S.sell_val.ctypes.data,
                             pB, out.ctypes.data)
    return out


class Split:
    """Local/halo split: local CRS over all rows (col < h); halo CRS over halo_rows (col >= h)."""

    def __init__(self, h, loc_row_ptr, loc_col, loc_val, halo_rows, halo_row_ptr, halo_col, halo_val):
        self.h = h
        self.loc_row_ptr, self.loc_col, self.loc_val = loc_row_ptr, loc_col, loc_val
        self.halo_rows, self.halo_row_ptr = halo_rows, halo_row_ptr
        self.halo_col, self.halo_val = halo_col, halo_val


def split_build(A, h: int) -> Split:
    lib = _load()
    keep, (rp, ci, va) = _csr(A)
    nhr = ctypes.c_int64(0)
    nh = lib.oracle_split_count(A.n_rows, rp, ci, h, ctypes.byref(nhr))
    nl = A.nnz - nh
    out = Split(h, np.empty(A.n_rows + 1, np.int32), np.empty(nl, np.int32), np.empty(nl, np.float64),
                np.empty(nhr.value, np.int32), np.empty(nhr.value + 1, np.int32),
                np.empty(nh, np.int32), np.empty(nh, np.float64))
    lib.oracle_split_fill(A.n_rows, rp, ci, va, h, out.loc_row_ptr.ctypes.data, out.loc_col.ctypes.data,
                          out.loc_val.ctypes.data, out.halo_rows.ctypes.data, out.halo_row_ptr.ctypes.data,
                          out.halo_col.ctypes.data, out.halo_val.ctypes.data)
    return out


def split_spmv(A_rows: int, S: Split, B) -> np.ndarray:
    """Local product writes C, then the halo product is added (Sec. 3.1)."""
    Bc, pB = _c(B, np.float64)
    C = np.empty(A_rows, dtype=np.float64)
    _load().oracle_split_spmv(A_rows, S.loc_row_ptr.ctypes.data, S.loc_col.ctypes.data,
                              S.loc_val.ctypes.data, len(S.halo_rows), S.halo_rows.ctypes.data,
                              S.halo_row_ptr.ctypes.data, S.halo_col.ctypes.data,
                              S.halo_val.ctypes.data, pB, C.ctypes.data)
    return C


class Sym:
    """Symmetric CRS: the entries on and above the diagonal of each row, in
    their order in the row (row_ptr[n_rows+1], col[nnz_u], val[nnz_u])."""

    def __init__(self, n_rows, row_ptr, col, val):
        self.n_rows, self.row_ptr, self.col, self.val = n_rows, row_ptr, col, val

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def is_symmetric(A) -> bool:
    """Square, and every strictly-upper entry (i, j, v) mirrored one to one by a
    strictly-lower entry (j, i, v) (values compared with -0.0 == +0.0)."""
    keep, (rp, ci, va) = _csr(A)
    r = _load().oracle_is_symmetric(A.n_rows, A.n_cols, rp, ci, va)
    if r < 0:
        raise MemoryError("oracle_is_symmetric: scratch allocation failed")
    return bool(r)


def sym_build(A) -> Sym:
    """Upper triangle (diagonal included) of a symmetric CRS matrix (Sec. 1.3.1)."""
    lib = _load()
    keep, (rp, ci, va) = _csr(A)
    n = lib.oracle_sym_count(A.n_rows, rp, ci)
    S = Sym(A.n_rows, np.empty(A.n_rows + 1, np.int32), np.empty(n, np.int32), np.empty(n, np.float64))
    lib.oracle_sym_fill(A.n_rows, rp, ci, va, S.row_ptr.ctypes.data, S.col.ctypes.data, S.val.ctypes.data)
    return S


def sym_spmv(S: Sym, B) -> np.ndarray:
    """C = A*B from the stored triangle: each stored u_ij adds u_ij*B_j to C_i
    and, off the diagonal, u_ij*B_i to C_j; rows in order."""
    Bc, pB = _c(B, np.float64)
    assert Bc.shape[0] >= S.n_rows
    C = np.empty(S.n_rows, dtype=np.float64)
    _load().oracle_sym_spmv(S.n_rows, S.row_ptr.ctypes.data, S.col.ctypes.data, S.val.ctypes.data, pB,
                            C.ctypes.data)
    return C


def max_err_ratio(y, ref, scale, tol: float) -> float:
    """max over entries of |y - ref| / (tol * scale); <= 1 passes.  A zero scale
    demands exact equality (returns inf on any difference)."""
    y = np.asarray(y, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.asarray(scale, dtype=np.float64)
    diff = np.abs(y - ref)
    bound = tol * scale
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(bound > 0, diff / np.where(bound > 0, bound, 1.0), np.where(diff > 0, np.inf, 0.0))
    return float(r.max()) if r.size else 0.0
