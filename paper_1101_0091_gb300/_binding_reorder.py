"""ctypes binding of the reordering entry points of include/spmv.h (same
names, argument marshalling only), with numpy/torch conveniences."""
from __future__ import annotations

import ctypes

import numpy as np

from ._binding import _check, _i32, _i64, _vp, load

_P = ctypes.POINTER
_SIGS = {
    "spmv_rcm": ([_i64, _vp, _vp, _vp], ctypes.c_int),
    "spmv_permute_csr": ([_i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "spmv_reorder_create": ([_i64, _vp, _P(_vp)], ctypes.c_int),
    "spmv_reorder_gather": ([_vp, _i32, _vp, _i64, _vp, _i64, _vp], ctypes.c_int),
    "spmv_reorder_scatter": ([_vp, _i32, _vp, _i64, _vp, _i64, _vp], ctypes.c_int),
    "spmv_reorder_destroy": ([_vp], ctypes.c_int),
}
_done = False


def _lib():
    global _done
    lib = load()
    if not _done:
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _done = True
    return lib


def _i32a(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def rcm(n: int, row_ptr, col_idx) -> np.ndarray:
    """RCM permutation (perm[new] = old) of a square CRS pattern (host)."""
    rp, ci = _i32a(row_ptr), _i32a(col_idx)
    perm = np.empty(n, np.int32)
    _check(_lib().spmv_rcm(n, rp.ctypes.data, ci.ctypes.data, perm.ctypes.data))
    return perm


def permute_csr(n: int, row_ptr, col_idx, val, perm):
    """Arrays (row_ptr, col_idx, val) of P A P^T (host)."""
    rp, ci, pm = _i32a(row_ptr), _i32a(col_idx), _i32a(perm)
    va = np.ascontiguousarray(val, dtype=np.float64)
    nnz = int(rp[-1]) if n > 0 else 0
    orp = np.empty(n + 1, np.int32)
    oci = np.empty(nnz, np.int32)
    ova = np.empty(nnz, np.float64)
    _check(_lib().spmv_permute_csr(n, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, pm.ctypes.data,
                                   orp.ctypes.data, oci.ctypes.data, ova.ctypes.data))
    return orp, oci, ova


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


class Reorder:
    """A permutation on the device: gather (original -> permuted row order)
    and scatter (permuted -> original) of (n, k) torch blocks."""

    def __init__(self, perm):
        pm = _i32a(perm)
        self.n = len(pm)
        h = ctypes.c_void_p()
        _check(_lib().spmv_reorder_create(self.n, pm.ctypes.data, ctypes.byref(h)))
        self.handle = h

    @staticmethod
    def _k_ld(t):
        return (1, 1) if t.dim() == 1 else (t.shape[1], t.stride(0))

    def gather(self, X, Y, stream=None) -> None:
        k, ldx = self._k_ld(X)
        _, ldy = self._k_ld(Y)
        _check(_lib().spmv_reorder_gather(self.handle, k, X.data_ptr(), ldx, Y.data_ptr(), ldy, _stream(stream)))

    def scatter(self, X, Y, stream=None) -> None:
        k, ldx = self._k_ld(X)
        _, ldy = self._k_ld(Y)
        _check(_lib().spmv_reorder_scatter(self.handle, k, X.data_ptr(), ldx, Y.data_ptr(), ldy, _stream(stream)))

    def close(self) -> None:
        if getattr(self, "handle", None) is not None:
            _check(_lib().spmv_reorder_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
