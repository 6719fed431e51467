"""ctypes binding of the batched entry points of include/spmv.h (same names,
argument marshalling only)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _binding as _b
from ._binding import _check, _i32, _i64, _vp, load

SPMV_BATCH_L1, SPMV_BATCH_L2, SPMV_BATCH_L4, SPMV_BATCH_L8, SPMV_BATCH_L32, SPMV_BATCH_ADAPT, SPMV_BATCH_SORTED = range(7)
SPMV_BATCH_N_POLICIES = 7
POLICY_NAMES = {0: "l1", 1: "l2", 2: "l4", 3: "l8", 4: "l32", 5: "adapt", 6: "sorted"}
AUTOTUNE_GRID = [(item, sched, ctas) for item in (256, 512, 1024, 2048, 4096) for sched in (0, 1) for ctas in (4, 7)]


class spmv_batch_config(ctypes.Structure):
    _fields_ = [("item_nnz", ctypes.c_int32), ("schedule", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


_P = ctypes.POINTER
_SIGS = {
    "spmv_batch_default_config": ([], spmv_batch_config),
    "spmv_batch_create": ([_P(_vp), _i32, _vp, _i32, _vp, _P(spmv_batch_config)], ctypes.c_int),
    "spmv_batch_set_io": ([_vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "spmv_batch_apply": ([_vp, _vp], ctypes.c_int),
    "spmv_batch_apply_host": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "spmv_batch_apply_host_async": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "spmv_batch_host_sync": ([_vp], ctypes.c_int),
    "spmv_batch_apply_separate": ([_vp, _vp], ctypes.c_int),
    "spmv_batch_set_config": ([_vp, _P(spmv_batch_config)], ctypes.c_int),
    "spmv_batch_get_config": ([_vp, _P(spmv_batch_config)], ctypes.c_int),
    "spmv_batch_set_policies": ([_vp, _vp], ctypes.c_int),
    "spmv_batch_autotune": ([_vp, _vp, _i32, _P(spmv_batch_config), _vp], ctypes.c_int),
    "spmv_batch_info": ([_vp, _P(_i64), _P(_i64), _P(_i64)], ctypes.c_int),
    "spmv_batch_destroy": ([_vp], ctypes.c_int),
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


def spmv_batch_default_config() -> spmv_batch_config:
    return _lib().spmv_batch_default_config()


def spmv_batch_create(plans, k: int, policies=None, cfg: spmv_batch_config | None = None):
    arr = (ctypes.c_void_p * len(plans))(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    pol = None
    if policies is not None:
        pol = np.ascontiguousarray(policies, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(_lib().spmv_batch_create(ctypes.byref(h), len(plans), ctypes.cast(arr, ctypes.c_void_p), k,
                                    pol.ctypes.data if pol is not None else None,
                                    ctypes.byref(cfg) if cfg is not None else None))
    return h


def spmv_batch_set_io(b, B_ptrs, ldb, C_ptrs, ldc) -> None:
    n = len(B_ptrs)
    Bp = (ctypes.c_void_p * n)(*B_ptrs)
    Cp = (ctypes.c_void_p * n)(*C_ptrs)
    lb = np.ascontiguousarray(ldb, dtype=np.int64) if ldb is not None else None
    lc = np.ascontiguousarray(ldc, dtype=np.int64) if ldc is not None else None
    _check(_lib().spmv_batch_set_io(b, ctypes.cast(Bp, ctypes.c_void_p), lb.ctypes.data if lb is not None else None,
                                    ctypes.cast(Cp, ctypes.c_void_p), lc.ctypes.data if lc is not None else None))


def spmv_batch_apply(b, stream: int = 0) -> None:
    _check(_lib().spmv_batch_apply(b, stream))


def spmv_batch_apply_separate(b, stream: int = 0) -> None:
    _check(_lib().spmv_batch_apply_separate(b, stream))


def spmv_batch_set_config(b, cfg: spmv_batch_config) -> None:
    _check(_lib().spmv_batch_set_config(b, ctypes.byref(cfg)))


def spmv_batch_get_config(b) -> spmv_batch_config:
    c = spmv_batch_config()
    _check(_lib().spmv_batch_get_config(b, ctypes.byref(c)))
    return c


def spmv_batch_set_policies(b, policies) -> None:
    pol = np.ascontiguousarray(policies, dtype=np.int32)
    _check(_lib().spmv_batch_set_policies(b, pol.ctypes.data))


def spmv_batch_autotune(b, stream: int = 0, reps: int = 5):
    best = spmv_batch_config()
    times = np.zeros(len(AUTOTUNE_GRID), dtype=np.float32)
    _check(_lib().spmv_batch_autotune(b, stream, reps, ctypes.byref(best), times.ctypes.data))
    return best, times


def spmv_batch_info(b):
    n, r, z = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib().spmv_batch_info(b, ctypes.byref(n), ctypes.byref(r), ctypes.byref(z)))
    return n.value, r.value, z.value


def spmv_batch_destroy(b) -> None:
    _check(_lib().spmv_batch_destroy(b))


def _host_ptr(a) -> int:
    return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data


def spmv_batch_apply_host(b, B_host_ptrs, C_host_ptrs, stream) -> None:
    n = len(B_host_ptrs)
    bp = (ctypes.c_void_p * n)(*B_host_ptrs)
    cp = (ctypes.c_void_p * n)(*C_host_ptrs)
    _check(_lib().spmv_batch_apply_host(b, bp, cp, stream))


def spmv_batch_apply_host_async(b, B_host_ptrs, C_host_ptrs, stream) -> None:
    n = len(B_host_ptrs)
    bp = (ctypes.c_void_p * n)(*B_host_ptrs)
    cp = (ctypes.c_void_p * n)(*C_host_ptrs)
    _check(_lib().spmv_batch_apply_host_async(b, bp, cp, stream))


def spmv_batch_host_sync(b) -> None:
    _check(_lib().spmv_batch_host_sync(b))


class Batch:
    """Owns one spmv_batch_handle over existing Plans (which must outlive it)."""

    def __init__(self, plans, k: int, policies=None, cfg: spmv_batch_config | None = None):
        self.plans = list(plans)
        self.k = k
        self.handle = spmv_batch_create([p.handle for p in self.plans], k, policies, cfg)

    def set_io(self, Bs, Cs) -> None:
        """Bs[m]: (n_cols_m, ldb) and Cs[m]: (n_rows_m, ldc) row-major CUDA float64 tensors."""
        spmv_batch_set_io(self.handle, [B.data_ptr() for B in Bs], [B.stride(0) for B in Bs],
                          [C.data_ptr() for C in Cs], [C.stride(0) for C in Cs])
        self._io = (Bs, Cs)

    def apply(self, stream=None) -> None:
        from . import _stream_handle
        spmv_batch_apply(self.handle, _stream_handle(stream))

    def apply_host(self, B_host, C_host, stream=None) -> None:
        """spmv_batch_apply_host: B_host[m] / C_host[m] are host float64 arrays or
        (pinned) CPU tensors of each member's block (ld = k); asynchronous."""
        from . import _stream_handle
        spmv_batch_apply_host(self.handle, [_host_ptr(b) for b in B_host], [_host_ptr(c) for c in C_host],
                              _stream_handle(stream))

    def apply_host_async(self, B_host, C_host, stream=None) -> None:
        """spmv_batch_apply_host_async: one pipelined step from page-locked host
        blocks (ld = k); the buffers must stay valid until host_sync()."""
        from . import _stream_handle
        spmv_batch_apply_host_async(self.handle, [_host_ptr(b) for b in B_host], [_host_ptr(c) for c in C_host],
                                    _stream_handle(stream))

    def host_sync(self) -> None:
        spmv_batch_host_sync(self.handle)

    def apply_separate(self, stream=None) -> None:
        from . import _stream_handle
        spmv_batch_apply_separate(self.handle, _stream_handle(stream))

    def set_config(self, item_nnz=None, schedule=None, ctas_per_sm=None) -> None:
        c = spmv_batch_get_config(self.handle)
        if item_nnz is not None:
            c.item_nnz = item_nnz
        if schedule is not None:
            c.schedule = schedule
        if ctas_per_sm is not None:
            c.ctas_per_sm = ctas_per_sm
        spmv_batch_set_config(self.handle, c)

    def config(self) -> spmv_batch_config:
        return spmv_batch_get_config(self.handle)

    def set_policies(self, policies) -> None:
        spmv_batch_set_policies(self.handle, policies)

    def autotune(self, stream=None, reps: int = 5):
        from . import _stream_handle
        return spmv_batch_autotune(self.handle, _stream_handle(stream), reps)

    def info(self):
        return spmv_batch_info(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None) is not None:
            spmv_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


_SIGS["spmv_batch_apply_noalloc"] = ([_i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp], ctypes.c_int)


def spmv_batch_apply_noalloc(n_rows, row_ptr_dev, col_dev, val_dev, B_dev, ldb, C_dev, ldc, k: int,
                             lanes=None, stream: int = 0) -> None:
    """Per-member lists (host side) of row counts and DEVICE pointers; marshalled into host arrays."""
    n = len(n_rows)
    rows = np.ascontiguousarray(n_rows, dtype=np.int64)
    ptrs = [(ctypes.c_void_p * n)(*p) for p in (row_ptr_dev, col_dev, val_dev, B_dev, C_dev)]
    lb = np.ascontiguousarray(ldb, dtype=np.int64) if ldb is not None else None
    lc = np.ascontiguousarray(ldc, dtype=np.int64) if ldc is not None else None
    ln = np.ascontiguousarray(lanes, dtype=np.int32) if lanes is not None else None
    c = lambda a: ctypes.cast(a, ctypes.c_void_p)  # noqa: E731
    _check(_lib().spmv_batch_apply_noalloc(
        n, rows.ctypes.data, c(ptrs[0]), c(ptrs[1]), c(ptrs[2]), c(ptrs[3]),
        lb.ctypes.data if lb is not None else None, c(ptrs[4]), lc.ctypes.data if lc is not None else None, k,
        ln.ctypes.data if ln is not None else None, stream))
