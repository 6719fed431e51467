"""ctypes binding of include/spmv.h: the same names, argument marshalling only.

Pointers are passed as integers (device pointers from ``torch.Tensor.data_ptr()``,
host pointers from numpy's ``ctypes.data``); streams as the integer handle
``torch.cuda.Stream.cuda_stream``.  Every call raises ``SpmvError`` on a status
other than SPMV_OK, with the library's message.  The library must have been
built (``paper_1101_0091_gb300.build.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

STATUS = {0: "SPMV_OK", 1: "SPMV_ERR_ARG", 2: "SPMV_ERR_CSR", 3: "SPMV_ERR_CUDA", 4: "SPMV_ERR_OOM",
          5: "SPMV_ERR_TIMEOUT", 6: "SPMV_ERR_UNSUPPORTED", 7: "SPMV_ERR_DEVICE"}

SPMV_VARIANT_AUTO = 0
SPMV_CRS_STAGED = 1
SPMV_CRS_L1, SPMV_CRS_L2, SPMV_CRS_L4, SPMV_CRS_L8, SPMV_CRS_L16, SPMV_CRS_L32 = 2, 3, 4, 5, 6, 7
SPMV_SELL = 8
SPMV_SYM = 9
SPMV_N_VARIANTS = 10
VARIANT_NAMES = {1: "crs_staged", 2: "crs_l1", 3: "crs_l2", 4: "crs_l4", 5: "crs_l8", 6: "crs_l16",
                 7: "crs_l32", 8: "sell", 9: "sym"}


class SpmvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class spmv_options(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("sell_sigma", ctypes.c_int32), ("val_fp32", ctypes.c_int32),
                ("max_k", ctypes.c_int32), ("split", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("halo_begin", ctypes.c_int64)]


class spmv_info(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("variant", ctypes.c_int32), ("sell_sigma", ctypes.c_int32), ("sell_slots", ctypes.c_int64),
                ("sell_chunks", ctypes.c_int64), ("n_halo_rows", ctypes.c_int64), ("halo_nnz", ctypes.c_int64),
                ("n_row_blocks", ctypes.c_int64), ("tile_nnz", ctypes.c_int32), ("val_fp32", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("sym_nnz", ctypes.c_int64), ("scattered", ctypes.c_double),
                ("sell256_fill", ctypes.c_double)]


_vp, _i32, _i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
_SIGS = {
    "spmv_default_options": ([], spmv_options),
    "spmv_last_error": ([], ctypes.c_char_p),
    "spmv_create": ([ctypes.POINTER(_vp), _i64, _i64, _i64, _vp, _vp, _vp, ctypes.POINTER(spmv_options)],
                    ctypes.c_int),
    "spmv_destroy": ([_vp], ctypes.c_int),
    "spmv_apply": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "spmv_apply_block": ([_vp, _vp, _i32, _i64, _vp, _i64, _vp], ctypes.c_int),
    "spmv_apply_split": ([_vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "spmv_apply_host": ([_vp, _vp, _i32, _vp, _vp], ctypes.c_int),
    "spmv_set_variant": ([_vp, _i32, _i32], ctypes.c_int),
    "spmv_get_info": ([_vp, ctypes.POINTER(spmv_info)], ctypes.c_int),
    "spmv_check": ([_vp, _vp], ctypes.c_int),
    "spmv_sell_export": ([_vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "spmv_split_export": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "spmv_sym_export": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "spmv_select": ([_vp, _vp, _i32, _vp, _vp, _vp, _vp], ctypes.c_int),
    "spmv_autotune": ([_vp, _i32, _vp, _i64, _vp, _i64, _vp, _vp, _i32, _i32, _vp, _vp, _vp], ctypes.c_int),
    "spmv_features": ([_i64, _i64, _vp, _vp, _i32, _vp], ctypes.c_int),
    "spmv_sell_build_host": ([_i64, _i64, _vp, _vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "spmv_split_build_host": ([_i64, _i64, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
                              ctypes.c_int),
    "spmv_sym_build_host": ([_i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "spmv_probe_fp64": ([_i32, _vp, _vp, _vp, _vp], ctypes.c_int),
    "spmv_probe_gather": ([_i64, _i32, _vp, _vp, _vp], ctypes.c_int),
}


def lib_path() -> str:
    return _build.LIB


def load():
    """Load the built library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built ({path} missing): run "
                                   "paper_1101_0091_gb300.build.build() first")
            lib = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _check(st: int):
    if st != 0:
        raise SpmvError(st, load().spmv_last_error().decode())


def spmv_default_options() -> spmv_options:
    return load().spmv_default_options()


def spmv_last_error() -> str:
    return load().spmv_last_error().decode()


def spmv_create(n_rows: int, n_cols: int, nnz: int, row_ptr: int, col_idx: int, val: int,
                opt: spmv_options | None = None):
    h = ctypes.c_void_p()
    _check(load().spmv_create(ctypes.byref(h), n_rows, n_cols, nnz, row_ptr, col_idx, val,
                              ctypes.byref(opt) if opt is not None else None))
    return h


def spmv_destroy(h) -> None:
    _check(load().spmv_destroy(h))


def spmv_apply(h, B_dev: int, C_dev: int, stream: int = 0) -> None:
    _check(load().spmv_apply(h, B_dev, C_dev, stream))


def spmv_apply_block(h, B_dev: int, k: int, ldb: int, C_dev: int, ldc: int, stream: int = 0) -> None:
    _check(load().spmv_apply_block(h, B_dev, k, ldb, C_dev, ldc, stream))


def spmv_apply_split(h, B_dev: int, B_halo_pinned: int, C_dev: int, main_stream: int = 0,
                     copy_stream: int = 0) -> None:
    _check(load().spmv_apply_split(h, B_dev, B_halo_pinned, C_dev, main_stream, copy_stream))


def spmv_apply_host(h, B_host: int, k: int, C_host: int, stream: int = 0) -> None:
    _check(load().spmv_apply_host(h, B_host, k, C_host, stream))


def spmv_set_variant(h, variant: int, sell_sigma: int = 1) -> None:
    _check(load().spmv_set_variant(h, variant, sell_sigma))


def spmv_get_info(h) -> spmv_info:
    info = spmv_info()
    _check(load().spmv_get_info(h, ctypes.byref(info)))
    return info


def spmv_check(h, stream: int = 0) -> None:
    _check(load().spmv_check(h, stream))


def spmv_sell_export(h, perm: int, chunk_ptr: int, chunk_len: int, sell_col: int, sell_val: int) -> None:
    _check(load().spmv_sell_export(h, perm, chunk_ptr, chunk_len, sell_col, sell_val))


def spmv_split_export(h, loc_row_ptr, loc_col, loc_val, halo_rows, halo_row_ptr, halo_col, halo_val) -> None:
    _check(load().spmv_split_export(h, loc_row_ptr, loc_col, loc_val, halo_rows, halo_row_ptr, halo_col, halo_val))


def spmv_sym_export(h, row_ptr: int, col: int, val: int) -> None:
    _check(load().spmv_sym_export(h, row_ptr, col, val))


def spmv_features(n_rows: int, n_cols: int, row_ptr: int, col_idx: int, k: int, out: int) -> None:
    _check(load().spmv_features(n_rows, n_cols, row_ptr, col_idx, k, out))


def spmv_sell_build_host(n_rows, n_cols, row_ptr, col_idx, val, sigma, n_chunks, n_slots, perm, chunk_ptr,
                         chunk_len, sell_col, sell_val) -> None:
    _check(load().spmv_sell_build_host(n_rows, n_cols, row_ptr, col_idx, val, sigma, n_chunks, n_slots, perm,
                                       chunk_ptr, chunk_len, sell_col, sell_val))


def spmv_split_build_host(n_rows, n_cols, row_ptr, col_idx, val, h, loc_nnz, n_halo_rows, halo_nnz, loc_row_ptr,
                          loc_col, loc_val, halo_rows, halo_row_ptr, halo_col, halo_val) -> None:
    _check(load().spmv_split_build_host(n_rows, n_cols, row_ptr, col_idx, val, h, loc_nnz, n_halo_rows, halo_nnz,
                                        loc_row_ptr, loc_col, loc_val, halo_rows, halo_row_ptr, halo_col, halo_val))


def spmv_sym_build_host(n_rows, n_cols, row_ptr, col_idx, val, sym_nnz, sym_row_ptr, sym_col, sym_val) -> None:
    _check(load().spmv_sym_build_host(n_rows, n_cols, row_ptr, col_idx, val, sym_nnz, sym_row_ptr, sym_col,
                                      sym_val))


class spmv_tuning(ctypes.Structure):
    _fields_ = [("prefetch_distance", ctypes.c_int32), ("reserved", ctypes.c_int32 * 7)]


_SIGS["spmv_set_tuning"] = ([_vp, ctypes.POINTER(spmv_tuning)], ctypes.c_int)
_SIGS["spmv_get_tuning"] = ([_vp, ctypes.POINTER(spmv_tuning)], ctypes.c_int)


def spmv_set_tuning(h, t: spmv_tuning) -> None:
    _check(load().spmv_set_tuning(h, ctypes.byref(t)))


def spmv_get_tuning(h) -> spmv_tuning:
    t = spmv_tuning()
    _check(load().spmv_get_tuning(h, ctypes.byref(t)))
    return t


_SIGS["spmv_apply_host_async"] = ([_vp, _vp, _i32, _vp, _vp], ctypes.c_int)
_SIGS["spmv_host_sync"] = ([_vp], ctypes.c_int)


def spmv_apply_host_async(h, B_host: int, k: int, C_host: int, stream: int = 0) -> None:
    _check(load().spmv_apply_host_async(h, B_host, k, C_host, stream))


def spmv_host_sync(h) -> None:
    _check(load().spmv_host_sync(h))


_SIGS["spmv_wait"] = ([_vp, _i32], ctypes.c_int)
_SIGS["spmv_selftest_wait_timeout"] = ([_i32], ctypes.c_int)


def spmv_wait(stream: int, timeout_ms: int) -> None:
    _check(load().spmv_wait(stream, timeout_ms))


def spmv_selftest_wait_timeout(limit_us: int) -> None:
    _check(load().spmv_selftest_wait_timeout(limit_us))


def spmv_probe_fp64(reps: int = 5) -> dict:
    """FP64 FMA rate of the current device (spmv_probe_fp64)."""
    g, ms, sms, mhz = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32(), ctypes.c_double()
    _check(load().spmv_probe_fp64(reps, ctypes.byref(g), ctypes.byref(ms), ctypes.byref(sms), ctypes.byref(mhz)))
    return {"gflops": g.value, "ms": ms.value, "sm_count": sms.value, "sm_mhz": mhz.value,
            "fma_per_clock_per_sm": g.value * 1e3 / (2 * sms.value * mhz.value) if mhz.value > 0 else None}


def spmv_probe_gather(n_elems: int, reps: int = 5) -> dict:
    """Random 8-byte read rate out of a buffer of n_elems doubles (spmv_probe_gather)."""
    r, ms, mhz = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().spmv_probe_gather(n_elems, reps, ctypes.byref(r), ctypes.byref(ms), ctypes.byref(mhz)))
    return {"gathers_per_s": r.value, "ms": ms.value, "sm_mhz": mhz.value}
