"""GB300 (sm_103a) CRS sparse matrix-vector multiply C = A*B.

The compute path is the C ABI library built from ``csrc/`` (see
``include/spmv.h``); this package only marshals arguments into it.  PyTorch is
used by callers for device memory and streams; nothing here computes on the
host.

    from paper_1101_0091_gb300 import Plan
    plan = Plan(n_rows, n_cols, row_ptr, col_idx, val)     # host numpy arrays
    plan.apply(B, C)                                       # torch CUDA float64 tensors
"""
from __future__ import annotations

import numpy as np

from . import _binding as _b
from ._binding import spmv_apply_host_async, spmv_host_sync, spmv_selftest_wait_timeout, spmv_wait  # noqa: F401
from ._binding import spmv_probe_fp64, spmv_probe_gather  # noqa: F401
from ._binding import (SpmvError, VARIANT_NAMES, load, spmv_apply, spmv_apply_block, spmv_apply_host,  # noqa: F401
                       spmv_apply_split, spmv_check, spmv_create, spmv_default_options, spmv_destroy,
                       spmv_get_info, spmv_last_error, spmv_options, spmv_sell_export, spmv_set_variant,
                       spmv_split_export, spmv_sym_export, spmv_features, spmv_set_tuning, spmv_get_tuning,
                       spmv_tuning, SPMV_VARIANT_AUTO, SPMV_CRS_STAGED, SPMV_CRS_L1, SPMV_CRS_L2,
                       SPMV_CRS_L4, SPMV_CRS_L8, SPMV_CRS_L16, SPMV_CRS_L32, SPMV_SELL, SPMV_SYM,
                       SPMV_N_VARIANTS, spmv_sell_build_host, spmv_split_build_host, spmv_sym_build_host)

from ._binding_batch import (AUTOTUNE_GRID, POLICY_NAMES, SPMV_BATCH_ADAPT, SPMV_BATCH_L1,  # noqa: F401,E402
                             SPMV_BATCH_L2, SPMV_BATCH_L4, SPMV_BATCH_L8, SPMV_BATCH_L32, SPMV_BATCH_N_POLICIES,
                             SPMV_BATCH_SORTED,
                             Batch, spmv_batch_apply, spmv_batch_apply_host, spmv_batch_apply_host_async,
                             spmv_batch_apply_noalloc, spmv_batch_host_sync,
                             spmv_batch_apply_separate,
                             spmv_batch_autotune,
                             spmv_batch_config, spmv_batch_create, spmv_batch_default_config, spmv_batch_destroy,
                             spmv_batch_get_config, spmv_batch_info, spmv_batch_set_config, spmv_batch_set_io,
                             spmv_batch_set_policies)

from ._binding_reorder import Reorder, permute_csr, rcm  # noqa: F401,E402
from ._binding_solver import (Solver, spmv_cg_solve, spmv_cg_summary, spmv_lanczos,  # noqa: F401,E402
                             spmv_solver_create, spmv_solver_destroy)
from ._binding_model import (spmv_model_adam_step, spmv_model_create, spmv_model_destroy,  # noqa: F401,E402
                             spmv_model_forward, spmv_model_get_params, spmv_model_info, spmv_model_load,
                             spmv_model_loss_grad, spmv_model_save, spmv_model_select, spmv_model_select_guarded,
                             spmv_model_set_normalizer,
                             spmv_model_set_params, spmv_model_train_step)

LANE_VARIANTS = {1: SPMV_CRS_L1, 2: SPMV_CRS_L2, 4: SPMV_CRS_L4, 8: SPMV_CRS_L8, 16: SPMV_CRS_L16,
                 32: SPMV_CRS_L32}


N_FEATURES = 34


def features(A, k: int = 1) -> np.ndarray:
    """Cost-model feature vector of a host CRS matrix (computed by the library)."""
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
    out = np.empty(N_FEATURES, dtype=np.float64)
    spmv_features(A.n_rows, A.n_cols, rp.ctypes.data, ci.ctypes.data, k, out.ctypes.data)
    return out


def _host_csr(A):
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
    va = np.ascontiguousarray(A.val, dtype=np.float64)
    return rp, ci, va


def sell_build(A, sigma: int = 1) -> dict:
    """spmv_sell_build_host: the SELL-32-sigma arrays of a host CRS matrix (no device)."""
    rp, ci, va = _host_csr(A)
    nc, ns = np.zeros(1, np.int64), np.zeros(1, np.int64)
    args = (A.n_rows, A.n_cols, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, sigma, nc.ctypes.data,
            ns.ctypes.data)
    spmv_sell_build_host(*args, None, None, None, None, None)
    out = {"perm": np.empty(A.n_rows, np.int32), "chunk_ptr": np.empty(int(nc[0]) + 1, np.int64),
           "chunk_len": np.empty(int(nc[0]), np.int32), "sell_col": np.empty(int(ns[0]), np.int32),
           "sell_val": np.empty(int(ns[0]), np.float64)}
    spmv_sell_build_host(*args, *(out[k].ctypes.data for k in ("perm", "chunk_ptr", "chunk_len", "sell_col",
                                                               "sell_val")))
    return out


def split_build(A, h: int) -> dict:
    """spmv_split_build_host: the local/halo split arrays at column h (no device)."""
    rp, ci, va = _host_csr(A)
    sz = np.zeros(3, np.int64)
    args = (A.n_rows, A.n_cols, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, h, sz[0:].ctypes.data,
            sz[1:].ctypes.data, sz[2:].ctypes.data)
    spmv_split_build_host(*args, None, None, None, None, None, None, None)
    nl, nh, hn = (int(x) for x in sz)
    out = {"loc_row_ptr": np.empty(A.n_rows + 1, np.int32), "loc_col": np.empty(nl, np.int32),
           "loc_val": np.empty(nl, np.float64), "halo_rows": np.empty(nh, np.int32),
           "halo_row_ptr": np.empty(nh + 1, np.int32), "halo_col": np.empty(hn, np.int32),
           "halo_val": np.empty(hn, np.float64)}
    spmv_split_build_host(*args, *(out[k].ctypes.data for k in ("loc_row_ptr", "loc_col", "loc_val", "halo_rows",
                                                                "halo_row_ptr", "halo_col", "halo_val")))
    return out


def sym_build(A) -> dict:
    """spmv_sym_build_host: the stored upper triangle of a symmetric host CRS matrix
    (raises SpmvError SPMV_ERR_UNSUPPORTED if A is not symmetric; no device)."""
    rp, ci, va = _host_csr(A)
    nz = np.zeros(1, np.int64)
    args = (A.n_rows, A.n_cols, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, nz.ctypes.data)
    spmv_sym_build_host(*args, None, None, None)
    out = {"row_ptr": np.empty(A.n_rows + 1, np.int32), "col": np.empty(int(nz[0]), np.int32),
           "val": np.empty(int(nz[0]), np.float64)}
    spmv_sym_build_host(*args, out["row_ptr"].ctypes.data, out["col"].ctypes.data, out["val"].ctypes.data)
    return out


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int:
    return t.data_ptr()


class Plan:
    """Owns one spmv_handle.  Host CRS arrays are copied at construction."""

    def __init__(self, n_rows: int, n_cols: int, row_ptr, col_idx, val, *, variant: int = SPMV_VARIANT_AUTO,
                 sell_sigma: int = 1, val_fp32: bool = False, max_k: int = 16, halo_begin: int | None = None):
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        va = np.ascontiguousarray(val, dtype=np.float64)
        o = spmv_default_options()
        o.variant, o.sell_sigma, o.val_fp32, o.max_k = variant, sell_sigma, int(val_fp32), max_k
        if halo_begin is not None:   # local/halo split at column halo_begin
            o.split, o.halo_begin = 1, halo_begin
        self.n_rows, self.n_cols = int(n_rows), int(n_cols)
        # nnz is the count of stored entries the caller hands over; the library
        # checks it against row_ptr[n_rows]
        self.handle = spmv_create(n_rows, n_cols, len(ci), rp.ctypes.data, ci.ctypes.data, va.ctypes.data, o)

    @classmethod
    def from_csr(cls, A, **kw) -> "Plan":
        return cls(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.val, **kw)

    def apply(self, B, C, stream=None) -> None:
        spmv_apply(self.handle, _ptr(B), _ptr(C), _stream_handle(stream))

    def apply_block(self, B, C, k: int | None = None, stream=None) -> None:
        """B: (n_cols, ldb) row-major, C: (n_rows, ldc) row-major; k defaults to B.shape[1]."""
        k = B.shape[1] if k is None else k
        spmv_apply_block(self.handle, _ptr(B), k, B.stride(0), _ptr(C), C.stride(0), _stream_handle(stream))

    def apply_split(self, B, B_halo_pinned, C, main_stream=None, copy_stream=None) -> None:
        ms = _stream_handle(main_stream)
        cs = ms if copy_stream is None else _stream_handle(copy_stream)
        spmv_apply_split(self.handle, _ptr(B), _ptr(B_halo_pinned), _ptr(C), ms, cs)

    def apply_host(self, B: np.ndarray, k: int = 1, stream=None) -> np.ndarray:
        """End to end from host memory: copies B in, multiplies, copies C back (synchronous)."""
        Bc = np.ascontiguousarray(B, dtype=np.float64)
        C = np.empty((self.n_rows, k) if k > 1 else self.n_rows, dtype=np.float64)
        spmv_apply_host(self.handle, Bc.ctypes.data, k, C.ctypes.data, _stream_handle(stream))
        return C

    def apply_host_ptr(self, B_ptr: int, k: int, C_ptr: int, stream=None) -> None:
        spmv_apply_host(self.handle, B_ptr, k, C_ptr, _stream_handle(stream))

    def apply_host_async(self, B_pinned, C_pinned, k: int = 1, stream=None) -> None:
        """Enqueue one pipelined end-to-end step (page-locked torch CPU tensors)."""
        _b.spmv_apply_host_async(self.handle, B_pinned.data_ptr(), k, C_pinned.data_ptr(), _stream_handle(stream))

    def host_sync(self) -> None:
        _b.spmv_host_sync(self.handle)

    def set_variant(self, variant: int, sell_sigma: int = 1) -> None:
        spmv_set_variant(self.handle, variant, sell_sigma)

    def info(self):
        return spmv_get_info(self.handle)

    def set_tuning(self, prefetch_distance: int | None = None) -> None:
        t = spmv_get_tuning(self.handle)
        if prefetch_distance is not None:
            t.prefetch_distance = prefetch_distance
        spmv_set_tuning(self.handle, t)

    def tuning(self):
        return spmv_get_tuning(self.handle)

    def check(self, stream=None) -> None:
        spmv_check(self.handle, _stream_handle(stream))

    def sell_export(self) -> dict:
        i = self.info()
        out = {"perm": np.empty(i.n_rows, np.int32), "chunk_ptr": np.empty(i.sell_chunks + 1, np.int64),
               "chunk_len": np.empty(i.sell_chunks, np.int32), "sell_col": np.empty(i.sell_slots, np.int32),
               "sell_val": np.empty(i.sell_slots, np.float64)}
        spmv_sell_export(self.handle, *(out[k].ctypes.data for k in ("perm", "chunk_ptr", "chunk_len", "sell_col",
                                                                     "sell_val")))
        return out

    def select(self, model_handle, k: int, outputs) -> int:
        """spmv_select: run the cost model on this plan's features for k
        right-hand sides and switch to its choice; outputs[o] = (variant, sigma)
        for network output o.  Returns o."""
        v = np.ascontiguousarray([o[0] for o in outputs], dtype=np.int32)
        sg = np.ascontiguousarray([o[1] for o in outputs], dtype=np.int32)
        ch = np.zeros(1, np.int32)
        _b._check(_b.load().spmv_select(self.handle, model_handle, k, v.ctypes.data, sg.ctypes.data,
                                        ch.ctypes.data, _stream_handle(None)))
        return int(ch[0])

    def autotune(self, B, C, candidates, k: int | None = None, reps: int = 7, stream=None):
        """spmv_autotune: exhaustive timed sweep over candidates [(variant, sigma)];
        the plan switches to the fastest.  Returns (index, median ms per candidate)."""
        kk = 1 if B.dim() == 1 else (B.shape[1] if k is None else k)
        ldb = 1 if B.dim() == 1 else B.stride(0)
        ldc = 1 if C.dim() == 1 else C.stride(0)
        v = np.ascontiguousarray([c[0] for c in candidates], dtype=np.int32)
        sg = np.ascontiguousarray([c[1] for c in candidates], dtype=np.int32)
        best = np.zeros(1, np.int32)
        times = np.zeros(len(candidates), np.float32)
        _b._check(_b.load().spmv_autotune(self.handle, kk, _ptr(B), ldb, _ptr(C), ldc, v.ctypes.data, sg.ctypes.data,
                                          len(candidates), reps, best.ctypes.data, times.ctypes.data,
                                          _stream_handle(stream)))
        return int(best[0]), times

    def sym_export(self) -> dict:
        i = self.info()
        out = {"row_ptr": np.empty(i.n_rows + 1, np.int32), "col": np.empty(i.sym_nnz, np.int32),
               "val": np.empty(i.sym_nnz, np.float64)}
        spmv_sym_export(self.handle, *(out[k].ctypes.data for k in ("row_ptr", "col", "val")))
        return out

    def split_export(self) -> dict:
        i = self.info()
        nl = i.nnz - i.halo_nnz
        out = {"loc_row_ptr": np.empty(i.n_rows + 1, np.int32), "loc_col": np.empty(nl, np.int32),
               "loc_val": np.empty(nl, np.float64), "halo_rows": np.empty(i.n_halo_rows, np.int32),
               "halo_row_ptr": np.empty(i.n_halo_rows + 1, np.int32), "halo_col": np.empty(i.halo_nnz, np.int32),
               "halo_val": np.empty(i.halo_nnz, np.float64)}
        keys = ("loc_row_ptr", "loc_col", "loc_val", "halo_rows", "halo_row_ptr", "halo_col", "halo_val")
        spmv_split_export(self.handle, *(out[k].ctypes.data for k in keys))
        return out

    def close(self) -> None:
        if getattr(self, "handle", None) is not None:
            spmv_destroy(self.handle)
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
