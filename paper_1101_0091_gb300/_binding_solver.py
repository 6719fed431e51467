"""ctypes binding of the iterative-solver entry points of include/spmv.h
(same names, argument marshalling only), and a small Solver wrapper."""
from __future__ import annotations

import ctypes

import numpy as np

from ._binding import _check, _i32, _vp, load


class spmv_cg_summary(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32), ("breakdown", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_P = ctypes.POINTER
_SIGS = {
    "spmv_solver_create": ([_vp, _i32, _P(_vp)], ctypes.c_int),
    "spmv_solver_destroy": ([_vp], ctypes.c_int),
    "spmv_cg_solve": ([_vp, _vp, _vp, _i32, ctypes.c_double, _i32, _vp, _vp, _vp, _P(spmv_cg_summary)],
                      ctypes.c_int),
    "spmv_lanczos": ([_vp, _vp, _i32, _vp, _vp, _vp], ctypes.c_int),
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


def spmv_solver_create(plan_handle, k: int):
    h = ctypes.c_void_p()
    _check(_lib().spmv_solver_create(plan_handle, k, ctypes.byref(h)))
    return h


def spmv_solver_destroy(h) -> None:
    _check(_lib().spmv_solver_destroy(h))


def spmv_cg_solve(h, B_dev: int, X_dev: int, max_iter: int, rtol: float, check_every: int, stream: int,
                  iterations_host: int, rr_host: int, summary: spmv_cg_summary) -> None:
    _check(_lib().spmv_cg_solve(h, B_dev, X_dev, max_iter, rtol, check_every, stream, iterations_host, rr_host,
                                ctypes.byref(summary)))


def spmv_lanczos(h, V0_dev: int, m: int, alpha_host: int, beta_host: int, stream: int) -> None:
    _check(_lib().spmv_lanczos(h, V0_dev, m, alpha_host, beta_host, stream))


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


class Solver:
    """CG and Lanczos on k columns through a plan (which must outlive it).
    Blocks are torch CUDA tensors of shape (n, k), row-major and contiguous."""

    def __init__(self, plan, k: int):
        self.plan, self.k = plan, int(k)
        self.handle = spmv_solver_create(plan.handle, self.k)

    def cg(self, B, X, max_iter: int = 1000, rtol: float = 1e-10, check_every: int = 10, stream=None):
        """Solves in place (X holds the initial guess).  Returns (iterations[k], rr[k], summary)."""
        assert B.is_contiguous() and X.is_contiguous()
        it = np.zeros(self.k, np.int32)
        rr = np.zeros(self.k, np.float64)
        s = spmv_cg_summary()
        spmv_cg_solve(self.handle, B.data_ptr(), X.data_ptr(), max_iter, rtol, check_every, _stream(stream),
                      it.ctypes.data, rr.ctypes.data, s)
        return it, rr, s

    def lanczos(self, V0, m: int, stream=None):
        """Returns (alpha[m, k], beta[m, k])."""
        assert V0.is_contiguous()
        a = np.zeros((m, self.k), np.float64)
        b = np.zeros((m, self.k), np.float64)
        spmv_lanczos(self.handle, V0.data_ptr(), m, a.ctypes.data, b.ctypes.data, _stream(stream))
        return a, b

    def close(self) -> None:
        if getattr(self, "handle", None) is not None:
            spmv_solver_destroy(self.handle)
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
