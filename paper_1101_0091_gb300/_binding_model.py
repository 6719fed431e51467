"""ctypes binding of the cost-model entry points of include/spmv.h (same
names, argument marshalling only)."""
from __future__ import annotations

import ctypes

import numpy as np

from ._binding import _check, _i32, _i64, _vp, load

_P = ctypes.POINTER
_SIGS = {
    "spmv_model_create": ([_P(_vp), _i32, _i32, _i32, _vp], ctypes.c_int),
    "spmv_model_info": ([_vp, _P(_i32), _P(_i32), _P(_i32), _P(_i64), _P(_i32)], ctypes.c_int),
    "spmv_model_set_params": ([_vp, _vp], ctypes.c_int),
    "spmv_model_get_params": ([_vp, _vp], ctypes.c_int),
    "spmv_model_set_normalizer": ([_vp, _vp, _vp], ctypes.c_int),
    "spmv_model_forward": ([_vp, _vp, _i32, _vp, _vp], ctypes.c_int),
    "spmv_model_loss_grad": ([_vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp], ctypes.c_int),
    "spmv_model_adam_step": ([_vp, _vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _vp],
                             ctypes.c_int),
    "spmv_model_train_step": ([_vp, _vp, _vp, _vp, _i32, ctypes.c_float, _vp, _vp], ctypes.c_int),
    "spmv_model_select": ([_vp, _vp, _i32, _vp, _vp, _vp], ctypes.c_int),
    "spmv_model_select_guarded": ([_vp, _vp, _i32, _i32, ctypes.c_float, _vp, _vp, _vp], ctypes.c_int),
    "spmv_model_save": ([_vp, ctypes.c_char_p], ctypes.c_int),
    "spmv_model_load": ([_P(_vp), ctypes.c_char_p], ctypes.c_int),
    "spmv_model_destroy": ([_vp], ctypes.c_int),
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


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def n_params(F: int, H: int, V: int) -> int:
    return H * F + H + H * H + H + V * H + V


def spmv_model_create(n_in: int, n_hidden: int, n_out: int, params) -> ctypes.c_void_p:
    p = _f32(params)
    assert p.size == n_params(n_in, n_hidden, n_out)
    h = ctypes.c_void_p()
    _check(_lib().spmv_model_create(ctypes.byref(h), n_in, n_hidden, n_out, p.ctypes.data))
    return h


def spmv_model_info(m):
    a, b, c, s = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    n = ctypes.c_int64()
    _check(_lib().spmv_model_info(m, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(n),
                                  ctypes.byref(s)))
    return a.value, b.value, c.value, n.value, s.value


def spmv_model_set_params(m, params) -> None:
    p = _f32(params)
    _check(_lib().spmv_model_set_params(m, p.ctypes.data))


def spmv_model_get_params(m) -> np.ndarray:
    F, H, V, n, _ = spmv_model_info(m)
    out = np.empty(n, dtype=np.float32)
    _check(_lib().spmv_model_get_params(m, out.ctypes.data))
    return out


def spmv_model_set_normalizer(m, mean, inv_std) -> None:
    a, b = _f32(mean), _f32(inv_std)
    _check(_lib().spmv_model_set_normalizer(m, a.ctypes.data, b.ctypes.data))


def spmv_model_forward(m, X_dev: int, M: int, Y_dev: int, stream: int = 0) -> None:
    _check(_lib().spmv_model_forward(m, X_dev, M, Y_dev, stream))


def spmv_model_loss_grad(m, X_dev: int, T_dev: int, mask_dev: int, M: int, loss_dev: int, grad_dev: int,
                         stream: int = 0) -> None:
    _check(_lib().spmv_model_loss_grad(m, X_dev, T_dev, mask_dev, M, loss_dev, grad_dev, stream))


def spmv_model_adam_step(m, grad_dev, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, stream: int = 0) -> None:
    _check(_lib().spmv_model_adam_step(m, grad_dev, lr, beta1, beta2, eps, stream))


def spmv_model_train_step(m, X_dev: int, T_dev: int, mask_dev: int, M: int, lr: float, loss_dev: int | None,
                          stream: int = 0) -> None:
    _check(_lib().spmv_model_train_step(m, X_dev, T_dev, mask_dev, M, lr, loss_dev, stream))


def spmv_model_select(m, features: np.ndarray, stream: int = 0):
    X = np.ascontiguousarray(features, dtype=np.float64)
    if X.ndim == 1:
        X = X.reshape(1, -1)
    F, H, V, _, _ = spmv_model_info(m)
    choice = np.empty(X.shape[0], dtype=np.int32)
    pred = np.empty((X.shape[0], V), dtype=np.float32)
    _check(_lib().spmv_model_select(m, X.ctypes.data, X.shape[0], choice.ctypes.data, pred.ctypes.data, stream))
    return choice, pred


def spmv_model_select_guarded(m, features: np.ndarray, fallback: int, margin: float, stream: int = 0):
    X = np.ascontiguousarray(features, dtype=np.float64)
    if X.ndim == 1:
        X = X.reshape(1, -1)
    F, H, V, _, _ = spmv_model_info(m)
    choice = np.empty(X.shape[0], dtype=np.int32)
    pred = np.empty((X.shape[0], V), dtype=np.float32)
    _check(_lib().spmv_model_select_guarded(m, X.ctypes.data, X.shape[0], fallback, margin, choice.ctypes.data,
                                            pred.ctypes.data, stream))
    return choice, pred


def spmv_model_save(m, path: str) -> None:
    _check(_lib().spmv_model_save(m, path.encode()))


def spmv_model_load(path: str) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(_lib().spmv_model_load(ctypes.byref(h), path.encode()))
    return h


def spmv_model_destroy(m) -> None:
    _check(_lib().spmv_model_destroy(m))
