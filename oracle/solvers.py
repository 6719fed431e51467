"""ORACLE — test infrastructure only.

Plain numpy FP64 restatements of the iterative solvers that consume the
sparse product.  Sec. 1.3.1 names Lanczos and Jacobi-Davidson as the methods
run on the Hamiltonian matrices, with the product as their most expensive
step; conjugate gradients is the matching method for the symmetric positive
definite Poisson matrix.  Both run on k independent columns at once, so every
product is one k-column SpMM.  Products use the oracle's CRS loop
(``oracle.spmm``); inner products are numpy sums over the rows of each
column, taken on a contiguous copy so that a column's result does not depend
on the columns beside it.

Conjugate gradients (Hestenes and Stiefel, J. Res. NBS 49, 1952), per column,
with X holding the initial guess:

    R = B - A X,  P = R,  rr = R.R,  tol2 = rtol^2 * B.B,  active = rr > tol2
    repeat while some column is active (at most max_iter times):
        Q = A P;  pq = P.Q
        for active columns:  alpha = rr / pq          (pq <= 0: breakdown, stop the column)
                             X += alpha P;  R -= alpha Q;  rr' = R.R
                             beta = rr' / rr;  P = R + beta P;  rr = rr';  iterations += 1
                             active = rr > tol2
    inactive columns are left exactly as they are.

Lanczos (J. Res. NBS 45, 1950), three-term recurrence without
reorthogonalisation, per column, from a start vector v0:

    beta_0 = |v0|,  v_1 = v0 / beta_0,  v_0 = 0
    for j = 1..m:  w = A v_j - beta_{j-1} v_{j-1};  alpha_j = w.v_j;  w = w - alpha_j v_j
                   beta_j = |w|;  v_{j+1} = w / beta_j       (beta_j = 0: the column stops)

returning alpha_1..m and beta_1..m; the eigenvalues of the tridiagonal T_m
(alpha on the diagonal, beta_1..m-1 beside it) are the Ritz values.
"""
from __future__ import annotations

import numpy as np

from . import spmm


def _cols(a) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    return a.reshape(-1, 1) if a.ndim == 1 else a


def _dot(U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Per-column inner products, each over a contiguous copy of its columns,
    so a column's result does not depend on how many columns run beside it."""
    return np.array([np.sum(np.ascontiguousarray(U[:, c]) * np.ascontiguousarray(V[:, c]))
                     for c in range(U.shape[1])])


def cg(A, B, X0=None, max_iter: int = 100, rtol: float = 1e-10):
    """Conjugate gradients on the k columns of B.  Returns (X, info) with
    info = {"iterations": int[k], "rr": float[k], "breakdown": bool[k],
            "alpha": [float[k] per iteration], "beta": [...], "rr_hist": [...]}."""
    B = _cols(B).copy()
    n, k = B.shape
    X = np.zeros_like(B) if X0 is None else _cols(X0).copy()
    R = B - spmm(A, X)
    P = R.copy()
    rr = _dot(R, R)
    tol2 = rtol * rtol * _dot(B, B)
    active = rr > tol2
    breakdown = np.zeros(k, dtype=bool)
    iters = np.zeros(k, dtype=np.int64)
    hist = {"alpha": [], "beta": [], "rr_hist": [rr.copy()]}
    for _ in range(max_iter):
        if not active.any():
            break
        Q = spmm(A, P)
        pq = _dot(P, Q)
        bad = active & ~(pq > 0)
        breakdown |= bad
        active &= ~bad
        alpha = np.where(active, rr / np.where(active, pq, 1.0), 0.0)
        X = np.where(active, X + alpha * P, X)
        R = np.where(active, R - alpha * Q, R)
        rr_new = _dot(R, R)
        beta = np.where(active, rr_new / np.where(active, rr, 1.0), 0.0)
        P = np.where(active, R + beta * P, P)
        rr = np.where(active, rr_new, rr)
        iters += active
        hist["alpha"].append(alpha)
        hist["beta"].append(beta)
        hist["rr_hist"].append(rr.copy())
        active &= rr > tol2
    info = {"iterations": iters, "rr": rr, "breakdown": breakdown, **hist}
    return X, info


def lanczos(A, V0, m: int, return_vectors: bool = False):
    """m Lanczos steps on each column of V0.  Returns (alpha[m, k], beta[m, k])
    and, with return_vectors, the basis V[m+1, n, k] (v_1 .. v_{m+1})."""
    V0 = _cols(V0)
    n, k = V0.shape
    beta0 = np.sqrt(_dot(V0, V0))
    live = beta0 > 0
    v = np.where(live, V0 / np.where(live, beta0, 1.0), 0.0)
    v_prev = np.zeros_like(v)
    b_prev = np.zeros(k)
    alphas = np.zeros((m, k))
    betas = np.zeros((m, k))
    basis = [v.copy()] if return_vectors else None
    for j in range(m):
        w = spmm(A, v) - b_prev * v_prev
        a = _dot(w, v)
        w = w - a * v
        b = np.sqrt(_dot(w, w))
        alphas[j] = np.where(live, a, 0.0)
        betas[j] = np.where(live, b, 0.0)
        live &= b > 0
        v_prev, b_prev = v, np.where(live, b, 0.0)
        v = np.where(live, w / np.where(live, b, 1.0), 0.0)
        if return_vectors:
            basis.append(v.copy())
    if return_vectors:
        return alphas, betas, np.stack(basis)
    return alphas, betas


def ritz_values(alpha: np.ndarray, beta: np.ndarray) -> np.ndarray:
    """Eigenvalues of the tridiagonal T (alpha on the diagonal, beta[:-1] beside it)."""
    m = len(alpha)
    T = np.diag(alpha) + np.diag(beta[:m - 1], 1) + np.diag(beta[:m - 1], -1)
    return np.linalg.eigvalsh(T)
