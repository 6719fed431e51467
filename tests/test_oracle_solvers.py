"""Pins of the oracle's iterative solvers (CG and Lanczos on k columns) to
things other than themselves: dense linear solves, finite termination, true
residuals, the closed-form spectrum of the 2D Laplacian, dense eigenvalues of
small matrices, and the Lanczos relations A V = V T + beta v e^T and V^T V = I."""
import math

import numpy as np
import pytest

import gen
import oracle
from oracle import solvers


def csr_from_dense(D):
    n = D.shape[0]
    rows, cols = np.nonzero(D)
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum(np.bincount(rows, minlength=n))
    return gen.CSR(n, D.shape[1], rp, cols.astype(np.int32), D[rows, cols].astype(np.float64))


def spd_dense(n, seed, cond=50.0):
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, cond, n)
    D = (Qm * ev) @ Qm.T
    return 0.5 * (D + D.T)


@pytest.mark.parametrize("seed", range(4))
def test_cg_matches_dense_solve(seed):
    D = spd_dense(30, seed)
    A = csr_from_dense(D)
    B = np.random.default_rng(seed).standard_normal((30, 3))
    X, info = solvers.cg(A, B, max_iter=300, rtol=1e-13)
    ref = np.linalg.solve(D, B)
    assert np.allclose(X, ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    assert not info["breakdown"].any()


def test_cg_finite_termination():
    """n distinct eigenvalues: CG reaches the solution in about n steps."""
    D = spd_dense(8, 7, cond=10.0)
    A = csr_from_dense(D)
    b = np.arange(1.0, 9.0)
    X, info = solvers.cg(A, b, max_iter=8, rtol=0.0)
    assert np.allclose(X[:, 0], np.linalg.solve(D, b), atol=1e-9)


def test_cg_poisson_true_residual_and_known_solution():
    """A * 1 = 1e-3 on the Poisson workload: with b = 1e-3 the solution is 1;
    at convergence the true residual |b - A x| matches the recurrence's."""
    A = gen.poisson3d_var(10)
    b = np.full(A.n_rows, 1e-3)
    X, info = solvers.cg(A, b, max_iter=2000, rtol=1e-12)
    true_r = b - oracle.spmv(A, X[:, 0])
    assert np.linalg.norm(true_r) <= 2e-12 * np.linalg.norm(b)
    assert abs(math.sqrt(info["rr"][0]) - np.linalg.norm(true_r)) <= 1e-3 * np.linalg.norm(b)
    assert np.allclose(X[:, 0], 1.0, atol=1e-8)


def test_cg_columns_freeze_independently():
    """A zero right-hand side never iterates; a column that converges early is
    left exactly as it was while the others continue."""
    A = gen.poisson3d_var(8)
    rng = np.random.default_rng(3)
    B = np.stack([np.zeros(A.n_rows), rng.standard_normal(A.n_rows), oracle.spmv(A, np.ones(A.n_rows))], 1)
    X, info = solvers.cg(A, B, max_iter=500, rtol=1e-6)
    assert info["iterations"][0] == 0 and np.all(X[:, 0] == 0)
    X_loose, info_l = solvers.cg(A, B[:, 1:2], max_iter=500, rtol=1e-6)
    assert np.array_equal(X[:, 1], X_loose[:, 0])        # freezing leaves the column untouched
    assert info["iterations"][1] == info_l["iterations"][0]
    assert info["iterations"][2] != info["iterations"][1]


def test_cg_breakdown_on_indefinite():
    D = np.diag([1.0, -1.0])
    A = csr_from_dense(D)
    X, info = solvers.cg(A, np.array([1.0, 1.0]), max_iter=10, rtol=1e-12)
    assert info["breakdown"][0]


def test_lanczos_small_dense_spectrum():
    """m = n steps reproduce the spectrum of a small symmetric matrix."""
    rng = np.random.default_rng(1)
    M = rng.standard_normal((6, 6))
    D = M + M.T
    A = csr_from_dense(D)
    a, b = solvers.lanczos(A, rng.standard_normal(6), 6)
    assert np.allclose(solvers.ritz_values(a[:, 0], b[:, 0]), np.linalg.eigvalsh(D), atol=1e-10)


def test_lanczos_laplace_extremal_eigenvalues():
    """2D Dirichlet Laplacian on 16 x 16: extreme eigenvalues 4 -+ 4 cos(pi/17)."""
    A = gen.laplace2d(16)
    v0 = gen.rhs_block(A.n_cols, 2, seed=4)
    a, b = solvers.lanczos(A, v0, 80)
    for c in range(2):
        ritz = solvers.ritz_values(a[:, c], b[:, c])
        assert abs(ritz[-1] - (4 + 4 * math.cos(math.pi / 17))) < 1e-9
        assert abs(ritz[0] - (4 - 4 * math.cos(math.pi / 17))) < 1e-9


def test_lanczos_relations():
    """A V_m = V_m T_m + beta_m v_{m+1} e_m^T and V_m^T V_m = I (few steps)."""
    A = gen.eigen_shaped(3000, window=1 << 9)
    v0 = gen.uniform(A.n_cols, seed=6)
    m = 12
    a, b, V = solvers.lanczos(A, v0, m, return_vectors=True)
    Vm = V[:m, :, 0].T                      # n x m
    T = np.diag(a[:, 0]) + np.diag(b[:m - 1, 0], 1) + np.diag(b[:m - 1, 0], -1)
    AV = np.stack([oracle.spmv(A, Vm[:, j]) for j in range(m)], 1)
    resid = AV - Vm @ T
    resid[:, -1] -= b[m - 1, 0] * V[m, :, 0]
    assert np.abs(resid).max() < 1e-12 * np.abs(AV).max()
    assert np.abs(Vm.T @ Vm - np.eye(m)).max() < 1e-10
