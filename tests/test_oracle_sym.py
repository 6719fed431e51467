"""Pins of the oracle's symmetric CRS (Sec. 1.3.1): the symmetry test against
dense transposition, the stored triangle against dense reassembly, and the
product from the triangle against exact integer arithmetic, extended-precision
dense products, the Laplacian's closed-form eigenpairs and the row-sum
invariant of the 3D Poisson workload."""
import math

import numpy as np
import pytest

import gen
import oracle

TOL = 1e-13


def dense_of(n_rows, n_cols, row_ptr, col, val) -> np.ndarray:
    D = np.zeros((n_rows, n_cols), dtype=np.float64)
    for i in range(n_rows):
        for j in range(row_ptr[i], row_ptr[i + 1]):
            D[i, col[j]] += val[j]
    return D


def sym_case(seed, n=None, integer=False, duplicates=False, shuffle=False, empty_rows=0.0):
    rng = np.random.default_rng(500 + seed)
    n = n or int(rng.integers(1, 80))
    A = gen.random_csr(n, n, 0.15, seed, integer=integer, empty_rows=empty_rows, duplicates=duplicates)
    return gen.symmetric_from(A, seed=seed, shuffle=shuffle)


@pytest.mark.parametrize("seed", range(8))
def test_symmetric_cases_match_dense_transpose(seed):
    S = sym_case(seed, duplicates=(seed % 2 == 0), shuffle=(seed % 3 == 0), empty_rows=0.1)
    D = dense_of(S.n_rows, S.n_cols, S.row_ptr, S.col_idx, S.val)
    assert np.array_equal(D, D.T)
    assert oracle.is_symmetric(S)


@pytest.mark.parametrize("seed", range(6))
def test_asymmetric_cases_are_rejected(seed):
    S = sym_case(seed, n=40)
    off = np.flatnonzero(S.col_idx != np.repeat(np.arange(S.n_rows), np.diff(S.row_ptr)))
    assert len(off) > 0
    j = off[seed % len(off)]
    # one value changed: the dense matrix is no longer symmetric
    bad = gen.CSR(S.n_rows, S.n_cols, S.row_ptr.copy(), S.col_idx.copy(), S.val.copy())
    bad.val[j] += 0.5
    D = dense_of(bad.n_rows, bad.n_cols, bad.row_ptr, bad.col_idx, bad.val)
    assert not np.array_equal(D, D.T)
    assert not oracle.is_symmetric(bad)
    # one mirror dropped
    keep = np.ones(S.nnz, bool)
    keep[j] = False
    rows = np.repeat(np.arange(S.n_rows), np.diff(S.row_ptr))[keep]
    rp = np.zeros(S.n_rows + 1, np.int32)
    rp[1:] = np.cumsum(np.bincount(rows, minlength=S.n_rows))
    dropped = gen.CSR(S.n_rows, S.n_cols, rp, S.col_idx[keep], S.val[keep])
    assert not oracle.is_symmetric(dropped)


def test_symmetry_special_cases():
    empty = gen.CSR(0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    assert oracle.is_symmetric(empty)
    diag = gen.CSR(3, 3, np.array([0, 1, 2, 3], np.int32), np.array([0, 1, 2], np.int32), np.array([1.0, -2, 3]))
    assert oracle.is_symmetric(diag)
    nonsq = gen.CSR(2, 3, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, 1.0]))
    assert not oracle.is_symmetric(nonsq)
    # -0.0 mirrors +0.0
    z = gen.CSR(2, 2, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), np.array([0.0, -0.0]))
    assert oracle.is_symmetric(z)
    # duplicates must mirror one to one: (0,1) = 1 + 2 against (1,0) = 3 is rejected
    split = gen.CSR(2, 2, np.array([0, 2, 3], np.int32), np.array([1, 1, 0], np.int32), np.array([1.0, 2.0, 3.0]))
    assert not oracle.is_symmetric(split)
    mirrored = gen.CSR(2, 2, np.array([0, 2, 4], np.int32), np.array([1, 1, 0, 0], np.int32),
                       np.array([1.0, 2.0, 2.0, 1.0]))
    assert oracle.is_symmetric(mirrored)


@pytest.mark.parametrize("seed", range(8))
def test_triangle_reassembles_the_matrix(seed):
    """U + (strictly upper part of U)^T equals the dense matrix, the triangle
    keeps (nnz + diagonal entries) / 2 entries, all on or above the diagonal."""
    S = sym_case(seed, duplicates=(seed % 2 == 1), shuffle=(seed % 2 == 0), empty_rows=0.1)
    T = oracle.sym_build(S)
    n = S.n_rows
    rows_u = np.repeat(np.arange(n), np.diff(T.row_ptr))
    assert np.all(T.col >= rows_u)
    n_diag = int(np.sum(S.col_idx == np.repeat(np.arange(n), np.diff(S.row_ptr))))
    assert T.nnz == (S.nnz + n_diag) // 2
    U = dense_of(n, n, T.row_ptr, T.col, T.val)
    assert np.array_equal(U + np.triu(U, 1).T, dense_of(n, n, S.row_ptr, S.col_idx, S.val))


@pytest.mark.parametrize("seed", range(6))
def test_triangle_product_integer_exact(seed):
    """Integer values with |v| <= 2^10: every partial sum is exact, so the
    product from the triangle equals the exact integer product bit for bit."""
    S = sym_case(seed, n=120, integer=True, duplicates=True, shuffle=(seed % 2 == 0), empty_rows=0.05)
    x = np.random.default_rng(seed).integers(-1024, 1025, S.n_cols).astype(np.float64)
    D = dense_of(S.n_rows, S.n_cols, S.row_ptr, S.col_idx, S.val).astype(np.int64)
    exact = (D @ x.astype(np.int64)).astype(np.float64)
    T = oracle.sym_build(S)
    assert np.array_equal(oracle.sym_spmv(T, x), exact)
    assert np.array_equal(oracle.spmv(S, x), exact)


@pytest.mark.parametrize("seed", range(6))
def test_triangle_product_dense_extended(seed):
    S = sym_case(seed, shuffle=True, duplicates=(seed % 2 == 0))
    x = np.random.default_rng(seed).uniform(-1, 1, S.n_cols)
    D = dense_of(S.n_rows, S.n_cols, S.row_ptr, S.col_idx, S.val).astype(np.longdouble)
    ref = (D @ x.astype(np.longdouble)).astype(np.float64)
    scale = oracle.abs_scale(S, x)
    y = oracle.sym_spmv(oracle.sym_build(S), x)
    assert oracle.max_err_ratio(y, ref, scale, TOL) <= 1.0


@pytest.mark.parametrize("p,q", [(1, 1), (3, 7), (64, 200), (256, 256)])
def test_triangle_product_laplace_eigenpairs(p, q):
    """2D Dirichlet Laplacian on a 256 x 256 grid: A v = lambda v for
    v(x, y) = sin(p pi (x+1)/257) sin(q pi (y+1)/257),
    lambda = 4 - 2 cos(p pi/257) - 2 cos(q pi/257)."""
    nx = 256
    A = gen.laplace2d(nx)
    assert oracle.is_symmetric(A)
    xs = np.arange(nx)
    sx = np.sin(np.pi * ((p * (xs + 1)) % (2 * (nx + 1))) / (nx + 1))
    sy = np.sin(np.pi * ((q * (xs + 1)) % (2 * (nx + 1))) / (nx + 1))
    v = (sy[:, None] * sx[None, :]).reshape(-1)
    lam = 4 - 2 * math.cos(p * math.pi / (nx + 1)) - 2 * math.cos(q * math.pi / (nx + 1))
    y = oracle.sym_spmv(oracle.sym_build(A), v)
    scale = oracle.abs_scale(A, v)
    assert np.all(np.abs(y - lam * v) <= TOL * scale + 8 * 2.2e-16 * np.abs(v).max() + 1e-15)


def test_triangle_product_poisson_row_sums():
    """3D Poisson workload: off-diagonals negative, diagonal = sum |off| + 1e-3,
    so A * 1 = 1e-3 in every row."""
    A = gen.poisson3d_var(12)
    assert oracle.is_symmetric(A)
    ones = np.ones(A.n_cols)
    y = oracle.sym_spmv(oracle.sym_build(A), ones)
    scale = oracle.abs_scale(A, ones)
    assert np.all(np.abs(y - 1e-3) <= TOL * scale)


def test_generated_workloads_are_symmetric():
    assert oracle.is_symmetric(gen.eigen_shaped(20000, window=1 << 12))
    assert oracle.is_symmetric(gen.poisson3d_var(9))
    assert not oracle.is_symmetric(gen.powerlaw(2000, seed=3))
