"""Reordering on the GPU: the device gather/scatter of k-column blocks equals
numpy indexing bit for bit, and a product through the RCM-permuted plan
(gather B, multiply, scatter C) matches the oracle's product of the original
matrix, at small sizes and on the full eigenproblem-shaped workload."""
import numpy as np
import pytest

import gen
import oracle
from oracle import reorder as oreorder
from gpu_util import TOL_FP64, assert_close, dev, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k,ld", [(1, 1), (3, 3), (4, 6)])
def test_gather_scatter_bit_exact(lib, k, ld):
    import torch
    n = 10_007
    perm = np.random.default_rng(k).permutation(n).astype(np.int32)
    X = np.random.default_rng(9).standard_normal((n, ld))
    Xd = dev(X)
    Y = torch.full((n, ld), 5.5, dtype=torch.float64, device="cuda")
    with lib.Reorder(perm) as r:
        r.gather(Xd[:, :k], Y[:, :k])
        Yh = host(Y)
        assert np.array_equal(Yh[:, :k], X[perm, :k]) and np.all(Yh[:, k:] == 5.5)
        Z = torch.full((n, ld), 5.5, dtype=torch.float64, device="cuda")
        r.scatter(Y[:, :k], Z[:, :k])
        assert np.array_equal(host(Z)[:, :k], X[:, :k])


def test_reorder_rejects_non_permutations(lib):
    with pytest.raises(lib.SpmvError):
        lib.Reorder(np.array([0, 0, 1], np.int32))
    with pytest.raises(lib.SpmvError):
        lib.Reorder(np.array([0, 3, 1], np.int32))


def product_through_rcm(lib, A, B, variant=None, sigma=1):
    import torch
    perm = lib.rcm(A.n_rows, A.row_ptr, A.col_idx)
    rp, ci, va = lib.permute_csr(A.n_rows, A.row_ptr, A.col_idx, A.val, perm)
    k = 1 if B.ndim == 1 else B.shape[1]
    kw = {} if variant is None else {"variant": variant, "sell_sigma": sigma}
    with lib.Plan(A.n_rows, A.n_cols, rp, ci, va, **kw) as p, lib.Reorder(perm) as r:
        Bd = dev(B.reshape(A.n_rows, k))
        Bp = torch.empty_like(Bd)
        Cp = torch.empty_like(Bd)
        C = torch.full_like(Bd, float("nan"))
        r.gather(Bd, Bp)
        p.apply_block(Bp, Cp, k)
        r.scatter(Cp, C)
        return host(C).reshape(B.shape), perm


@pytest.mark.parametrize("name", ["laplace", "eigen", "ragged"])
def test_product_through_permuted_plan(lib, name):
    A = {"laplace": lambda: gen.laplace2d(40),
         "eigen": lambda: gen.eigen_shaped(30_000, window=1 << 13),
         "ragged": lambda: gen.symmetric_from(gen.random_csr(3000, 3000, 0.003, 4, integer=True, empty_rows=0.2),
                                              seed=4, shuffle=True)}[name]()
    B = gen.uniform(A.n_cols, seed=2)
    y, perm = product_through_rcm(lib, A, B)
    assert np.array_equal(perm, oreorder.rcm(A))
    assert_close(y, A, B)
    Bk = gen.rhs_block(A.n_cols, 4, seed=3)
    yk, _ = product_through_rcm(lib, A, Bk, variant=lib.SPMV_SELL, sigma=256)
    assert_close(yk, A, Bk)


def test_integer_product_exact(lib):
    A = gen.symmetric_from(gen.random_csr(5000, 5000, 0.002, 6, integer=True, duplicates=True), seed=6)
    B = np.random.default_rng(6).integers(-1024, 1025, A.n_cols).astype(np.float64)
    y, _ = product_through_rcm(lib, A, B)
    assert_close(y, A, B, exact=True)


def test_eigen_full_rcm(lib):
    """Full eigenproblem-shaped workload: RCM permutation, sampled rows of the
    product through the permuted plan against the oracle."""
    A = gen.eigen_shaped()
    B = gen.uniform(A.n_cols, seed=0)
    y, perm = product_through_rcm(lib, A, B, variant=lib.SPMV_SELL, sigma=4096)
    assert sorted(perm[:1000].tolist()) == sorted(set(perm[:1000].tolist()))
    rows = np.unique(np.concatenate([np.arange(300), np.arange(A.n_rows - 300, A.n_rows),
                                     np.random.default_rng(7).integers(0, A.n_rows, 20_000)]))
    lens = (A.row_ptr[rows + 1] - A.row_ptr[rows]).astype(np.int64)
    rp = np.zeros(len(rows) + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    idx = np.concatenate([np.arange(A.row_ptr[r], A.row_ptr[r + 1]) for r in rows])
    S = gen.CSR(len(rows), A.n_cols, rp.astype(np.int32), A.col_idx[idx], A.val[idx])
    ref = oracle.spmv(S, B)
    assert oracle.max_err_ratio(y[rows], ref, oracle.abs_scale(S, B), TOL_FP64) <= 1.0
