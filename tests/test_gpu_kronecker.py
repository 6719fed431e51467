"""The HMeP / HMEp numberings of Sec. 1.3.1 on the GPU.  The eigenproblem-shaped
matrix lives on an n1 x n2 product basis (400 x n2); its Kronecker-transposed
numbering (the second factor contiguous -> the first factor contiguous) is the
permutation perm[p*n1 + e] = e*n2 + p.  Products through the renumbered matrix
P A P^T (built by spmv_permute_csr) with the CRS_L1 and SELL plans, and
through spmv_reorder's gather of B and scatter of C, match the oracle's CRS
loop element by element: at 1e-13 * sum|a b| on random values, bit for bit on
integer values, on a small basis and on the full 400 x 15,504 matrix (sampled
rows)."""
import numpy as np
import pytest

import gen
import oracle
from oracle import reorder as oreorder
from gpu_util import TOL_FP64, assert_close, dev, host

pytestmark = pytest.mark.gpu

N1 = 400
PLANS = [("crs_l1", 2, 1), ("sell_s256", 8, 256), ("sell_s4096", 8, 4096)]


def index_map(n1, n2):
    """perm[new] = old of the renumbering, from its definition e*n2 + p -> p*n1 + e."""
    q = np.arange(n1 * n2, dtype=np.int64)
    return ((q % n1) * n2 + q // n1).astype(np.int32)


def through_renumbered(lib, A, Ap, perm, B, variant, sigma):
    """(C_renumbered, C_original): P A P^T times the gathered B, and that result
    scattered back to the original numbering."""
    import torch
    k = 1 if B.ndim == 1 else B.shape[1]
    with lib.Plan(Ap.n_rows, Ap.n_cols, Ap.row_ptr, Ap.col_idx, Ap.val, variant=variant, sell_sigma=sigma) as p, \
            lib.Reorder(perm) as r:
        Bd = dev(B.reshape(A.n_rows, k))
        Bp = torch.full_like(Bd, float("nan"))
        Cp = torch.full_like(Bd, float("nan"))
        C = torch.full_like(Bd, float("nan"))
        r.gather(Bd, Bp)
        p.apply_block(Bp, Cp, k)
        r.scatter(Cp, C)
        p.check()
        return host(Cp).reshape(B.shape), host(C).reshape(B.shape)


def renumbered(lib, A, perm):
    rp, ci, va = lib.permute_csr(A.n_rows, A.row_ptr, A.col_idx, A.val, perm)
    return gen.CSR(A.n_rows, A.n_cols, rp, ci, va)


@pytest.mark.parametrize("integer", [False, True])
def test_kronecker_numbering_small_basis(lib, integer):
    n2 = 40
    A = gen.eigen_shaped(N1 * n2, window=1 << 13)
    if integer:
        A.val = np.random.default_rng(3).integers(-1024, 1025, A.nnz).astype(np.float64)
    perm = gen.kronecker_transpose(N1, n2)
    assert np.array_equal(perm, index_map(N1, n2))
    Ap = renumbered(lib, A, perm)
    ref = oreorder.permute_csr(A, perm)                 # the oracle's P A P^T, byte for byte
    assert np.array_equal(Ap.row_ptr, ref.row_ptr) and np.array_equal(Ap.col_idx, ref.col_idx)
    assert np.array_equal(Ap.val.view(np.uint64), ref.val.view(np.uint64))
    for k in (1, 4):
        if integer:
            B = np.random.default_rng(k).integers(-1024, 1025, (A.n_cols, k)).astype(np.float64)
        else:
            B = gen.rhs_block(A.n_cols, k, seed=k)
        B = B[:, 0].copy() if k == 1 else B
        Bp = B[perm]
        for name, variant, sigma in PLANS:
            yp, y = through_renumbered(lib, A, Ap, perm, B, variant, sigma)
            assert_close(yp, Ap, Bp, exact=integer)     # the renumbered product itself
            assert_close(y, A, B, exact=integer)        # back in the original numbering
            assert np.array_equal(yp, y[perm])          # the scatter only moves rows


def test_kronecker_numbering_full_eigenproblem(lib):
    """Full 400 x 15,504 basis (6,201,600 rows): the product through the
    Kronecker-transposed numbering against the oracle on 20,600 sampled rows
    (first and last 300 and 20,000 at random), for CRS_L1 and SELL-32-4096."""
    A = gen.eigen_shaped()
    n2 = A.n_rows // N1
    perm = gen.kronecker_transpose(N1, n2)
    assert A.n_rows == N1 * 15_504 and np.array_equal(perm, index_map(N1, n2))
    Ap = renumbered(lib, A, perm)
    B = gen.uniform(A.n_cols, seed=0)
    rows = np.unique(np.concatenate([np.arange(300), np.arange(A.n_rows - 300, A.n_rows),
                                     np.random.default_rng(11).integers(0, A.n_rows, 20_000)]))
    lens = (A.row_ptr[rows + 1] - A.row_ptr[rows]).astype(np.int64)
    rp = np.zeros(len(rows) + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    idx = np.concatenate([np.arange(A.row_ptr[r], A.row_ptr[r + 1]) for r in rows])
    S = gen.CSR(len(rows), A.n_cols, rp.astype(np.int32), A.col_idx[idx], A.val[idx])
    ref, scale = oracle.spmv(S, B), oracle.abs_scale(S, B)
    for name, variant, sigma in (PLANS[0], PLANS[2]):
        yp, y = through_renumbered(lib, A, Ap, perm, B, variant, sigma)
        assert not np.isnan(y).any()
        assert oracle.max_err_ratio(y[rows], ref, scale, TOL_FP64) <= 1.0, name
        assert np.array_equal(yp, y[perm])
