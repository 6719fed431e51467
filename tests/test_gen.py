"""The seeded input generators produce the workloads' stated shapes and structure."""
import numpy as np
import pytest

import gen


def check_csr(A, sorted_cols=True, distinct=True):
    assert A.row_ptr[0] == 0 and np.all(np.diff(A.row_ptr) >= 0) and A.row_ptr[-1] == len(A.col_idx)
    assert len(A.val) == len(A.col_idx)
    if A.nnz:
        assert A.col_idx.min() >= 0 and A.col_idx.max() < A.n_cols
    for i in range(0, A.n_rows, max(1, A.n_rows // 500)):
        c = A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]
        if sorted_cols:
            assert np.all(np.diff(c) > 0 if distinct else np.diff(c) >= 0)


def test_laplace2d_shape():
    A = gen.laplace2d(256)
    check_csr(A)
    assert (A.n_rows, A.nnz) == (65536, 326656)
    assert set(np.unique(A.val).tolist()) == {-1.0, 4.0}


def test_poisson3d_shape_and_values():
    n = 10
    A = gen.poisson3d_var(n)
    check_csr(A)
    assert A.nnz == 7 * n ** 3 - 6 * n * n
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    off = A.col_idx != rows
    assert np.all(A.val[off] <= -1.0) and np.all(A.val[off] > -2.0)
    d = A.val[~off]
    offsum = np.zeros(A.n_rows)
    np.add.at(offsum, rows[off], -A.val[off])
    assert np.allclose(d, offsum + 1e-3, rtol=1e-15, atol=1e-15)
    offsets = set(np.unique(A.col_idx - rows).tolist())
    assert offsets == {-n * n, -n, -1, 0, 1, n, n * n}


def test_poisson3d_full_size_count():
    """The 280^3 workload has 21,952,000 rows and 153,193,600 nonzeros (closed form)."""
    n = 280
    assert n ** 3 == 21_952_000 and 7 * n ** 3 - 6 * n * n == 153_193_600


def test_eigen_shaped_structure():
    N, W = 50000, 1 << 14
    A = gen.eigen_shaped(N, seed=0, window=W)
    check_csr(A)
    rows = np.repeat(np.arange(N), np.diff(A.row_ptr))
    d = A.col_idx - rows
    assert np.abs(d).max() <= W
    # expected Nnzr = 1 + 2*2*0.7 + 2*5 = 13.8 (minus a thin edge effect)
    assert abs(A.nnz / N - 13.8) < 0.1
    assert np.all(np.diff(A.row_ptr) >= 1)          # every row has its diagonal
    band = (np.abs(d) >= 1) & (np.abs(d) <= 2)
    assert abs(band.sum() / (4 * N) - 0.7) < 0.01
    assert np.all(np.abs(A.val[d != 0]) <= 1.0)
    assert 400 * 15504 == 6_201_600                  # the full-size dimension (Sec. 1.3.1)


def test_powerlaw_batch_members():
    ms = [gen.powerlaw_batch_member(m) for m in range(6)]
    for A in ms:
        check_csr(A)
        assert 1000 <= A.n_rows <= 200000
        L = A.row_lengths()
        assert L.min() >= 1 and L.max() <= min(2000, A.n_rows)
    # deterministic, and members differ
    again = gen.powerlaw_batch_member(3)
    assert np.array_equal(again.col_idx, ms[3].col_idx) and np.array_equal(again.val, ms[3].val)
    assert ms[0].n_rows != ms[1].n_rows


def test_powerlaw_mean_length():
    """Truncated discrete power law alpha = 2.2 on [1, 2000] has mean ~3.0."""
    A = gen.powerlaw(200000, seed=5)
    L = np.arange(1, 2001, dtype=np.float64)
    w = L ** -2.2
    mean = (L * w).sum() / w.sum()
    assert abs(A.nnz / A.n_rows - mean) < 0.1
    assert abs(mean - 3.02) < 0.05


def test_uniform_rhs():
    v = gen.uniform(100000, seed=0)
    assert v.min() >= -1.0 and v.max() < 1.0 and abs(v.mean()) < 0.01
    assert np.array_equal(v, gen.uniform(100000, seed=0))
    assert not np.array_equal(v[:100], gen.uniform(100, seed=1))


def test_kronecker_transpose_is_the_index_map():
    """Sec. 1.3.1: the two numberings of the n1 x n2 product basis differ in
    which factor is contiguous.  The renumbering takes old index e*n2 + p to
    new index p*n1 + e, so perm[new] = old is perm[p*n1 + e] = e*n2 + p.
    Pinned by a hand-worked 2 x 3 case, by the map written out with loops,
    and by the inverse map decoded from the new index (q = p*n1 + e)."""
    # 2 x 3: old (e, p) -> new p*2 + e: (0,0)->0 (1,0)->1 (0,1)->2 (1,1)->3 (0,2)->4 (1,2)->5
    assert gen.kronecker_transpose(2, 3).tolist() == [0, 3, 1, 4, 2, 5]
    for n1, n2 in ((3, 5), (400, 7), (7, 400)):
        perm = gen.kronecker_transpose(n1, n2)
        ref = np.empty(n1 * n2, np.int64)
        for e in range(n1):
            for p in range(n2):
                ref[p * n1 + e] = e * n2 + p
        assert np.array_equal(perm, ref)
        assert np.array_equal(np.sort(perm), np.arange(n1 * n2))      # a permutation
    n1, n2 = 400, 15_504                                             # the full eigenproblem basis
    perm = gen.kronecker_transpose(n1, n2)
    q = np.arange(n1 * n2, dtype=np.int64)
    assert perm.dtype == np.int32 and np.array_equal(perm, (q % n1) * n2 + q // n1)
    inv = np.empty_like(q)
    inv[perm] = q
    old = np.arange(n1 * n2, dtype=np.int64)
    assert np.array_equal(inv, (old % n2) * n1 + old // n2)          # old e*n2 + p sits at p*n1 + e
