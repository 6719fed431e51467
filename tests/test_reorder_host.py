"""The library's host-side reordering (RCM permutation, symmetric CRS
permutation) equals the oracle's byte for byte; invalid inputs are rejected.
Host code only: runs without a GPU."""
import numpy as np
import pytest

import gen
from oracle import reorder as oreorder


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1101_0091_gb300 as m
    return m


CASES = {
    "laplace": lambda: gen.laplace2d(20),
    "poisson": lambda: gen.poisson3d_var(7),
    "eigen": lambda: gen.eigen_shaped(4000, window=1 << 9),
    "random_sym": lambda: gen.symmetric_from(gen.random_csr(500, 500, 0.01, 3, duplicates=True), seed=3,
                                             shuffle=True),
    "unsymmetric_pattern": lambda: gen.random_csr(400, 400, 0.01, 5, empty_rows=0.2),
    "shuffled_grid": lambda: oreorder.permute_csr(gen.laplace2d(15),
                                                  np.random.default_rng(1).permutation(225).astype(np.int32)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_rcm_bit_exact(lib, name):
    A = CASES[name]()
    perm = lib.rcm(A.n_rows, A.row_ptr, A.col_idx)
    assert np.array_equal(perm, oreorder.rcm(A))


@pytest.mark.parametrize("name", sorted(CASES))
def test_permute_csr_bit_exact(lib, name):
    A = CASES[name]()
    perm = oreorder.rcm(A)
    rp, ci, va = lib.permute_csr(A.n_rows, A.row_ptr, A.col_idx, A.val, perm)
    ref = oreorder.permute_csr(A, perm)
    assert np.array_equal(rp, ref.row_ptr) and np.array_equal(ci, ref.col_idx)
    assert va.tobytes() == ref.val.tobytes()


def test_bad_inputs(lib):
    A = gen.laplace2d(4)
    with pytest.raises(lib.SpmvError):
        lib.permute_csr(A.n_rows, A.row_ptr, A.col_idx, A.val, np.zeros(A.n_rows, np.int32))
    with pytest.raises(lib.SpmvError):
        lib.permute_csr(A.n_rows, A.row_ptr, A.col_idx, A.val, np.arange(1, A.n_rows + 1, dtype=np.int32))
    bad = A.col_idx.copy()
    bad[0] = A.n_rows
    with pytest.raises(lib.SpmvError):
        lib.rcm(A.n_rows, A.row_ptr, bad)
    assert lib.rcm(0, np.zeros(1, np.int32), np.zeros(0, np.int32)).size == 0
