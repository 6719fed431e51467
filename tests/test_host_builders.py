"""The library's host-side format builders (SELL-C-sigma, local/halo split,
symmetric triangle), called through the C ABI without a device, equal the
oracle's builders byte for byte on ragged, duplicated, unsorted, empty and
full-structure matrices; bad input is refused with the documented status."""
import json
import os

import numpy as np
import pytest

import gen
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def spmv():
    from paper_1101_0091_gb300 import build
    build.build()
    import paper_1101_0091_gb300 as lib
    return lib


def empty(n_rows, n_cols):
    return gen.CSR(n_rows, n_cols, np.zeros(n_rows + 1, np.int32), np.zeros(0, np.int32), np.zeros(0))


MATS = {
    "ragged_dup_unsorted": lambda: gen.random_csr(2011, 1500, 0.01, 3, empty_rows=0.3, duplicates=True,
                                                  unsorted=True),
    "powerlaw": lambda: gen.powerlaw(20_000, seed=2),
    "eigen": lambda: gen.eigen_shaped(40_000, window=1 << 14),
    "poisson": lambda: gen.poisson3d_var(12),
    "all_rows_empty": lambda: empty(77, 50),
    "no_rows": lambda: empty(0, 10),
    "one_by_one": lambda: gen.CSR(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([-0.0])),
}


@pytest.mark.parametrize("sigma", [1, 32, 256, 4096, 1 << 20])
@pytest.mark.parametrize("name", sorted(MATS))
def test_sell_bytes_equal_oracle(spmv, name, sigma):
    A = MATS[name]()
    got = spmv.sell_build(A, sigma)
    ref = oracle.sell_build(A, 32, sigma)
    assert np.array_equal(got["perm"], ref.perm)
    assert np.array_equal(got["chunk_ptr"], ref.chunk_ptr)
    assert np.array_equal(got["chunk_len"], ref.chunk_len)
    assert np.array_equal(got["sell_col"], ref.sell_col)
    assert got["sell_val"].tobytes() == ref.sell_val.tobytes()


def test_sell_hand_example(spmv):
    d = json.load(open(os.path.join(GOLD, "sell_example.json")))
    rp = np.array(d["row_ptr"], np.int32)
    A = gen.CSR(len(rp) - 1, 6, rp, np.array(d["col_idx"], np.int32), np.array(d["val"]))
    got = spmv.sell_build(A, d["sigma"])
    ref = oracle.sell_build(A, 32, d["sigma"])
    assert np.array_equal(got["perm"], ref.perm) and np.array_equal(got["chunk_len"], ref.chunk_len)
    assert got["sell_val"].tobytes() == ref.sell_val.tobytes()


@pytest.mark.parametrize("frac", [0.0, 0.1, 0.5, 1.0])
@pytest.mark.parametrize("name", ["ragged_dup_unsorted", "powerlaw", "poisson", "all_rows_empty", "no_rows"])
def test_split_bytes_equal_oracle(spmv, name, frac):
    A = MATS[name]()
    h = int(round(A.n_cols * (1 - frac)))
    got = spmv.split_build(A, h)
    ref = oracle.split_build(A, h)
    for key in ("loc_row_ptr", "loc_col", "halo_rows", "halo_row_ptr", "halo_col"):
        assert np.array_equal(got[key], getattr(ref, key)), key
    for key in ("loc_val", "halo_val"):
        assert got[key].tobytes() == getattr(ref, key).tobytes(), key


def sym_case(seed, n, duplicates=False, shuffle=False, empty_rows=0.0, density=None):
    density = density if density is not None else min(1.0, 6.0 / max(n, 1))
    A = gen.random_csr(n, n, density, seed, empty_rows=empty_rows, duplicates=duplicates)
    return gen.symmetric_from(A, seed=seed, shuffle=shuffle)


SYM = {
    "laplace": lambda: gen.laplace2d(40),
    "poisson": lambda: gen.poisson3d_var(12),
    "eigen": lambda: gen.eigen_shaped(30_000, window=1 << 13),
    "ragged_dup_shuffled": lambda: sym_case(3, 3001, duplicates=True, shuffle=True, empty_rows=0.2),
    "dense_rows": lambda: sym_case(4, 300, density=0.5),
    "diagonal_only": lambda: gen.CSR(5, 5, np.arange(6, dtype=np.int32), np.arange(5, dtype=np.int32),
                                     np.arange(5, dtype=np.float64)),
    "all_rows_empty": lambda: empty(9, 9),
}


@pytest.mark.parametrize("name", sorted(SYM))
def test_sym_bytes_equal_oracle(spmv, name):
    A = SYM[name]()
    got = spmv.sym_build(A)
    ref = oracle.sym_build(A)
    assert np.array_equal(got["row_ptr"], ref.row_ptr)
    assert np.array_equal(got["col"], ref.col)
    assert got["val"].tobytes() == ref.val.tobytes()


def test_refusals(spmv):
    A = gen.poisson3d_var(6)
    bad = gen.CSR(A.n_rows, A.n_cols, A.row_ptr.copy(), A.col_idx.copy(), A.val)
    bad.col_idx[5] = A.n_cols                       # column out of range
    for call in (lambda: spmv.sell_build(bad, 1), lambda: spmv.split_build(bad, 10), lambda: spmv.sym_build(bad)):
        with pytest.raises(spmv.SpmvError) as e:
            call()
        assert e.value.status == 2                  # SPMV_ERR_CSR
    with pytest.raises(spmv.SpmvError) as e:
        spmv.sell_build(A, 0)
    assert e.value.status == 1                      # SPMV_ERR_ARG: sigma < 1
    for h in (-1, A.n_cols + 1):
        with pytest.raises(spmv.SpmvError) as e:
            spmv.split_build(A, h)
        assert e.value.status == 1                  # SPMV_ERR_ARG: h out of range
    U = gen.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.val.copy())
    U.val[3] += 1.0                                 # an entry no longer matches its mirror
    with pytest.raises(spmv.SpmvError) as e:
        spmv.sym_build(U)
    assert e.value.status == 6                      # SPMV_ERR_UNSUPPORTED
    R = gen.random_csr(30, 40, 0.1, 1)
    with pytest.raises(spmv.SpmvError) as e:
        spmv.sym_build(R)                           # not square
    assert e.value.status == 6
