"""Pins of the oracle's SELL-C-sigma and local/halo split builders: hand-worked
examples, structural properties checked by independent code, and exact
agreement of the products with the CRS loop."""
import json
import os

import numpy as np
import pytest

import gen
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def csr_of(d):
    rp = np.array(d["row_ptr"], np.int32)
    return gen.CSR(len(rp) - 1, 6, rp, np.array(d["col_idx"], np.int32), np.array(d["val"], np.float64))


def test_sell_hand_example():
    d = load("sell_example.json")
    S = oracle.sell_build(csr_of(d), C=d["C"], sigma=d["sigma"])
    assert S.perm.tolist() == d["perm"]
    assert S.chunk_len.tolist() == d["chunk_len"]
    assert S.chunk_ptr.tolist() == d["chunk_ptr"]
    assert S.sell_col.tolist() == d["sell_col"]
    assert S.sell_val.tolist() == d["sell_val"]
    assert S.beta == pytest.approx(9 / 14)


def sell_properties(A, S, C, sigma):
    n = A.n_rows
    L = np.diff(A.row_ptr)
    assert sorted(S.perm.tolist()) == list(range(n))
    for w0 in range(0, n, sigma):
        w = S.perm[w0:w0 + sigma]
        assert sorted(w.tolist()) == list(range(w0, min(w0 + sigma, n)))  # stays in its window
        lw = L[w]
        assert np.all(lw[:-1] >= lw[1:])                                   # descending
        for a in range(len(w) - 1):                                        # stable on ties
            if lw[a] == lw[a + 1]:
                assert w[a] < w[a + 1]
    nc = (n + C - 1) // C
    assert len(S.chunk_len) == nc
    for c in range(nc):
        rows = S.perm[c * C:(c + 1) * C]
        assert S.chunk_len[c] == (L[rows].max() if len(rows) else 0)
        assert S.chunk_ptr[c + 1] - S.chunk_ptr[c] == C * S.chunk_len[c]
    # rebuild every row from the column-major slots and compare with CRS
    for c in range(nc):
        for t in range(C):
            r = c * C + t
            slots = S.chunk_ptr[c] + np.arange(S.chunk_len[c]) * C + t
            if r >= n:
                assert np.all(S.sell_val[slots] == 0.0) and np.all(S.sell_col[slots] == 0)
                continue
            o = S.perm[r]
            a, b = A.row_ptr[o], A.row_ptr[o + 1]
            ln = b - a
            assert np.array_equal(S.sell_col[slots[:ln]], A.col_idx[a:b])
            assert np.array_equal(S.sell_val[slots[:ln]], A.val[a:b])
            pad = slots[ln:]
            assert np.all(S.sell_val[pad] == 0.0) and not np.signbit(S.sell_val[pad]).any()
            assert np.all(S.sell_col[pad] == (A.col_idx[b - 1] if ln > 0 else 0))


@pytest.mark.parametrize("C,sigma", [(32, 1), (32, 256), (32, 4096), (4, 3), (8, 1000)])
def test_sell_properties_random(C, sigma):
    A = gen.csr_from_lengths(np.random.default_rng(C + sigma).integers(0, 40, 1000), 700, seed=3)
    S = oracle.sell_build(A, C=C, sigma=sigma)
    sell_properties(A, S, C, sigma)


def test_sell_product_equals_crs_bitwise():
    """Same per-row summation order; padding adds +0.0 to a sum that starts at
    +0.0, so the SELL product equals the CRS loop bit for bit."""
    A = gen.eigen_shaped(5000, seed=1, window=1 << 10)
    B = gen.uniform(A.n_cols, seed=1)
    ref = oracle.spmv(A, B)
    for sigma in (1, 256, 4096):
        S = oracle.sell_build(A, 32, sigma)
        assert np.array_equal(oracle.sell_spmv(S, B), ref)


def test_sell_sigma_improves_fill():
    """Sorting inside sigma-windows can only lower the padding of the chunks."""
    A = gen.eigen_shaped(20000, seed=0, window=1 << 12)
    betas = [oracle.sell_build(A, 32, s).beta for s in (1, 256, 4096)]
    assert betas[0] <= betas[1] <= betas[2] <= 1.0
    assert betas[2] > 0.97


def test_split_hand_example():
    d = load("split_example.json")
    S = oracle.split_build(csr_of(d), d["h"])
    for key in ("loc_row_ptr", "loc_col", "loc_val", "halo_rows", "halo_row_ptr", "halo_col", "halo_val"):
        assert getattr(S, key).tolist() == d[key], key


@pytest.mark.parametrize("h", [0, 1, 350, 699, 700])
def test_split_reconstructs_matrix(h):
    A = gen.random_csr(500, 700, 0.02, 21, empty_rows=0.1, duplicates=True, unsorted=True)
    S = oracle.split_build(A, h)
    hr = set(S.halo_rows.tolist())
    assert S.halo_rows.tolist() == sorted(hr)
    k = 0
    for i in range(A.n_rows):
        row = list(zip(A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]].tolist(), A.val[A.row_ptr[i]:A.row_ptr[i + 1]].tolist()))
        loc = list(zip(S.loc_col[S.loc_row_ptr[i]:S.loc_row_ptr[i + 1]].tolist(),
                       S.loc_val[S.loc_row_ptr[i]:S.loc_row_ptr[i + 1]].tolist()))
        assert loc == [e for e in row if e[0] < h]
        far = [e for e in row if e[0] >= h]
        assert (i in hr) == (len(far) > 0)
        if far:
            assert S.halo_rows[k] == i
            got = list(zip(S.halo_col[S.halo_row_ptr[k]:S.halo_row_ptr[k + 1]].tolist(),
                           S.halo_val[S.halo_row_ptr[k]:S.halo_row_ptr[k + 1]].tolist()))
            assert got == far
            k += 1
    assert k == len(S.halo_rows)


def test_split_product():
    A = gen.random_csr(400, 400, 0.03, 8, integer=True)
    B = np.random.default_rng(8).integers(-1024, 1025, 400).astype(np.float64)
    S = oracle.split_build(A, 360)
    assert np.array_equal(oracle.split_spmv(A.n_rows, S, B), oracle.spmv(A, B))  # exact integers
    A = gen.poisson3d_var(12)
    B = gen.uniform(A.n_cols)
    S = oracle.split_build(A, A.n_cols - A.n_cols // 10)
    y = oracle.split_spmv(A.n_rows, S, B)
    assert oracle.max_err_ratio(y, oracle.spmv(A, B), oracle.abs_scale(A, B), 1e-13) <= 1.0
