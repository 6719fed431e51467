"""The index structures the library builds (SELL-C-sigma, local/halo split) equal
the oracle's builders byte for byte, and the split product with its overlapped
halo copy matches the oracle."""
import json
import os

import numpy as np
import pytest

import gen
import oracle
from gpu_util import TOL_FP64, assert_close, dev, host

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def sell_equal(got: dict, ref: oracle.Sell):
    assert np.array_equal(got["perm"], ref.perm)
    assert np.array_equal(got["chunk_ptr"], ref.chunk_ptr)
    assert np.array_equal(got["chunk_len"], ref.chunk_len)
    assert np.array_equal(got["sell_col"], ref.sell_col)
    assert got["sell_val"].tobytes() == ref.sell_val.tobytes()


def test_sell_hand_example(lib):
    d = json.load(open(os.path.join(GOLD, "sell_example.json")))
    rp = np.array(d["row_ptr"], np.int32)
    A = gen.CSR(len(rp) - 1, 6, rp, np.array(d["col_idx"], np.int32), np.array(d["val"]))
    # the library's chunk height is 32, so compare with the oracle at C = 32
    with lib.Plan.from_csr(A, variant=lib.SPMV_SELL, sell_sigma=d["sigma"]) as p:
        sell_equal(p.sell_export(), oracle.sell_build(A, 32, d["sigma"]))


@pytest.mark.parametrize("sigma", [1, 256, 4096, 100000])
@pytest.mark.parametrize("name", ["eigen", "powerlaw", "ragged"])
def test_sell_bit_exact(lib, name, sigma):
    A = {"eigen": lambda: gen.eigen_shaped(60_000, window=1 << 15),
         "powerlaw": lambda: gen.powerlaw(20_000, seed=2),
         "ragged": lambda: gen.random_csr(2011, 1500, 0.01, 3, empty_rows=0.3, duplicates=True,
                                          unsorted=True)}[name]()
    with lib.Plan.from_csr(A, variant=lib.SPMV_SELL, sell_sigma=sigma) as p:
        info = p.info()
        ref = oracle.sell_build(A, 32, sigma)
        assert info.sell_slots == int(ref.chunk_ptr[-1]) and info.sell_chunks == ref.n_chunks
        sell_equal(p.sell_export(), ref)


def split_equal(got: dict, ref: oracle.Split):
    for key in ("loc_row_ptr", "loc_col", "halo_rows", "halo_row_ptr", "halo_col"):
        assert np.array_equal(got[key], getattr(ref, key)), key
    for key in ("loc_val", "halo_val"):
        assert got[key].tobytes() == getattr(ref, key).tobytes(), key


@pytest.mark.parametrize("frac", [0.0, 0.1, 0.5, 1.0])
def test_split_bit_exact(lib, frac):
    A = gen.poisson3d_var(30)
    h = A.n_cols - int(A.n_cols * frac)
    with lib.Plan.from_csr(A, halo_begin=h) as p:
        ref = oracle.split_build(A, h)
        assert p.info().n_halo_rows == len(ref.halo_rows)
        split_equal(p.split_export(), ref)


def run_split(lib, p, A, B, h, two_streams=True):
    import torch
    Bd = dev(B.copy())
    Bd[h:] = float("nan")                           # the halo part arrives only through the copy
    halo = torch.from_numpy(B[h:].copy()).pin_memory()
    C = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    cs = torch.cuda.Stream() if two_streams else None
    p.apply_split(Bd, halo, C, torch.cuda.current_stream(), cs)
    p.check()
    assert np.array_equal(host(Bd), B)
    return host(C)


@pytest.mark.parametrize("two_streams", [True, False])
@pytest.mark.parametrize("fp32", [False, True])
def test_split_product(lib, two_streams, fp32):
    A = gen.poisson3d_var(40)
    h = A.n_cols - A.n_cols // 10
    B = gen.uniform(A.n_cols, seed=5)
    with lib.Plan.from_csr(A, halo_begin=h, val_fp32=fp32) as p:
        y = run_split(lib, p, A, B, h, two_streams)
    if fp32:
        A32 = gen.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.val.astype(np.float32).astype(np.float64))
        ref = oracle.split_spmv(A.n_rows, oracle.split_build(A32, h), B)
        assert oracle.max_err_ratio(y, ref, oracle.abs_scale(A, B), TOL_FP64) <= 1.0
        assert_close(y, A, B, tol=2e-7)
    else:
        ref = oracle.split_spmv(A.n_rows, oracle.split_build(A, h), B)
        assert oracle.max_err_ratio(y, ref, oracle.abs_scale(A, B), TOL_FP64) <= 1.0
        assert_close(y, A, B)


@pytest.mark.parametrize("vname", ["SPMV_CRS_STAGED", "SPMV_CRS_L1", "SPMV_CRS_L8", "SPMV_SELL", "SPMV_SYM"])
def test_split_every_plan_variant(lib, vname):
    """The local pass runs the plan's CRS kernel (CRS_L1 for SELL and SYM
    plans); every choice gives the oracle's split product."""
    A = gen.poisson3d_var(30)
    h = A.n_cols - A.n_cols // 7
    B = gen.uniform(A.n_cols, seed=11)
    with lib.Plan.from_csr(A, halo_begin=h, variant=getattr(lib, vname), sell_sigma=64) as p:
        y = run_split(lib, p, A, B, h)
    ref = oracle.split_spmv(A.n_rows, oracle.split_build(A, h), B)
    assert oracle.max_err_ratio(y, ref, oracle.abs_scale(A, B), TOL_FP64) <= 1.0
    assert_close(y, A, B)


def test_split_integer_exact(lib):
    A = gen.random_csr(5000, 5000, 0.002, 9, integer=True, empty_rows=0.1)
    h = 4100
    B = np.random.default_rng(9).integers(-1024, 1025, A.n_cols).astype(np.float64)
    with lib.Plan.from_csr(A, halo_begin=h) as p:
        y = run_split(lib, p, A, B, h)
    assert np.array_equal(y, oracle.spmv(A, B))


def test_split_repeated_calls(lib):
    """Back-to-back split products on two streams reuse the plan's events safely."""
    import torch
    A = gen.poisson3d_var(36)
    h = A.n_cols - A.n_cols // 10
    with lib.Plan.from_csr(A, halo_begin=h) as p:
        cs = torch.cuda.Stream()
        Bd = dev(np.zeros(A.n_cols))
        C = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        for it in range(4):
            B = gen.uniform(A.n_cols, seed=100 + it)
            Bd[:h] = torch.from_numpy(B[:h]).cuda()
            halo = torch.from_numpy(B[h:].copy()).pin_memory()
            p.apply_split(Bd, halo, C, torch.cuda.current_stream(), cs)
            torch.cuda.current_stream().synchronize()
            assert_close(host(C), A, B)
        p.check()
