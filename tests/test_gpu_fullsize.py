"""Parity at the full workload sizes, in the launch configuration the benchmark
times, on sampled rows the oracle computes one by one (the oracle runs the
same row loop on the sampled rows only)."""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import TOL_FP32VAL, TOL_FP64, dev, host

pytestmark = pytest.mark.gpu


def sample_rows(n, seed, count=30_000, edge=500):
    rng = np.random.default_rng(seed)
    rows = np.concatenate([np.arange(min(edge, n)), np.arange(max(0, n - edge), n), rng.integers(0, n, count)])
    return np.unique(rows)


def sub_csr(A, rows):
    lens = (A.row_ptr[rows + 1] - A.row_ptr[rows]).astype(np.int64)
    rp = np.zeros(len(rows) + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    idx = np.concatenate([np.arange(A.row_ptr[r], A.row_ptr[r + 1]) for r in rows]) if len(rows) else np.zeros(0, int)
    return gen.CSR(len(rows), A.n_cols, rp.astype(np.int32), A.col_idx[idx], A.val[idx])


def check_sampled(y, A, B, rows, tol=TOL_FP64, f32val=False):
    S = sub_csr(A, rows)
    if f32val:
        ref = oracle.spmm(S, B.reshape(-1, 1), f32val=True)[:, 0]
    else:
        ref = oracle.spmv(S, B)
    r = oracle.max_err_ratio(y[rows], ref, oracle.abs_scale(S, B), tol)
    assert r <= 1.0, r
    return r


@pytest.fixture(scope="module")
def poisson280():
    return gen.poisson3d_var(280)


def test_poisson280_staged_and_split(lib, poisson280):
    import torch
    A = poisson280
    assert (A.n_rows, A.nnz) == (21_952_000, 153_193_600)
    B = gen.uniform(A.n_cols, seed=0)
    h = A.n_cols - A.n_cols // 10
    rows = sample_rows(A.n_rows, 1)
    with lib.Plan.from_csr(A, halo_begin=h) as p:
        Bd = dev(B)
        C = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
        p.apply(Bd, C)                         # the plan's default kernel (CRS_L1 on this stencil)
        p.check()
        y = host(C)
        assert p.info().variant == lib.SPMV_CRS_L1 and not np.isnan(y).any()
        check_sampled(y, A, B, rows)
        # CRS_STAGED (bulk copies of each row block's tile + mbarrier) on every row: the whole
        # product against the oracle's loop, and bit for bit against CRS_L1 where rows are short
        p.set_variant(lib.SPMV_CRS_STAGED)
        C.fill_(float("nan"))
        p.apply(Bd, C)
        p.check()
        ys = host(C)
        assert not np.isnan(ys).any()
        ref = oracle.spmv(A, B)
        assert oracle.max_err_ratio(ys, ref, oracle.abs_scale(A, B), TOL_FP64) <= 1.0
        assert np.array_equal(ys, y)           # thread per row in both: the same summation order
        p.set_variant(lib.SPMV_CRS_L1)
        # split product with the halo copied from pinned host memory on a side stream
        halo = torch.from_numpy(B[h:].copy()).pin_memory()
        Bd[h:] = float("nan")
        C.fill_(float("nan"))
        p.apply_split(Bd, halo, C, torch.cuda.current_stream(), torch.cuda.Stream())
        p.check()
        y2 = host(C)
        assert not np.isnan(y2).any()
        check_sampled(y2, A, B, rows)


def test_poisson280_fp32_values(lib, poisson280):
    import torch
    A = poisson280
    B = gen.uniform(A.n_cols, seed=0)
    rows = sample_rows(A.n_rows, 2, count=10_000)
    with lib.Plan.from_csr(A, val_fp32=True) as p:
        C = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        p.apply(dev(B), C)
        p.check()
        y = host(C)
    r32 = check_sampled(y, A, B, rows, f32val=True)
    r64 = check_sampled(y, A, B, rows, tol=TOL_FP32VAL)
    print(f"poisson280 FP32 values: max |err| / (2e-7 sum|ab|) vs the FP64 oracle = {r64:.4f}; "
          f"vs the oracle's FP32-value loop / (1e-13 sum|ab|) = {r32:.4f}")


def test_eigen_full_staged_and_sell(lib):
    import torch
    A = gen.eigen_shaped()
    assert A.n_rows == 6_201_600
    B = gen.uniform(A.n_cols, seed=0)
    rows = sample_rows(A.n_rows, 3)
    with lib.Plan.from_csr(A) as p:
        Bd = dev(B)
        C = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        for vid, sigma in [(lib.SPMV_CRS_STAGED, 1), (lib.SPMV_SELL, 1), (lib.SPMV_SELL, 256),
                           (lib.SPMV_SELL, 4096), (lib.SPMV_CRS_L4, 1)]:
            p.set_variant(vid, sigma)
            C.fill_(float("nan"))
            p.apply(Bd, C)
            p.check()
            check_sampled(host(C), A, B, rows)


@pytest.mark.parametrize("fp32", [False, True])
def test_poisson280_symmetric(lib, poisson280, fp32):
    """Symmetric CRS on the full 3D Poisson workload: sampled rows of the product
    against the oracle's CRS loop over the full rows; A * 1 = 1e-3 in every row."""
    import torch
    A = poisson280
    B = gen.uniform(A.n_cols, seed=0)
    rows = sample_rows(A.n_rows, 4, count=10_000)
    with lib.Plan.from_csr(A, variant=lib.SPMV_SYM, val_fp32=fp32) as p:
        assert p.info().sym_nnz == (A.nnz + A.n_rows) // 2
        C = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
        p.apply(dev(B), C)
        y = host(C)
        assert not np.isnan(y).any()
        check_sampled(y, A, B, rows, f32val=fp32)
        if not fp32:
            ones = np.ones(A.n_cols)
            p.apply(dev(ones), C)
            y1 = host(C)
            S = sub_csr(A, rows)
            assert np.all(np.abs(y1[rows] - 1e-3) <= TOL_FP64 * oracle.abs_scale(S, ones))


@pytest.mark.parametrize("k", [2, 16])
def test_poisson280_spmm_column_split(lib, poisson280, k):
    """k right-hand sides on the full 3D Poisson workload through CRS_L1's
    column-split kernel (a full 16-byte aligned block, as the benchmark's
    SpMM section runs it), on sampled rows against the oracle's k-column loop;
    the same product from a block 8 bytes off alignment (thread-per-row
    scalar form) gives the same bits."""
    import torch
    A = poisson280
    B = gen.rhs_block(A.n_cols, k, seed=k)
    rows = sample_rows(A.n_rows, 6 + k, count=10_000)
    with lib.Plan.from_csr(A) as p:
        Bd = dev(B)
        C = torch.full((A.n_rows, k), float("nan"), dtype=torch.float64, device="cuda")
        p.apply_block(Bd, C, k)
        p.check()
        y = host(C)
        flat = torch.empty(A.n_rows * k + 1, dtype=torch.float64, device="cuda")
        Co = flat[1:].view(A.n_rows, k)
        p.apply_block(Bd, Co, k)
        same = bool(torch.equal(C, Co))
        del Bd, C, flat, Co
    assert same
    S = sub_csr(A, rows)
    ref = oracle.spmm(S, B)
    assert oracle.max_err_ratio(y[rows], ref, oracle.abs_scale(S, B), TOL_FP64) <= 1.0


def test_eigen_full_sell_spmm_k4(lib):
    """SELL-32-4096 with k = 4 on the eigenproblem-shaped workload (the column-split
    SELL kernel), on sampled rows."""
    import torch
    A = gen.eigen_shaped()
    k = 4
    B = gen.rhs_block(A.n_cols, k, seed=3)
    rows = sample_rows(A.n_rows, 9, count=10_000)
    with lib.Plan.from_csr(A, variant=lib.SPMV_SELL, sell_sigma=4096) as p:
        C = torch.full((A.n_rows, k), float("nan"), dtype=torch.float64, device="cuda")
        p.apply_block(dev(B), C, k)
        p.check()
        y = host(C)
    assert not np.isnan(y).any()
    S = sub_csr(A, rows)
    ref = oracle.spmm(S, B)
    assert oracle.max_err_ratio(y[rows], ref, oracle.abs_scale(S, B), TOL_FP64) <= 1.0


def test_eigen_full_symmetric(lib):
    import torch
    A = gen.eigen_shaped()
    B = gen.uniform(A.n_cols, seed=0)
    rows = sample_rows(A.n_rows, 5)
    with lib.Plan.from_csr(A, variant=lib.SPMV_SYM) as p:
        C = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
        p.apply(dev(B), C)
        y = host(C)
        assert not np.isnan(y).any()
        check_sampled(y, A, B, rows)


def test_batch512_full_size_sampled(lib):
    """The 512-member uneven batch, k = 4, in the configuration the benchmark
    times (sorted policy, autotuned, graph replay), on 40 sampled rows per
    member plus every row of the members' longest rows."""
    import torch
    As = [gen.powerlaw_batch_member(m) for m in range(512)]
    Bs = [gen.rhs_block(A.n_cols, 4, seed=0, stream=2 * m + 1) for m, A in enumerate(As)]
    plans = [lib.Plan.from_csr(A) for A in As]
    Bd = [dev(B) for B in Bs]
    Cd = [torch.full((A.n_rows, 4), float("nan"), dtype=torch.float64, device="cuda") for A in As]
    with lib.Batch(plans, 4, [lib.SPMV_BATCH_SORTED] * len(As)) as b:
        b.set_io(Bd, Cd)
        b.autotune(reps=1)
        for _ in range(2):
            b.apply()
        torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    for m, (A, B, C) in enumerate(zip(As, Bs, Cd)):
        y = host(C)
        assert not np.isnan(y).any(), m
        L = A.row_lengths()
        rows = np.unique(np.concatenate([rng.integers(0, A.n_rows, 40), np.argsort(L)[-3:]]))
        S = sub_csr(A, rows)
        ref = oracle.spmm(S, B)
        assert oracle.max_err_ratio(y[rows], ref, oracle.abs_scale(S, B), TOL_FP64) <= 1.0, m
    for p in plans:
        p.close()


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("k", [1, 4, 8, 16])
def test_laplace256_block_precision(lib, k, fp32):
    """The 2D Laplacian workload with k right-hand sides, FP64 vs FP32 values:
    its values (4, -1) are exact in FP32, so both forms meet the FP64 bound."""
    A = gen.laplace2d(256)
    B = gen.rhs_block(A.n_cols, k, seed=k) if k > 1 else gen.uniform(A.n_cols, seed=1)
    with lib.Plan.from_csr(A, val_fp32=fp32) as p:
        y = run_block(p, B)
    ref = oracle.spmm(A, B.reshape(A.n_cols, -1))
    S = oracle.abs_scale(A, B.reshape(A.n_cols, -1))
    Y = y.reshape(A.n_rows, -1)
    per_col = [oracle.max_err_ratio(Y[:, c], ref[:, c], S[:, c], TOL_FP64) for c in range(ref.shape[1])]
    abs_err = np.abs(Y - ref).max(axis=0)
    print(f"laplace256 k={k} {'f32' if fp32 else 'f64'} values: per-column max |err|/(1e-13*sum|ab|) "
          f"{np.round(per_col, 4).tolist()}, max |err| {abs_err.tolist()}")
    assert max(per_col) <= 1.0


def run_block(p, B):
    import torch
    Bd = dev(B)
    C = torch.full(B.shape if B.ndim == 2 else (p.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    if B.ndim == 1:
        p.apply(Bd, C)
    else:
        p.apply_block(Bd, C)
    p.check()
    return host(C)
