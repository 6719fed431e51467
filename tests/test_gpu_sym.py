"""Symmetric CRS (Sec. 1.3.1) on the GPU: the stored triangle equals the
oracle's builder byte for byte, and the product through the C ABI matches the
oracle's CRS loop over the full matrix (bit-exact on integer data, within
1e-13 * sum |a*b| per row otherwise) for k = 1..16, FP32 values, strided
blocks, pipelined host steps and the degenerate cases."""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import TOL_FP64, assert_close, dev, host, run

pytestmark = pytest.mark.gpu


def sym_case(seed, n, integer=False, duplicates=False, shuffle=False, empty_rows=0.0, density=None):
    density = density if density is not None else min(1.0, 6.0 / max(n, 1))
    A = gen.random_csr(n, n, density, seed, integer=integer, empty_rows=empty_rows, duplicates=duplicates)
    return gen.symmetric_from(A, seed=seed, shuffle=shuffle)


CASES = {
    "laplace64": lambda: gen.laplace2d(64),
    "poisson20": lambda: gen.poisson3d_var(20),
    "eigen": lambda: gen.eigen_shaped(50_000, window=1 << 14),
    "ragged_dup_shuffled": lambda: sym_case(3, 3001, duplicates=True, shuffle=True, empty_rows=0.2),
    "dense_rows": lambda: sym_case(4, 300, density=0.5),
}


def sym_equal(got: dict, ref: oracle.Sym):
    assert np.array_equal(got["row_ptr"], ref.row_ptr)
    assert np.array_equal(got["col"], ref.col)
    assert got["val"].tobytes() == ref.val.tobytes()


@pytest.mark.parametrize("name", sorted(CASES))
def test_triangle_bit_exact(lib, name):
    A = CASES[name]()
    with lib.Plan.from_csr(A, variant=lib.SPMV_SYM) as p:
        ref = oracle.sym_build(A)
        assert p.info().sym_nnz == ref.nnz
        sym_equal(p.sym_export(), ref)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("k", [1, 3, 4, 16])
def test_product_fp64(lib, name, k):
    A = CASES[name]()
    B = gen.rhs_block(A.n_cols, k, seed=7) if k > 1 else gen.uniform(A.n_cols, seed=7)
    with lib.Plan.from_csr(A, variant=lib.SPMV_SYM) as p:
        assert_close(run(p, B, k), A, B)


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_product_integer_exact(lib, seed, k):
    A = sym_case(seed, 2500, integer=True, duplicates=True, shuffle=(seed % 2 == 0), empty_rows=0.1)
    rng = np.random.default_rng(seed)
    B = rng.integers(-1024, 1025, (A.n_cols, k)).astype(np.float64)
    B = B[:, 0].copy() if k == 1 else B
    with lib.Plan.from_csr(A, variant=lib.SPMV_SYM) as p:
        assert_close(run(p, B, k), A, B, exact=True)


@pytest.mark.parametrize("name", ["poisson20", "eigen"])
@pytest.mark.parametrize("k", [1, 4])
def test_product_fp32_values(lib, name, k):
    A = CASES[name]()
    B = gen.rhs_block(A.n_cols, k, seed=9) if k > 1 else gen.uniform(A.n_cols, seed=9)
    with lib.Plan.from_csr(A, variant=lib.SPMV_SYM, val_fp32=True) as p:
        assert_close(run(p, B, k), A, B, f32val=True)


def test_product_fp32_special_values(lib):
    """Subnormal and huge values take the hardware widening path."""
    A = sym_case(11, 500)
    A.val[::7] = 1e-41
    A = gen.symmetric_from(A)  # keep the mirrors equal after the edit
    B = gen.uniform(A.n_cols, seed=3)
    with lib.Plan.from_csr(A, variant=lib.SPMV_SYM, val_fp32=True) as p:
        assert_close(run(p, B), A, B, f32val=True)


def test_strided_block_keeps_other_columns(lib):
    """ldb, ldc > k: only C[:, :k] is written; the rest keeps its contents."""
    import torch
    A = CASES["poisson20"]()
    k, ldb, ldc = 3, 5, 7
    Bfull = gen.rhs_block(A.n_cols, ldb, seed=5)
    Bd = dev(Bfull)
    C = torch.full((A.n_rows, ldc), 123.25, dtype=torch.float64, device="cuda")
    with lib.Plan.from_csr(A, variant=lib.SPMV_SYM) as p:
        lib.spmv_apply_block(p.handle, Bd.data_ptr(), k, ldb, C.data_ptr(), ldc, 0)
        Ch = host(C)
    assert_close(np.ascontiguousarray(Ch[:, :k]), A, np.ascontiguousarray(Bfull[:, :k]))
    assert np.all(Ch[:, k:] == 123.25)


def test_repeated_calls_overwrite(lib):
    """Each apply overwrites C: a second call gives the same result, not twice it."""
    A = sym_case(5, 4000, integer=True)
    B = np.random.default_rng(1).integers(-50, 51, A.n_cols).astype(np.float64)
    import torch
    Bd = dev(B)
    C = torch.full((A.n_rows,), 7.0, dtype=torch.float64, device="cuda")
    with lib.Plan.from_csr(A, variant=lib.SPMV_SYM) as p:
        p.apply(Bd, C)
        first = host(C).copy()
        p.apply(Bd, C)
        assert np.array_equal(host(C), first)
    assert_close(first, A, B, exact=True)


def test_pipelined_host_steps(lib):
    import torch
    A = CASES["eigen"]()
    with lib.Plan.from_csr(A, variant=lib.SPMV_SYM) as p:
        Bs = [torch.from_numpy(gen.rhs_block(A.n_cols, 2, seed=40 + s)).pin_memory() for s in range(3)]
        Cs = [torch.empty((A.n_rows, 2), dtype=torch.float64).pin_memory() for _ in range(3)]
        for B, C in zip(Bs, Cs):
            p.apply_host_async(B, C, 2)
        p.host_sync()
        for B, C in zip(Bs, Cs):
            assert_close(C.numpy(), A, B.numpy())


def test_degenerate_cases(lib):
    one = gen.CSR(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.5]))
    with lib.Plan.from_csr(one, variant=lib.SPMV_SYM) as p:
        assert np.array_equal(run(p, np.array([4.0])), [10.0])
    diag = gen.CSR(5, 5, np.arange(6, dtype=np.int32), np.arange(5, dtype=np.int32), np.arange(1.0, 6.0))
    with lib.Plan.from_csr(diag, variant=lib.SPMV_SYM) as p:
        assert np.array_equal(run(p, np.ones(5)), np.arange(1.0, 6.0))
    empty_rows = gen.CSR(4, 4, np.zeros(5, np.int32), np.zeros(0, np.int32), np.zeros(0))
    with lib.Plan.from_csr(empty_rows, variant=lib.SPMV_SYM) as p:
        assert p.info().sym_nnz == 0
        assert np.array_equal(run(p, np.ones(4)), np.zeros(4))
    none = gen.CSR(0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    with lib.Plan.from_csr(none, variant=lib.SPMV_SYM) as p:
        assert p.info().n_rows == 0


def test_rejects_asymmetric_and_keeps_variant(lib):
    A = sym_case(2, 200)
    off = np.flatnonzero(A.col_idx != np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr)))
    A.val[off[0]] += 1.0
    assert not oracle.is_symmetric(A)
    with lib.Plan.from_csr(A, variant=lib.SPMV_CRS_L1) as p:
        with pytest.raises(lib.SpmvError) as e:
            p.set_variant(lib.SPMV_SYM)
        assert e.value.status == 6 and "not symmetric" in str(e.value)
        assert p.info().variant == lib.SPMV_CRS_L1 and p.info().sym_nnz == 0
        B = gen.uniform(A.n_cols, seed=1)
        assert_close(run(p, B), A, B)
    rect = gen.random_csr(30, 40, 0.1, 1)
    with pytest.raises(lib.SpmvError) as e:
        lib.Plan.from_csr(rect, variant=lib.SPMV_SYM)
    assert e.value.status == 6 and "square" in str(e.value)


def test_export_before_build_is_unsupported(lib):
    A = CASES["laplace64"]()
    with lib.Plan.from_csr(A) as p:
        with pytest.raises(lib.SpmvError) as e:
            p.sym_export()
        assert e.value.status == 6


def test_switching_between_sym_and_crs(lib):
    A = CASES["poisson20"]()
    B = gen.uniform(A.n_cols, seed=2)
    with lib.Plan.from_csr(A) as p:
        y0 = run(p, B)
        p.set_variant(lib.SPMV_SYM)
        y1 = run(p, B)
        p.set_variant(lib.SPMV_CRS_L1)
        assert np.array_equal(run(p, B), y0)
    assert_close(y1, A, B)
    assert oracle.max_err_ratio(y1, y0, oracle.abs_scale(A, B), 2 * TOL_FP64) <= 1.0


def test_graph_replays(lib):
    """The zeroing of C and the kernel are captured together, so a captured
    apply replayed several times with new B contents stays correct."""
    import torch
    A = sym_case(8, 20_000, integer=True, duplicates=True)
    rng = np.random.default_rng(8)
    Bd = torch.zeros(A.n_cols, dtype=torch.float64, device="cuda")
    C = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    with lib.Plan.from_csr(A, variant=lib.SPMV_SYM) as p:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            p.apply(Bd, C, s)  # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            p.apply(Bd, C, torch.cuda.current_stream())
        for r in range(4):
            B = rng.integers(-1024, 1025, A.n_cols).astype(np.float64)
            Bd.copy_(torch.from_numpy(B))
            g.replay()
            assert_close(host(C), A, B, exact=True)
        p.check()


@pytest.mark.parametrize("distance", [0, 1, 152, 100000])
def test_prefetch_distance_is_result_neutral(lib, distance):
    A = sym_case(9, 30_000, integer=True, duplicates=True, shuffle=True, empty_rows=0.05)
    B = np.random.default_rng(distance).integers(-1024, 1025, (A.n_cols, 4)).astype(np.float64)
    with lib.Plan.from_csr(A, variant=lib.SPMV_SYM) as p:
        p.set_tuning(prefetch_distance=distance)
        assert_close(run(p, B, 4), A, B, exact=True)
        assert_close(run(p, B[:, 0].copy()), A, B[:, 0].copy(), exact=True)
