"""GPU parity of every CRS/SELL variant against the oracle (single vector and
blocks of k right-hand sides, FP64 and FP32-stored values), edge cases and
error paths, all through the C ABI."""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import TOL_FP32VAL, TOL_FP64, assert_close, dev, host, run

pytestmark = pytest.mark.gpu

VARIANTS = [("crs_staged", 1, 1), ("crs_l1", 2, 1), ("crs_l2", 3, 1), ("crs_l4", 4, 1), ("crs_l8", 5, 1),
            ("crs_l16", 6, 1), ("crs_l32", 7, 1), ("sell_s1", 8, 1), ("sell_s256", 8, 256),
            ("sell_s4096", 8, 4096)]
VIDS = [v[0] for v in VARIANTS]

_CASES = {}


def case(name):
    if name not in _CASES:
        if name == "laplace256":          # the 2D 5-point workload at full size
            _CASES[name] = gen.laplace2d(256)
        elif name == "poisson40":         # 3D variable-coefficient stencil, 64,000 rows
            _CASES[name] = gen.poisson3d_var(40)
        elif name == "eigen":             # eigenproblem-shaped, many tiles
            _CASES[name] = gen.eigen_shaped(150_000, window=1 << 16)
        elif name == "powerlaw":          # rows up to 2000 long (warp-per-row blocks)
            _CASES[name] = gen.powerlaw(30_000, seed=1)
        elif name == "ragged":            # unsorted, duplicates, empty rows, odd sizes
            _CASES[name] = gen.random_csr(1037, 911, 0.012, 5, empty_rows=0.2, duplicates=True, unsorted=True)
        elif name == "integer":
            _CASES[name] = gen.random_csr(3001, 2999, 0.004, 6, integer=True, empty_rows=0.05, duplicates=True)
    return _CASES[name]


def make(lib, A, vid, sigma, **kw):
    return lib.Plan.from_csr(A, variant=vid, sell_sigma=sigma, **kw)


@pytest.mark.parametrize("name", ["laplace256", "poisson40", "eigen", "powerlaw", "ragged"])
@pytest.mark.parametrize("variant", VARIANTS, ids=VIDS)
def test_spmv_matches_oracle(lib, name, variant):
    A = case(name)
    B = gen.uniform(A.n_cols, seed=7)
    with make(lib, A, variant[1], variant[2]) as p:
        assert p.info().variant == variant[1]
        assert_close(run(p, B), A, B)


@pytest.mark.parametrize("variant", VARIANTS, ids=VIDS)
def test_integer_bit_exact(lib, variant):
    """Integer values |v| <= 2^10 and short rows: every partial sum is exact, so
    any summation order gives the oracle's result bit for bit."""
    A = case("integer")
    B = np.random.default_rng(0).integers(-1024, 1025, A.n_cols).astype(np.float64)
    with make(lib, A, variant[1], variant[2]) as p:
        assert_close(run(p, B), A, B, exact=True)
        Bk = np.random.default_rng(1).integers(-1024, 1025, (A.n_cols, 4)).astype(np.float64)
        assert_close(run(p, Bk), A, Bk, exact=True)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8, 13, 16])
@pytest.mark.parametrize("variant", [VARIANTS[0], VARIANTS[1], VARIANTS[4], VARIANTS[6], VARIANTS[8]],
                         ids=["crs_staged", "crs_l1", "crs_l8", "crs_l32", "sell_s256"])
def test_spmm_block(lib, k, variant):
    for name in ("laplace256", "powerlaw"):
        A = case(name)
        B = gen.rhs_block(A.n_cols, k, seed=k)
        with make(lib, A, variant[1], variant[2]) as p:
            assert_close(run(p, B), A, B)


def test_spmm_leading_dimensions(lib):
    """ldb > k and ldc > k: only the first k columns are read and written."""
    import torch
    A = case("eigen")
    k = 3
    B = gen.rhs_block(A.n_cols, 8, seed=3)
    with lib.Plan.from_csr(A) as p:
        Bd = dev(B)
        C = torch.full((A.n_rows, 6), 7.0, dtype=torch.float64, device="cuda")
        p.apply_block(Bd, C, k)
        y = host(C)
        assert np.all(y[:, k:] == 7.0)
        assert_close(np.ascontiguousarray(y[:, :k]), A, np.ascontiguousarray(B[:, :k]))


@pytest.mark.parametrize("k", [2, 4, 8, 16])
@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("vname", ["SPMV_CRS_L1", "SPMV_CRS_STAGED", "SPMV_SELL", "SPMV_CRS_L4", "SPMV_CRS_L32"])
def test_spmm_16_byte_and_scalar_paths_identical(lib, k, fp32, vname):
    """A full contiguous, 16-byte aligned block of k >= 2 columns takes the
    16-byte paths (the column-split kernels of CRS_L1, STAGED and SELL; 16-byte
    gathers in the L-lanes kernels); the same product from blocks 8 bytes off
    alignment takes scalar accesses.  Each column's sum is formed in the same
    order, so the bits are the same."""
    import torch
    A = case("powerlaw")
    B = gen.rhs_block(A.n_cols, k, seed=20 + k)
    with lib.Plan.from_csr(A, val_fp32=fp32, variant=getattr(lib, vname), sell_sigma=64) as p:
        Bd = dev(B)
        C = torch.empty((A.n_rows, k), dtype=torch.float64, device="cuda")
        p.apply_block(Bd, C, k)
        y_vec = host(C)
        flat_b = torch.zeros(A.n_cols * k + 1, dtype=torch.float64, device="cuda")
        Bo = flat_b[1:].view(A.n_cols, k)
        Bo.copy_(Bd)
        flat_c = torch.zeros(A.n_rows * k + 1, dtype=torch.float64, device="cuda")
        Co = flat_c[1:].view(A.n_rows, k)
        p.apply_block(Bo, Co, k)
        y_scalar = host(Co)
    assert np.array_equal(y_vec, y_scalar)
    assert_close(y_vec, A, B, f32val=fp32, tol=TOL_FP64)


@pytest.mark.parametrize("variant", VARIANTS, ids=VIDS)
def test_fp32_values(lib, variant):
    """FP32-stored values: equal (to FP64 rounding) to the oracle's loop over
    float-rounded values, and within 2e-7 * sum|ab| of the FP64 product."""
    A = case("eigen")
    B = gen.uniform(A.n_cols, seed=9)
    Bk = gen.rhs_block(A.n_cols, 4, seed=10)
    with make(lib, A, variant[1], variant[2], val_fp32=True) as p:
        assert p.info().val_fp32 == 1
        y = run(p, B)
        assert_close(y, A, B, tol=TOL_FP64, f32val=True)
        assert_close(y, A, B, tol=TOL_FP32VAL)
        yk = run(p, Bk)
        assert_close(yk, A, Bk, tol=TOL_FP64, f32val=True)
        assert_close(yk, A, Bk, tol=TOL_FP32VAL)


@pytest.mark.parametrize("subnormals", [False, True], ids=["normal_only", "with_subnormals"])
@pytest.mark.parametrize("variant", [VARIANTS[0], VARIANTS[1], VARIANTS[2], VARIANTS[7]],
                         ids=["crs_staged", "crs_l1", "crs_l2", "sell"])
def test_fp32_widening_special_values(lib, variant, subnormals):
    """FP32 storage widens exactly: the integer-pipe path (zeros of both signs and
    normals across the exponent range, including the smallest and largest
    normal floats) and the hardware path the plan picks when subnormal floats
    are present."""
    vals = [0.0, -0.0, 1.0, -1.0, 3.1415926535, 1e-30, -2.5e30, 3.4e38, 1.2e-38, 1.17549435e-38,
            -3.4028234e38, 123456.789, -0.1]
    if subnormals:
        vals += [1e-40, -7e-45, 6.0e-39]
    vals = np.array(vals, dtype=np.float64)
    n = len(vals)
    A = gen.CSR(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), vals)
    B = np.ones(n)
    with make(lib, A, variant[1], variant[2], val_fp32=True) as p:
        y = run(p, B)
    ref = vals.astype(np.float32).astype(np.float64) + 0.0   # 0.0 + x turns -0 into +0, as the loop does
    assert np.array_equal(y, ref)
    assert np.array_equal(np.signbit(y), np.signbit(ref))


def test_edge_cases(lib):
    # no rows at all
    A = gen.CSR(0, 5, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    with lib.Plan.from_csr(A) as p:
        p.apply(dev(np.ones(5)), dev(np.zeros(1)))
        p.check()
    # only empty rows: C is overwritten with +0.0 by every variant
    A = gen.CSR(700, 5, np.zeros(701, np.int32), np.zeros(0, np.int32), np.zeros(0))
    for _, vid, sig in VARIANTS:
        with make(lib, A, vid, sig) as p:
            y = run(p, np.ones(5))
            assert np.array_equal(y, np.zeros(700)) and not np.signbit(y).any()
    # 1 x 1
    A = gen.CSR(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0]))
    for _, vid, sig in VARIANTS:
        with make(lib, A, vid, sig) as p:
            assert run(p, np.array([-2.5]))[0] == -7.5


@pytest.mark.parametrize("variant", VARIANTS, ids=VIDS)
def test_row_length_boundaries(lib, variant):
    """Rows of length 63/64/65 (the warp-row threshold), longer than a tile,
    mixed with empty and short rows, with an odd nnz and an odd row count."""
    lens = [0, 1, 63, 64, 65, 2, 0, 7, 600, 5000, 12000, 3, 1, 0, 9999] + [5] * 513 + [1]
    A = gen.csr_from_lengths(lens, 20000, seed=11)
    assert A.nnz % 2 == 1
    B = gen.uniform(A.n_cols, seed=12)
    with make(lib, A, variant[1], variant[2]) as p:
        assert_close(run(p, B), A, B)
        Bk = gen.rhs_block(A.n_cols, 4, seed=13)
        assert_close(run(p, Bk), A, Bk)


def test_deterministic(lib):
    A = case("powerlaw")
    B = gen.uniform(A.n_cols, seed=1)
    for _, vid, sig in VARIANTS:
        with make(lib, A, vid, sig) as p:
            assert np.array_equal(run(p, B), run(p, B))


def test_apply_host_end_to_end(lib):
    A = case("eigen")
    B = gen.uniform(A.n_cols, seed=2)
    Bk = gen.rhs_block(A.n_cols, 4, seed=3)
    with lib.Plan.from_csr(A) as p:
        assert np.array_equal(p.apply_host(B), run(p, B))
        assert np.array_equal(p.apply_host(Bk, k=4), run(p, Bk))


def test_set_variant_switches(lib):
    A = case("poisson40")
    B = gen.uniform(A.n_cols, seed=4)
    with lib.Plan.from_csr(A) as p:
        assert p.info().variant == lib.SPMV_CRS_L1   # the default (AUTO) kernel
        assert p.tuning().prefetch_distance == 456   # three CTAs per SM ahead
        for _, vid, sig in VARIANTS:
            p.set_variant(vid, sig)
            assert p.info().variant == vid
            assert_close(run(p, B), A, B)


@pytest.mark.parametrize("name,scattered", [("eigen", True), ("poisson40", False), ("laplace256", False),
                                             ("integer", True)])
def test_auto_variant_follows_the_gather_pattern(lib, name, scattered):
    """AUTO runs SELL-32-256 without the L2 prefetch on matrices whose rows
    gather at scattered addresses (the eigenproblem-shaped matrix, a random
    sparse matrix: SELL-32-256 fills its slots well on both), and CRS_L1 with
    the prefetch on stencils; either way the product matches the oracle."""
    A = case(name)
    B = (np.random.default_rng(5).integers(-1024, 1025, A.n_cols).astype(np.float64) if name == "integer"
         else gen.uniform(A.n_cols, seed=5))
    with lib.Plan.from_csr(A) as p:
        i, t = p.info(), p.tuning()
        if scattered:
            assert (i.variant, i.sell_sigma, t.prefetch_distance) == (lib.SPMV_SELL, 256, 0)
        else:
            assert (i.variant, t.prefetch_distance) == (lib.SPMV_CRS_L1, 456)
        assert_close(run(p, B), A, B, exact=(name == "integer"))


def _auto_analysis(A):
    """The AUTO test restated from its definition: about 4096 evenly spaced
    sample rows; an entry (i, c) is regular when row i-1 holds column c-1 or
    row i+1 holds c+1; and the fill of SELL-32-256 from the row lengths."""
    n = A.n_rows
    tot = sc = 0
    if n >= 3:
        step = max(1, (n - 2) // 4096)
        for i in range(1, n - 1, step):
            prev = set(A.col_idx[A.row_ptr[i - 1]:A.row_ptr[i]].tolist())
            nxt = set(A.col_idx[A.row_ptr[i + 1]:A.row_ptr[i + 2]].tolist())
            for c in A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]].tolist():
                tot += 1
                sc += not ((c - 1) in prev or (c + 1) in nxt)
    L = np.diff(A.row_ptr).astype(np.int64)
    slots = 0
    for w in range(0, n, 256):
        lw = np.sort(L[w:w + 256])[::-1]
        slots += sum(32 * int(lw[c:c + 32].max()) for c in range(0, len(lw), 32))
    return (sc / tot if tot else 0.0), (A.nnz / slots if slots else 1.0)


@pytest.mark.parametrize("name", ["eigen", "poisson40", "laplace256", "integer", "powerlaw", "ragged"])
def test_auto_analysis_reported_in_info(lib, name):
    """spmv_info reports the two numbers AUTO decides on; they equal the rule
    restated in Python (the sample, the counts and the fill are exact)."""
    A = case(name)
    want_sc, want_fill = _auto_analysis(A)
    with lib.Plan.from_csr(A) as p:
        i = p.info()
        assert i.scattered == pytest.approx(want_sc, rel=1e-14, abs=0)
        assert i.sell256_fill == pytest.approx(want_fill, rel=1e-14, abs=0)
        auto_sell = i.scattered > 0.3 and i.sell256_fill >= 0.85
        assert (i.variant == lib.SPMV_SELL) == auto_sell


def test_error_paths(lib):
    A = case("ragged")
    with lib.Plan.from_csr(A, max_k=4) as p:
        B = dev(np.ones(A.n_cols))
        C = dev(np.zeros(A.n_rows))
        for bad_k in (0, 5, 17):
            with pytest.raises(lib.SpmvError) as e:
                lib.spmv_apply_block(p.handle, B.data_ptr(), bad_k, bad_k + 1, C.data_ptr(), bad_k + 1, 0)
            assert e.value.status == 1
        with pytest.raises(lib.SpmvError) as e:
            lib.spmv_apply_block(p.handle, B.data_ptr(), 2, 1, C.data_ptr(), 2, 0)
        assert e.value.status == 1
        with pytest.raises(lib.SpmvError) as e:
            p.apply_split(B, B, C)
        assert e.value.status == 6
        with pytest.raises(lib.SpmvError) as e:
            p.set_variant(99)
        assert e.value.status == 1
        with pytest.raises(lib.SpmvError) as e:
            p.sell_export()
        assert e.value.status == 6
        p.check()


@pytest.mark.parametrize("variant", VARIANTS, ids=VIDS)
def test_prefetch_tuning_keeps_results(lib, variant):
    """The L2 prefetch distance is a pure performance knob: results are identical."""
    A = case("eigen")
    B = gen.uniform(A.n_cols, seed=21)
    with make(lib, A, variant[1], variant[2]) as p:
        base = run(p, B)
        for d in (1, 7, 300, 100000):
            p.set_tuning(prefetch_distance=d)
            assert p.tuning().prefetch_distance == d
            assert np.array_equal(run(p, B), base)
        with pytest.raises(lib.SpmvError):
            p.set_tuning(prefetch_distance=-1)


@pytest.mark.parametrize("k", [1, 4])
def test_pipelined_host_steps(lib, k):
    """Pipelined end-to-end steps (two device buffer sets, copy-in/out streams)
    give every step's own product, also when the buffers are reused."""
    import torch
    A = case("poisson40")
    steps = 5
    Bs = [gen.uniform(A.n_cols * k, seed=50 + i).reshape(A.n_cols, k) if k > 1 else gen.uniform(A.n_cols, seed=50 + i)
          for i in range(steps)]
    Bp = [torch.from_numpy(B.copy()).pin_memory() for B in Bs]
    Cp = [torch.full(B.shape[:1] if k == 1 else (A.n_rows, k), float("nan"), dtype=torch.float64).pin_memory()
          for B in Bs]
    with lib.Plan.from_csr(A) as p:
        for i in range(steps):
            p.apply_host_async(Bp[i], Cp[i], k)
        p.host_sync()
        for i in range(steps):
            assert_close(Cp[i].numpy(), A, Bs[i])
        # same host buffers again: results are overwritten in step order
        for i in range(steps):
            p.apply_host_async(Bp[steps - 1 - i], Cp[i], k)
        p.host_sync()
        for i in range(steps):
            assert_close(Cp[i].numpy(), A, Bs[steps - 1 - i])


def test_zero_initialised_options_build_the_default_plan(lib):
    """spmv_create with a zero-initialised spmv_options, with NULL options and
    with spmv_default_options() builds the same plan (AUTO -> CRS_L1, FP64
    values, no split) and the same product bit for bit; nnz is the caller's
    count of stored entries."""
    import torch
    A = case("powerlaw")
    B = dev(gen.uniform(A.n_cols, seed=3))
    rp, ci, va = (np.ascontiguousarray(x) for x in (A.row_ptr, A.col_idx, A.val))
    outs, infos = [], []
    for opt in (lib.spmv_options(), None, lib.spmv_default_options()):
        h = lib.spmv_create(A.n_rows, A.n_cols, A.nnz, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, opt)
        try:
            C = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
            lib.spmv_apply(h, B.data_ptr(), C.data_ptr(), torch.cuda.current_stream().cuda_stream)
            outs.append(host(C))
            i = lib.spmv_get_info(h)
            infos.append((i.variant, i.val_fp32, i.n_halo_rows, i.halo_nnz, i.sell_sigma))
        finally:
            lib.spmv_destroy(h)
    assert infos[0] == infos[1] == infos[2]
    assert infos[0][1:4] == (0, 0, 0)            # FP64 values, no split
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    assert_close(outs[0], A, gen.uniform(A.n_cols, seed=3))


def test_auto_sell_plan_forms(lib):
    """A plan whose AUTO kernel is SELL-32-256 (scattered gathers) through every
    product form: k-column blocks with ld > k and an 8-byte offset, FP32-stored
    values (2e-7 against the FP64 oracle, 1e-13 against its FP32-value loop),
    and the local/halo split (the local pass runs CRS_L1)."""
    import torch
    A = case("eigen")
    with lib.Plan.from_csr(A) as p:
        assert p.info().variant == lib.SPMV_SELL
        for k in (1, 3, 4, 16):
            ld = k + 3
            Bh = gen.rhs_block(A.n_cols, k, seed=20 + k)
            Bbuf = torch.zeros(A.n_cols * ld + 1, dtype=torch.float64, device="cuda")
            Bv = Bbuf[1:].view(A.n_cols, ld)              # 8 bytes off 16-byte alignment
            Bv[:, :k] = torch.from_numpy(Bh).cuda()
            Cbuf = torch.full((A.n_rows * ld + 1,), float("nan"), dtype=torch.float64, device="cuda")
            Cv = Cbuf[1:].view(A.n_rows, ld)
            p.apply_block(Bv, Cv, k)
            p.check()
            y = host(Cv)
            assert_close(y[:, :k], A, Bh)
            assert np.isnan(y[:, k:]).all()                 # nothing beyond the k columns is written
    B = gen.uniform(A.n_cols, seed=21)
    with lib.Plan.from_csr(A, val_fp32=True) as p:
        assert p.info().variant == lib.SPMV_SELL
        y = run(p, B)
        assert_close(y, A, B, tol=TOL_FP32VAL)
        assert_close(y, A, B, f32val=True)
    h = A.n_cols - A.n_cols // 7
    with lib.Plan.from_csr(A, halo_begin=h) as p:
        assert p.info().variant == lib.SPMV_SELL
        Bd = dev(B)
        halo = torch.from_numpy(B[h:].copy()).pin_memory()
        Bd[h:] = float("nan")
        C = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
        p.apply_split(Bd, halo, C, torch.cuda.current_stream(), torch.cuda.Stream())
        p.check()
        assert_close(host(C), A, B)


@pytest.mark.parametrize("shape", [(0, 0), (0, 5), (5, 0), (1, 1), (2, 7), (3, 3)])
def test_auto_tiny_and_empty_shapes(lib, shape):
    """AUTO's row sample on matrices too small to sample (fewer than three
    rows) or without entries: the plan builds on CRS_L1 (a zero scattered
    share where nothing is sampled; where something is, SELL-32-256 fills too
    few of its slots here to be chosen), and the product is the oracle's."""
    n, m = shape
    rng = np.random.default_rng(n * 10 + m)
    rp = np.zeros(n + 1, np.int32)
    cols, vals = [], []
    for i in range(n):
        c = np.sort(rng.choice(m, size=min(m, 2), replace=False)) if m else np.zeros(0, np.int64)
        cols.append(c)
        vals.append(rng.integers(-5, 6, len(c)).astype(np.float64))
        rp[i + 1] = rp[i] + len(c)
    A = gen.CSR(n, m, rp, np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32),
                np.concatenate(vals) if vals else np.zeros(0))
    with lib.Plan.from_csr(A) as p:
        i = p.info()
        assert i.variant == lib.SPMV_CRS_L1
        if n < 3 or m == 0:
            assert i.scattered == 0.0
        if n and m:
            B = rng.integers(-5, 6, m).astype(np.float64)
            assert_close(run(p, B), A, B, exact=True)
