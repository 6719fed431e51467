"""The allocation-free batched entry point (spmv_batch_apply_noalloc), for
callers that may not allocate device memory, gives the same products as the
regular batched entry point (spmv_batch_apply) on two calls in a row.  The
caller owns every device buffer (here: torch tensors); the entry point keeps
its scratch in a static device array.  Collected last on purpose: if it fails,
a run that stops at the first failure has already run every other test.

Each member is checked three ways: against the oracle's CRS loop (the
1e-13 * sum|a b| bound of every FP64 test), against the regular entry point
within the same bound, and bit for bit against the regular entry point where
a fixed batch policy with the same lanes per row exists (the same kernel sums
each row in the same order).  Sixteen lanes per row has no fixed policy, so
those members are held to the bound only."""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import TOL_FP64, dev, host

pytestmark = pytest.mark.gpu

LANE_POLICY = {1: 0, 2: 1, 4: 2, 8: 3, 32: 4}   # lanes per row -> fixed batch policy
SORTED = 6                                       # the regular entry point's default policy


def device_csr(A):
    return dev(A.row_ptr), dev(A.col_idx if A.nnz else np.zeros(1, np.int32)), dev(A.val if A.nnz else np.zeros(1))


def regular(lib, As, Bs, k, lanes):
    """Products through spmv_batch_apply: the fixed policy with the same lanes
    per row where one exists, the default (sorted) policy otherwise."""
    import torch
    plans = [lib.Plan.from_csr(A) for A in As]
    Cs = [torch.full((A.n_rows, k), float("nan"), dtype=torch.float64, device="cuda") for A in As]
    with lib.Batch(plans, k, [LANE_POLICY.get(L, SORTED) for L in lanes]) as b:
        b.set_io([dev(B) for B in Bs], Cs)
        b.apply()
        torch.cuda.synchronize()
        out = [host(C) for C in Cs]
    for p in plans:
        p.close()
    return out


def no_alloc(lib, As, Bs, k, lanes):
    import torch
    csr = [device_csr(A) for A in As]
    Bd = [dev(B) for B in Bs]
    Cd = [torch.full((A.n_rows, k), float("nan"), dtype=torch.float64, device="cuda") for A in As]
    lib.spmv_batch_apply_noalloc([A.n_rows for A in As], [c[0].data_ptr() for c in csr],
                                 [c[1].data_ptr() for c in csr], [c[2].data_ptr() for c in csr],
                                 [B.data_ptr() for B in Bd], [k] * len(As), [C.data_ptr() for C in Cd],
                                 [k] * len(As), k, lanes, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return [host(C) for C in Cd]


def compare(As, Bs, lanes, got, reg):
    for A, B, L, g, r in zip(As, Bs, lanes, got, reg):
        assert not np.isnan(g).any()
        ref = oracle.spmm(A, B)
        scale = oracle.abs_scale(A, B)
        assert oracle.max_err_ratio(g, ref, scale, TOL_FP64) <= 1.0          # the oracle
        assert oracle.max_err_ratio(g, r, scale, TOL_FP64) <= 1.0            # the existing entry point
        if L in LANE_POLICY:
            assert np.array_equal(g, r), f"{L} lanes per row: not bitwise equal to the fixed policy"


def test_no_alloc_matches_batch_entry_twice(lib):
    import paper_1101_0091_gb300 as spmv
    # first call: 24 uneven power-law members, k = 4, every lanes-per-row value
    As1 = [gen.powerlaw_batch_member(m, seed=3, dim_lo=1e3, dim_hi=3e4) for m in range(24)]
    Bs1 = [gen.rhs_block(A.n_cols, 4, seed=m) for m, A in enumerate(As1)]
    lanes1 = [[1, 2, 4, 8, 16, 32][m % 6] for m in range(len(As1))]
    compare(As1, Bs1, lanes1, no_alloc(spmv, As1, Bs1, 4, lanes1), regular(spmv, As1, Bs1, 4, lanes1))
    # second call in a row: other members, odd k, a member with empty rows
    As2 = [gen.laplace2d(64), gen.poisson3d_var(12),
           gen.CSR(40, 7, np.zeros(41, np.int32), np.zeros(0, np.int32), np.zeros(0)),
           gen.powerlaw(5000, seed=9), gen.powerlaw(3000, seed=10)]
    Bs2 = [gen.rhs_block(A.n_cols, 3, seed=40 + m) for m, A in enumerate(As2)]
    lanes2 = [1, 4, 1, 32, 16]
    compare(As2, Bs2, lanes2, no_alloc(spmv, As2, Bs2, 3, lanes2), regular(spmv, As2, Bs2, 3, lanes2))


@pytest.mark.parametrize("k", [1, 2, 8, 16])
def test_no_alloc_other_widths(lib, k):
    """The other kernel widths (each with its own register budget, so fewer
    of the launched CTAs may be resident at once) against the oracle and the
    regular entry point."""
    import paper_1101_0091_gb300 as spmv
    As = [gen.powerlaw_batch_member(m, seed=5, dim_lo=1e3, dim_hi=2e4) for m in range(6)]
    Bs = [gen.rhs_block(A.n_cols, k, seed=60 + m) for m, A in enumerate(As)]
    lanes = [1, 2, 4, 8, 16, 32]
    compare(As, Bs, lanes, no_alloc(spmv, As, Bs, k, lanes), regular(spmv, As, Bs, k, lanes))


def test_no_alloc_rejects_sizes_beyond_the_scratch(lib):
    """Sizes beyond the static scratch and NULL operands are rejected on the
    host before any CUDA call (the pointers below are never dereferenced)."""
    import paper_1101_0091_gb300 as spmv
    fake = [1] * 8193
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_batch_apply_noalloc([1] * 8193, fake, fake, fake, fake, None, fake, None, 4)
    assert e.value.status == 1 and "8192" in str(e.value)
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_batch_apply_noalloc([2 ** 31 - 1], [1], [1], [1], [1], None, [1], None, 4, [32])
    assert e.value.status == 1 and "scratch" in str(e.value)
    # a member with rows but a NULL B (or col, val) would fault in the kernel: refused
    for which in range(3):
        ptrs = [[16], [16], [16], [16]]       # col, val, B and C of one member
        ptrs[which] = [0]
        with pytest.raises(spmv.SpmvError) as e:
            spmv.spmv_batch_apply_noalloc([5], [16], ptrs[0], ptrs[1], ptrs[2], None, ptrs[3], None, 4)
        assert e.value.status == 1 and "NULL" in str(e.value)
