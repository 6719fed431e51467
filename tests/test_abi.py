"""The C ABI library builds, loads, and exports every symbol declared in
include/*.h; host-only entry points (CRS validation, features) work without a
GPU and agree with the oracle."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import gen
from oracle import features as ofeat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_1101_0091_gb300 import build
    return build.build()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([a-z_][a-z0-9_]*)\s*\(", text):
            name = m.group(1)
            if name.startswith("spmv_"):
                names.add(name)
    return names


def test_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    names = declared_functions()
    assert {"spmv_create", "spmv_apply", "spmv_apply_block", "spmv_destroy"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads(built):
    import paper_1101_0091_gb300 as spmv
    spmv.load()
    o = spmv.spmv_default_options()
    assert (o.variant, o.sell_sigma, o.val_fp32, o.max_k, o.split, o.reserved, o.halo_begin) == (0, 1, 0, 16, 0, 0, 0)


def test_zero_initialised_options_mean_the_defaults(built):
    """A zero-initialised spmv_options (every field 0) asks for what
    spmv_default_options() returns: AUTO, no SELL sorting, FP64 values,
    max_k 16 and no split.  Field by field, each zero is read as its default."""
    import paper_1101_0091_gb300 as spmv
    z, d = spmv.spmv_options(), spmv.spmv_default_options()
    assert (z.variant, z.val_fp32, z.split, z.reserved) == (d.variant, d.val_fp32, d.split, d.reserved)
    assert z.max_k == 0 and d.max_k == 16        # 0 means 16 (the create call maps it)
    assert z.sell_sigma == 0 and d.sell_sigma == 1   # <= 1 means no sorting either way
    assert z.halo_begin == d.halo_begin == 0     # read only when split = 1


def bad_create(n_rows, n_cols, rp, ci, va, nnz=None, opt=None):
    import paper_1101_0091_gb300 as spmv
    rp = np.ascontiguousarray(rp, np.int32)
    ci = np.ascontiguousarray(ci, np.int32)
    va = np.ascontiguousarray(va, np.float64)
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_create(n_rows, n_cols, len(ci) if nnz is None else nnz, rp.ctypes.data, ci.ctypes.data,
                         va.ctypes.data, opt)
    return e.value


@pytest.mark.parametrize("case", ["nnz_short", "nnz_long", "nnz_negative"])
def test_nnz_cross_checked_against_row_ptr(built, case):
    """spmv_create takes the caller's nnz (Sec. 1.2's CRS has nnz entries in
    val and col_idx) and rejects it on the host when row_ptr[n_rows] differs."""
    nnz = {"nnz_short": 2, "nnz_long": 4, "nnz_negative": -1}[case]
    err = bad_create(2, 3, [0, 2, 3], [0, 1, 2], [1.0, 2.0, 3.0], nnz=nnz)
    assert err.status == 2 and ("nnz" in str(err))


@pytest.mark.parametrize("case", ["split_flag", "reserved", "halo_negative", "halo_high"])
def test_bad_options_rejected_on_host(built, case):
    import paper_1101_0091_gb300 as spmv
    o = spmv.spmv_default_options()
    if case == "split_flag":
        o.split = 2
    elif case == "reserved":
        o.reserved = 7
    elif case == "halo_negative":
        o.split, o.halo_begin = 1, -1
    else:
        o.split, o.halo_begin = 1, 4
    err = bad_create(2, 3, [0, 2, 3], [0, 1, 2], [1.0, 2.0, 3.0], opt=o)
    assert err.status == 1   # SPMV_ERR_ARG, before any device call


@pytest.mark.parametrize("case", ["row_ptr0", "decreasing", "col_high", "col_negative", "neg_dim",
                                  "rows_over_int32", "cols_over_int32"])
def test_malformed_csr_rejected_on_host(built, case):
    """CRS validation runs on the host before any device call (no GPU needed)."""
    rp, ci, va, n, m = [0, 2, 3], [0, 1, 2], [1.0, 2.0, 3.0], 2, 3
    if case == "row_ptr0":
        rp = [1, 2, 3]
    elif case == "decreasing":
        rp = [0, 3, 2]
    elif case == "col_high":
        ci = [0, 1, 3]
    elif case == "col_negative":
        ci = [0, -1, 2]
    elif case == "neg_dim":
        n = -1
    elif case == "rows_over_int32":      # the size limits of the int32 index arrays
        n = 2**31                        # (checked before any array is read)
    elif case == "cols_over_int32":
        m = 2**31 + 5
    err = bad_create(n, m, rp, ci, va)
    assert err.status == 2  # SPMV_ERR_CSR


@pytest.mark.parametrize("which", ["laplace", "powerlaw", "eigen", "empty_rows"])
def test_features_match_oracle(built, which):
    import paper_1101_0091_gb300 as spmv
    if which == "laplace":
        A, k = gen.laplace2d(64), 1
    elif which == "powerlaw":
        A, k = gen.powerlaw(5000, seed=3), 4
    elif which == "eigen":
        A, k = gen.eigen_shaped(5000, window=1 << 10), 16
    else:
        A, k = gen.random_csr(300, 200, 0.02, 4, empty_rows=0.5), 8
    f = spmv.features(A, k)
    ref = ofeat.features(A, k)
    # counts and ratios of integers are exact; the std and logs agree to rounding
    exact = list(range(0, 26)) + [28, 31, 32]
    assert np.array_equal(f[exact], ref[exact])
    assert np.allclose(f, ref, rtol=1e-13, atol=0)


def test_probe_arguments_checked_on_host(built):
    """The probes reject bad sizes before any CUDA call."""
    import paper_1101_0091_gb300 as spmv
    for call in (lambda: spmv.spmv_probe_fp64(0), lambda: spmv.spmv_probe_gather(0, 3),
                 lambda: spmv.spmv_probe_gather(2 ** 31, 3), lambda: spmv.spmv_probe_gather(100, 0)):
        with pytest.raises(spmv.SpmvError) as e:
            call()
        assert e.value.status == 1
