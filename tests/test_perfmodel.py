"""The code-balance model (Eq. 1, Eq. 2) and the kappa calculator reproduce the
numbers the paper prints (fixture tests/golden/paper_numbers.json)."""
import json
import os

import pytest

from paper_1101_0091_gb300 import perfmodel as pm

with open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")) as f:
    P = json.load(f)


def test_eq1_limits():
    d = P["nehalem_socket"]
    assert pm.code_balance_crs(15) == pytest.approx(6.8)
    assert round(pm.perf_limit(d["spmv_bandwidth_gbs"], d["nnzr"]), 2) == d["limit_at_spmv_bandwidth_gflops"]
    assert round(pm.perf_limit(d["stream_bandwidth_gbs"], d["nnzr"]), 2) == d["limit_at_stream_bandwidth_gflops"]


def test_kappa_from_measurement():
    d = P["nehalem_socket"]
    k = pm.kappa_from_measurement(d["spmv_bandwidth_gbs"], d["spmv_gflops"], d["nnzr"])
    assert k == pytest.approx(2.4889, abs=1e-4)
    assert round(k, 1) == d["kappa_printed"]
    # the paper's 37.3 bytes/row uses the unrounded kappa
    assert round(pm.kappa_bytes_per_row(k, d["nnzr"]), 1) == d["kappa_bytes_per_row_printed"]
    assert round(pm.b_loads(k, d["nnzr"])) == d["b_loaded_times_printed"]
    assert d["spmv_bandwidth_gbs"] / d["stream_bandwidth_gbs"] > d["spmv_over_stream_printed_lower_bound"]
    # kappa = 0 reproduces the model itself
    assert pm.kappa_from_measurement(18.1, pm.perf_limit(18.1, 15), 15) == pytest.approx(0, abs=1e-12)


def test_hmep_numbering():
    d, n = P["hmep_numbering"], P["nehalem_socket"]
    k0 = pm.kappa_from_measurement(n["spmv_bandwidth_gbs"], n["spmv_gflops"], n["nnzr"])
    assert d["kappa_printed"] / k0 - 1 == pytest.approx(d["extra_b_transfer_increase_printed"], abs=0.03)
    drop = pm.code_balance_crs(15, d["kappa_printed"]) / pm.code_balance_crs(15, k0) - 1
    assert drop == pytest.approx(d["performance_drop_printed_about"], abs=0.03)


def test_eq2_split_penalty():
    d = P["split_penalty"]
    assert round(pm.split_penalty(7), 2) == d["nnzr_7_printed"]
    assert round(pm.split_penalty(15), 2) == d["nnzr_15_printed"]
    assert pm.code_balance_split(7) - pm.code_balance_crs(7) == pytest.approx(8 / 7)
    # "even less if kappa > 0"
    assert pm.split_penalty(7, 2.0) < pm.split_penalty(7)


def test_gpu_min_traffic():
    # 3D 7-point stencil on 280^3: 21,952,000 rows, 153,193,600 nonzeros
    t = pm.gpu_min_traffic(21_952_000, 21_952_000, 153_193_600)
    assert t.bytes_min == 2_277_363_204
    assert t.flops == 306_387_200
    # 2D 5-point on 256^2
    assert pm.gpu_min_traffic(65536, 65536, 326656).bytes_min == 5_230_596
    assert pm.gpu_min_traffic(65536, 65536, 326656, k=4, val_bytes=4).bytes_min == 326656 * 8 + 4 * 65537 + 64 * 65536
    # code balance of a square matrix equals V_min / flops
    n, nnz = 1000, 7000
    assert pm.gpu_code_balance(7.0) == pytest.approx(pm.gpu_min_traffic(n, n, nnz).bytes_min / (2 * nnz), rel=1e-3)
    assert pm.kappa_gpu(1.1e9, 1.0e9, 10 ** 8) == pytest.approx(1.0)


def test_sym_traffic_halves_the_matrix_stream():
    """Symmetric storage keeps (nnz + n) / 2 entries: the val/col part of V_min
    tends to one half of CRS's as Nnzr grows (Sec. 1.3.1), and the
    flops stay those of the full product."""
    n = 1000
    for nnzr in (7, 15, 101):
        nnz = n * nnzr
        full = pm.gpu_min_traffic(n, n, nnz)
        sym = pm.gpu_sym_min_traffic(n, nnz, (nnz + n) // 2)
        assert sym.flops == full.flops
        rest = 4 * (n + 1) + 16 * n
        ratio = (sym.bytes_min - rest) / (full.bytes_min - rest)
        assert ratio == pytest.approx((nnzr + 1) / (2 * nnzr))
