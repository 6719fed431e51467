"""The bench's secondary bounds (host logic), worked by hand on tiny inputs:
the far-entry count behind the eigenproblem request roof, the batch's per-row
mixed bound and its random-read DRAM bound."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
import gen  # noqa: E402


def csr(n_rows, n_cols, rows):
    rp = np.zeros(n_rows + 1, np.int32)
    for i, r in enumerate(rows):
        rp[i + 1] = rp[i] + len(r)
    ci = np.array([c for r in rows for c in r], np.int32)
    return gen.CSR(n_rows, n_cols, rp, ci, np.ones(len(ci)))


def test_far_entries_counts_distances_beyond_the_reach():
    # row 0: 0 (d 0), 32 (d 32, near), 33 (d 33, far); row 40: 7 (d 33, far), 40 (d 0); row 41: 100 (d 59, far)
    rows = [[0, 32, 33]] + [[] for _ in range(39)] + [[7, 40], [100]]
    A = csr(42, 128, rows)
    assert bench.far_entries(A) == 3
    assert bench.far_entries(A, reach=58) == 1
    assert bench.far_entries(A, reach=59) == 0


def test_mixed_row_bound_by_hand(monkeypatch):
    monkeypatch.setitem(bench.MACHINE, "fp64_gflops", 1000.0)
    hbm = 100.0   # GB/s: 1 byte = 0.01 ns
    # row of 1 entry: HBM 80 B -> 0.8 ns, FP64 8 flops -> 0.008 ns: 0.8 ns
    # row of 100 entries: HBM 1268 B -> 12.68 ns, FP64 800 flops -> 0.8 ns: 12.68 ns
    # empty row: HBM 68 B -> 0.68 ns
    A = csr(3, 200, [[0], list(range(100)), []])
    r = bench.mixed_row_bound([A], kern_s=28.32e-9, hbm=hbm)
    assert r["mixed_bound_us"] == pytest.approx(round((0.8 + 12.68 + 0.68) * 1e-3, 1))
    assert r["mixed_frac"] == pytest.approx(0.5, abs=1e-4)
    # FP64-bound rows: at 1 GFLOP/s, 8 flops per entry take 8 ns while 12 B take 0.12 ns
    monkeypatch.setitem(bench.MACHINE, "fp64_gflops", 1.0)
    r = bench.mixed_row_bound([csr(1, 10, [list(range(10))])], kern_s=160e-9, hbm=hbm)
    assert r["mixed_frac"] == pytest.approx(0.5, abs=1e-4)   # 80 ns of FP64 time against 1.88 ns of HBM


def test_random_dram_bound_by_hand(monkeypatch):
    monkeypatch.setitem(bench.MACHINE, "dram_gathers_per_s", 1e9)   # one 64-byte block per ns
    As = [csr(4, 16, [[0], [1], [2], [3]]), csr(2, 8, [[0], [1]])]
    b_bytes = 8 * 4 * (16 + 8)                 # k = 4: 32 B per column, 24 columns = 768 B = 12 blocks
    bytes_min = b_bytes + 1000                 # 1000 B more streamed at 100 GB/s: 10 ns
    r = bench.random_dram_bound(As, bytes_min, 100.0, kern_s=44e-9)
    assert r["random_dram_bound_us"] == pytest.approx(0.0, abs=1e-9)   # 22 ns rounds to 0.0 us
    assert r["random_dram_frac"] == pytest.approx(22.0 / 44.0, abs=1e-4)
    monkeypatch.setitem(bench.MACHINE, "dram_gathers_per_s", None)
    assert bench.random_dram_bound(As, bytes_min, 100.0, kern_s=44e-9) == {}
