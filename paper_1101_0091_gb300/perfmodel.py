"""Node-level performance model of the CRS spMVM (Sec. 1.2, Eq. 1; Sec. 3.1, Eq. 2)
and its restatement for one GPU with HBM.

Paper form (cache-based CPU, write-allocate on C):

    B_CRS   = (12 + 24/Nnzr + kappa) / 2  =  6 + 12/Nnzr + kappa/2   bytes/flop   (Eq. 1)
    B_split =                                6 + 20/Nnzr + kappa/2   bytes/flop   (Eq. 2)

12 bytes per inner iteration are val (8) + col_idx (4); 16/Nnzr is the update
of C(i) (write-allocate + evict); 8/Nnzr is one load of B; kappa is the extra
B traffic per inner iteration; each inner iteration does 2 flops.  Reading used
here: kappa is the TOTAL extra bytes per nonzero beyond one load of B, so one
full extra reload of B adds 8/Nnzr (this reproduces the worked numbers of
Sec. 2: kappa = 2.5 from 18.1 GB/s and 2.25 GFlop/s, i.e. 37.3 bytes per row).

GPU form (no write-allocate on stores; row_ptr counted):

    V_min = nnz*(s_val + 4) + 4*(n_rows + 1) + 8*k*n_rows + 8*k*n_cols   bytes

with s_val = 8 (FP64 values) or 4 (FP32 values); flops = 2*k*nnz.  Measured
DRAM bytes beyond V_min, per nonzero, is the GPU kappa.
"""
from __future__ import annotations

from dataclasses import dataclass


def code_balance_crs(nnzr: float, kappa: float = 0.0) -> float:
    """Eq. 1: bytes per flop of the CRS loop."""
    return (12.0 + 24.0 / nnzr + kappa) / 2.0


def code_balance_split(nnzr: float, kappa: float = 0.0) -> float:
    """Eq. 2: bytes per flop when C is written twice (local + non-local pass)."""
    return 6.0 + 20.0 / nnzr + kappa / 2.0


def perf_limit(bandwidth: float, nnzr: float, kappa: float = 0.0) -> float:
    """Upper performance limit = bandwidth / code balance (units: bandwidth unit / (B/flop))."""
    return bandwidth / code_balance_crs(nnzr, kappa)


def kappa_from_measurement(bandwidth: float, performance: float, nnzr: float) -> float:
    """Solve Eq. 1 for kappa from the bandwidth drawn and the flop rate achieved
    (same units, e.g. GB/s and GFlop/s)."""
    return 2.0 * bandwidth / performance - 12.0 - 24.0 / nnzr


def kappa_bytes_per_row(kappa: float, nnzr: float) -> float:
    """Extra B traffic per matrix row (kappa is per inner iteration)."""
    return kappa * nnzr


def b_loads(kappa: float, nnzr: float) -> float:
    """How many times B is loaded in total: once, plus kappa*Nnzr/8 extra loads."""
    return 1.0 + kappa * nnzr / 8.0


def split_penalty(nnzr: float, kappa: float = 0.0) -> float:
    """Relative slowdown of the split kernel predicted by Eq. 2 vs Eq. 1."""
    return code_balance_split(nnzr, kappa) / code_balance_crs(nnzr, kappa) - 1.0


# --------------------------------------------------------------- GPU restatement

@dataclass(frozen=True)
class Traffic:
    bytes_min: int   # algorithmic minimum of DRAM bytes for one product
    flops: int       # 2 * k * nnz


def gpu_min_traffic(n_rows: int, n_cols: int, nnz: int, k: int = 1, val_bytes: int = 8) -> Traffic:
    """V_min for C = A*B with k right-hand sides (B read once, C written once)."""
    b = nnz * (val_bytes + 4) + 4 * (n_rows + 1) + 8 * k * n_rows + 8 * k * n_cols
    return Traffic(int(b), int(2 * k * nnz))


def gpu_sym_min_traffic(n: int, nnz: int, nnz_upper: int, k: int = 1, val_bytes: int = 8) -> Traffic:
    """V_min of the symmetric CRS product (Sec. 1.3.1) of a square matrix: the
    stored triangle (nnz_upper entries on or above the diagonal) is read once,
    B read once and C written once.  The flops are those of the full product."""
    b = nnz_upper * (val_bytes + 4) + 4 * (n + 1) + 8 * k * n + 8 * k * n
    return Traffic(int(b), int(2 * k * nnz))


def gpu_split_extra_bytes(n_halo_rows: int, k: int = 1) -> int:
    """Extra DRAM bytes of the split: the halo pass re-reads and re-writes C on
    halo rows (16k B each), plus the halo row list and its row pointers (8 B)."""
    return int(n_halo_rows * (16 * k + 8) + 4)


def gpu_code_balance(nnzr: float, kappa: float = 0.0, k: int = 1, val_bytes: int = 8) -> float:
    """Bytes per flop of the GPU form for a square matrix."""
    return (val_bytes + 4 + (4 + 16 * k) / nnzr + kappa) / (2.0 * k)


def kappa_gpu(dram_bytes: float, bytes_min: float, nnz: int) -> float:
    """Measured extra bytes per nonzero beyond V_min."""
    return (dram_bytes - bytes_min) / nnz if nnz else 0.0


def roofline_time(bytes_min: float, flops: float, hbm_gbs: float, fp64_gflops: float | None = None) -> float:
    """Lower bound on the product time in seconds: max(bytes/BW, flops/FP64 peak)."""
    t = bytes_min / (hbm_gbs * 1e9)
    if fp64_gflops:
        t = max(t, flops / (fp64_gflops * 1e9))
    return t
