"""Seeded synthetic inputs (CRS matrices and right-hand sides).

Inputs only: this package holds none of the spMVM arithmetic.  The oracle and
the GPU path both consume what it produces and share nothing else.  The C
generators in ``gen.c`` are compiled on first use with the host C compiler.

Workloads (shapes of the paper's test matrices, Sec. 1.3.1):

* ``laplace2d(256)``        2D 5-point Laplacian, N = 65,536, nnz = 326,656.
* ``poisson3d_var(280)``    3D 7-point variable-coefficient Poisson, N = 21,952,000,
                            nnz = 153,193,600 (stand-in for the sAMG matrix, Nnzr ~ 7).
* ``eigen_shaped(6201600)`` symmetric eigenproblem-shaped matrix, N = 400 x 15,504
                            (stand-in for the HMeP Holstein-Hubbard matrix, Nnzr ~ 14).
* ``powerlaw_batch(512)``   512 uneven random matrices with power-law row lengths.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "_build", "libspmvgen.so")
_lock = threading.Lock()
_lib = None

# Streams of the counter-seeded generator: matrix and right-hand side of a
# single-matrix workload; member m of a batch uses 2m (matrix) and 2m+1 (RHS).
STREAM_MATRIX = 0
STREAM_RHS = 1


def build(force: bool = False) -> str:
    """Compile gen.c into a shared library (plain gcc, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Csr(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.POINTER(ctypes.c_int32)), ("col_idx", ctypes.POINTER(ctypes.c_int32)),
                ("val", ctypes.POINTER(ctypes.c_double))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Csr)
            i64, u64, dbl, i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
            lib.gen_free.argtypes = [P]
            lib.gen_laplace2d.argtypes = [i64, i64, P]
            lib.gen_poisson3d_var.argtypes = [i64, u64, u64, P]
            lib.gen_eigen_shaped.argtypes = [i64, i64, i32, dbl, u64, u64, P]
            lib.gen_powerlaw.argtypes = [i64, dbl, dbl, dbl, i64, i64, u64, u64, P]
            lib.gen_powerlaw_dim.argtypes = [u64, u64, dbl, dbl]
            lib.gen_powerlaw_dim.restype = i64
            lib.gen_uniform.argtypes = [u64, u64, i64, dbl, dbl, ctypes.c_void_p]
            _lib = lib
    return _lib


@dataclass
class CSR:
    """A CRS matrix on the host: row_ptr int32[n_rows+1], col_idx int32[nnz], val float64[nnz]."""
    n_rows: int
    n_cols: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1]) if self.n_rows > 0 else 0

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)


def _take(fn, *args) -> CSR:
    lib = _load()
    c = _Csr()
    rc = fn(*args, ctypes.byref(c))
    if rc != 0:
        raise RuntimeError(f"generator failed with code {rc}")
    try:
        n, nnz = c.n_rows, c.nnz
        rp = np.ctypeslib.as_array(c.row_ptr, shape=(n + 1,)).copy()
        ci = np.ctypeslib.as_array(c.col_idx, shape=(max(nnz, 1),))[:nnz].copy()
        va = np.ctypeslib.as_array(c.val, shape=(max(nnz, 1),))[:nnz].copy()
        return CSR(int(n), int(c.n_cols), rp, ci, va)
    finally:
        lib.gen_free(ctypes.byref(c))


def laplace2d(nx: int = 256, ny: int | None = None) -> CSR:
    """2D 5-point Dirichlet Laplacian: 4 on the diagonal, -1 for each grid neighbour; row i = x + nx*y."""
    return _take(_load().gen_laplace2d, nx, nx if ny is None else ny)


def poisson3d_var(n: int = 280, seed: int = 0) -> CSR:
    """3D 7-point variable-coefficient Poisson stencil on an n^3 grid; row i = x + n*(y + n*z)."""
    return _take(_load().gen_poisson3d_var, n, seed, STREAM_MATRIX)


def eigen_shaped(n: int = 6_201_600, seed: int = 0, window: int = 1 << 20, pairs: int = 5,
                 band_p: float = 0.7) -> CSR:
    """Symmetric eigenproblem-shaped matrix (diagonal N(0,1), +-1/+-2 bands kept with band_p,
    `pairs` scattered symmetric partners per row within +-window)."""
    return _take(_load().gen_eigen_shaped, n, window, pairs, band_p, seed, STREAM_MATRIX)


def powerlaw(n: int, alpha: float = 2.2, lmin: int = 1, lmax: int = 2000, seed: int = 0,
             stream: int = STREAM_MATRIX, dim_lo: float = 1e3, dim_hi: float = 2e5) -> CSR:
    """Random square matrix with power-law row lengths; n <= 0 draws n log-uniformly in [dim_lo, dim_hi]."""
    return _take(_load().gen_powerlaw, n, dim_lo, dim_hi, alpha, lmin, lmax, seed, stream)


def powerlaw_batch_member(m: int, seed: int = 0, alpha: float = 2.2, lmax: int = 2000,
                          dim_lo: float = 1e3, dim_hi: float = 2e5) -> CSR:
    """Member m of the uneven batch: dimension log-uniform in [dim_lo, dim_hi], stream 2m."""
    return powerlaw(0, alpha, 1, lmax, seed, 2 * m, dim_lo, dim_hi)


def powerlaw_batch(count: int = 512, seed: int = 0, **kw) -> list[CSR]:
    return [powerlaw_batch_member(m, seed, **kw) for m in range(count)]


def uniform(n: int, seed: int = 0, stream: int = STREAM_RHS, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n values uniform in [lo, hi) from generator (seed, stream)."""
    out = np.empty(n, dtype=np.float64)
    _load().gen_uniform(seed, stream, n, lo, hi, out.ctypes.data)
    return out


def rhs_block(n: int, k: int, seed: int = 0, stream: int = STREAM_RHS) -> np.ndarray:
    """Row-major n x k block of right-hand sides, U[-1, 1)."""
    return uniform(n * k, seed, stream).reshape(n, k)


# ---------------------------------------------------------------- small cases
# Small seeded matrices for parity tests, drawn with numpy's PCG64 generator.

def random_csr(n_rows: int, n_cols: int, density: float, seed: int, *, integer: bool = False,
               max_abs: int = 1 << 10, empty_rows: float = 0.0, duplicates: bool = False,
               unsorted: bool = False) -> CSR:
    """Random CRS matrix.  integer=True draws integer values in [-max_abs, max_abs];
    empty_rows forces that fraction of rows to be empty; duplicates repeats some
    column indices inside rows; unsorted shuffles the entry order of each row."""
    rng = np.random.default_rng(seed)
    lens = rng.binomial(n_cols, density, size=n_rows) if n_cols > 0 else np.zeros(n_rows, dtype=np.int64)
    if empty_rows > 0:
        lens[rng.random(n_rows) < empty_rows] = 0
    cols, vals = [], []
    for r in range(n_rows):
        L = int(lens[r])
        if L == 0:
            cols.append(np.zeros(0, np.int32)); vals.append(np.zeros(0))
            continue
        c = np.sort(rng.choice(n_cols, size=L, replace=False)).astype(np.int32)
        if duplicates and L > 1:
            c[rng.integers(0, L)] = c[rng.integers(0, L)]
            c = np.sort(c)
        if unsorted:
            rng.shuffle(c)
        if integer:
            v = rng.integers(-max_abs, max_abs + 1, size=L).astype(np.float64)
        else:
            v = rng.uniform(-1.0, 1.0, size=L)
        cols.append(c); vals.append(v)
    rp = np.zeros(n_rows + 1, dtype=np.int32)
    rp[1:] = np.cumsum(lens)
    ci = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    va = np.concatenate(vals).astype(np.float64) if vals else np.zeros(0)
    return CSR(n_rows, n_cols, rp, ci, va)


def csr_from_lengths(lengths, n_cols: int, seed: int, integer: bool = False) -> CSR:
    """CRS matrix with the given row lengths, distinct uniform columns per row."""
    rng = np.random.default_rng(seed)
    lengths = np.asarray(lengths, dtype=np.int64)
    rp = np.zeros(len(lengths) + 1, dtype=np.int32)
    rp[1:] = np.cumsum(lengths)
    cols = [np.sort(rng.choice(n_cols, size=int(L), replace=False)) for L in lengths]
    ci = np.concatenate(cols).astype(np.int32) if len(cols) else np.zeros(0, np.int32)
    nnz = int(rp[-1])
    va = (rng.integers(-1024, 1025, size=nnz).astype(np.float64) if integer
          else rng.uniform(-1.0, 1.0, size=nnz))
    return CSR(len(lengths), n_cols, rp, ci, va)


def symmetric_from(A: CSR, seed: int = 0, shuffle: bool = False) -> CSR:
    """Symmetric square matrix (n = A.n_rows) from A's entries with
    row <= col < n: each such entry (i, j, v) is kept and, off the diagonal,
    mirrored as (j, i, v), so duplicates mirror one to one.  Entries of a row
    are in ascending column order (stable), or in a seeded random order."""
    n = A.n_rows
    r = np.repeat(np.arange(n, dtype=np.int64), np.diff(A.row_ptr).astype(np.int64))
    c = A.col_idx.astype(np.int64)
    v = A.val.astype(np.float64)
    keep = (c >= r) & (c < n)
    r, c, v = r[keep], c[keep], v[keep]
    off = r != c
    R = np.concatenate([r, c[off]])
    Cc = np.concatenate([c, r[off]])
    V = np.concatenate([v, v[off]])
    if shuffle:
        order = np.lexsort((np.random.default_rng(seed).random(len(R)), R))
    else:
        order = np.lexsort((Cc, R))
    rp = np.zeros(n + 1, dtype=np.int32)
    rp[1:] = np.cumsum(np.bincount(R, minlength=n))
    return CSR(n, n, rp, Cc[order].astype(np.int32), V[order])


def kronecker_transpose(n1: int = 400, n2: int = 15_504) -> np.ndarray:
    """Renumbering of an n1 x n2 product basis from index e*n2 + p (the second
    factor contiguous) to p*n1 + e (the first factor contiguous), as a
    permutation perm[new] = old: perm[p*n1 + e] = e*n2 + p.  Sec. 1.3.1's two
    numberings of the Hamiltonian basis differ in exactly this way."""
    e = np.arange(n1, dtype=np.int64)
    p = np.arange(n2, dtype=np.int64)
    return (e[None, :] * n2 + p[:, None]).reshape(-1).astype(np.int32)
