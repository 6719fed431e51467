"""ORACLE — test infrastructure only.

Matrix features that the cost model reads (row-length histogram, bandwidth,
column spread), written with plain numpy.  The library computes the same
vector in its own host code; the tests compare the two.

Feature vector (34 entries, float64), for a CRS matrix with n rows, nnz
nonzeros, row lengths L_i, and k right-hand sides:

  [0:13]   fraction of rows in length bin b, b(L) = 0 for L = 0, else
           min(1 + floor(log2 L), 12)   (bin 12 holds L >= 2048)
  [13:26]  fraction of nonzeros in the rows of bin b
  [26]     log2(1 + n)
  [27]     log2(1 + nnz)
  [28]     nnz / n                         (the paper's N_nzr)
  [29]     log2(1 + max L)
  [30]     std(L) / (1 + N_nzr)            (population standard deviation)
  [31]     max |i - j| / n_cols            (matrix bandwidth, relative)
  [32]     mean over non-empty rows of (max col - min col) / n_cols
  [33]     log2(k)
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 34
N_BINS = 13


def length_bin(L: np.ndarray) -> np.ndarray:
    L = np.asarray(L, dtype=np.int64)
    out = np.zeros(L.shape, dtype=np.int64)
    pos = L > 0
    # 1 + floor(log2 L) is the bit length of L
    bl = np.array([int(x).bit_length() for x in L[pos]], dtype=np.int64)
    out[pos] = np.minimum(bl, N_BINS - 1)
    return out


def features(A, k: int = 1) -> np.ndarray:
    n, ncols = A.n_rows, A.n_cols
    rp = np.asarray(A.row_ptr, dtype=np.int64)
    ci = np.asarray(A.col_idx, dtype=np.int64)
    L = np.diff(rp)
    nnz = int(rp[-1]) if n > 0 else 0
    f = np.zeros(N_FEATURES, dtype=np.float64)
    if n > 0:
        b = length_bin(L)
        for t in range(N_BINS):
            sel = b == t
            f[t] = sel.sum() / n
            f[N_BINS + t] = (L[sel].sum() / nnz) if nnz > 0 else 0.0
    f[26] = np.log2(1.0 + n)
    f[27] = np.log2(1.0 + nnz)
    mean = nnz / n if n > 0 else 0.0
    f[28] = mean
    f[29] = np.log2(1.0 + (L.max() if n > 0 else 0))
    f[30] = (np.sqrt(np.mean((L - mean) ** 2)) if n > 0 else 0.0) / (1.0 + mean)
    denom = max(1, ncols)
    if nnz > 0:
        rows = np.repeat(np.arange(n, dtype=np.int64), L)
        f[31] = np.abs(rows - ci).max() / denom
        ne = np.nonzero(L > 0)[0]
        spans = np.array([ci[rp[i]:rp[i + 1]].max() - ci[rp[i]:rp[i + 1]].min() for i in ne], dtype=np.int64)
        f[32] = spans.sum() / (len(ne) * denom)
    f[33] = np.log2(k)
    return f
