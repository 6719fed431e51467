"""Pins of the oracle's CRS loop (Sec. 1.2) to things other than itself:
dense brute force, exact integer arithmetic, special matrices, the closed-form
eigenpairs of the 2D Laplacian, and invariants of the generated workloads."""
import math
from fractions import Fraction

import numpy as np
import pytest

import gen
import oracle

TOL = 1e-13


def dense_of(A) -> np.ndarray:
    """Dense matrix assembled entry by entry (duplicates summed)."""
    D = np.zeros((A.n_rows, A.n_cols), dtype=np.float64)
    for i in range(A.n_rows):
        for j in range(A.row_ptr[i], A.row_ptr[i + 1]):
            D[i, A.col_idx[j]] += A.val[j]
    return D


def exact_product(A, B) -> list:
    """Exact rational product sum_j a_ij * b_j (Python Fractions)."""
    out = []
    for i in range(A.n_rows):
        s = Fraction(0)
        for j in range(A.row_ptr[i], A.row_ptr[i + 1]):
            s += Fraction(float(A.val[j])) * Fraction(float(B[A.col_idx[j]]))
        out.append(s)
    return out


@pytest.mark.parametrize("seed", range(6))
def test_dense_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    n, m = int(rng.integers(1, 65)), int(rng.integers(1, 65))
    A = gen.random_csr(n, m, 0.3, seed, empty_rows=0.1, duplicates=(seed % 2 == 0), unsorted=(seed % 3 == 0))
    B = rng.uniform(-1, 1, m)
    C = oracle.spmv(A, B)
    exact = exact_product(A, B)
    S = oracle.abs_scale(A, B)
    for i in range(n):
        assert abs(Fraction(C[i]) - exact[i]) <= Fraction(TOL) * Fraction(S[i]), i
    # and against numpy's dense product in extended precision
    D = dense_of(A).astype(np.longdouble)
    ref = (D @ B.astype(np.longdouble)).astype(np.float64)
    assert oracle.max_err_ratio(C, ref, S, TOL) <= 1.0


@pytest.mark.parametrize("seed", range(4))
def test_integer_exact(seed):
    """|values| <= 2^10 with short rows: every partial sum is an exact double, so
    the result must equal the exact integer product bit for bit."""
    rng = np.random.default_rng(seed)
    A = gen.random_csr(200, 150, 0.05, seed, integer=True, empty_rows=0.05, duplicates=True)
    B = rng.integers(-1024, 1025, 150).astype(np.float64)
    C = oracle.spmv(A, B)
    exact = exact_product(A, B)
    assert all(C[i] == float(exact[i]) for i in range(A.n_rows))
    assert all(Fraction(C[i]) == exact[i] for i in range(A.n_rows))


def test_empty_rows_identity_permutation_and_1x1():
    # all rows empty
    A = gen.CSR(5, 3, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0))
    assert np.array_equal(oracle.spmv(A, np.ones(3)), np.zeros(5))
    assert not np.signbit(oracle.spmv(A, np.ones(3))).any()
    # 1x1
    A = gen.CSR(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0]))
    assert oracle.spmv(A, np.array([-2.5]))[0] == -7.5
    # identity and a permutation
    n = 97
    rng = np.random.default_rng(1)
    B = rng.uniform(-1, 1, n)
    I = gen.CSR(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    assert np.array_equal(oracle.spmv(I, B), B)
    p = rng.permutation(n).astype(np.int32)
    P = gen.CSR(n, n, np.arange(n + 1, dtype=np.int32), p, np.ones(n))
    assert np.array_equal(oracle.spmv(P, B), B[p])


def test_laplace2d_sine_modes():
    """2D 5-point Dirichlet Laplacian on 256x256: v = sin(p pi (x+1)/257) sin(q pi (y+1)/257)
    is an eigenvector with lambda = 4 - 2cos(p pi/257) - 2cos(q pi/257)."""
    nx = 256
    A = gen.laplace2d(nx)
    assert A.n_rows == 65536 and A.nnz == 326656
    x = np.arange(nx)
    for p, q in [(1, 1), (3, 7), (128, 200), (256, 256)]:
        # reduce p*(x+1) modulo 2*(nx+1) in integers so that the argument of sin is
        # below 2*pi and carries one rounding only
        sx = np.sin(math.pi * ((p * (x + 1)) % (2 * (nx + 1))) / (nx + 1))
        sy = np.sin(math.pi * ((q * (x + 1)) % (2 * (nx + 1))) / (nx + 1))
        v = (sy[:, None] * sx[None, :]).reshape(-1)       # row i = x + nx*y
        lam = 4 - 2 * math.cos(p * math.pi / (nx + 1)) - 2 * math.cos(q * math.pi / (nx + 1))
        Av = oracle.spmv(A, v)
        S = oracle.abs_scale(A, v)
        # loop rounding (1e-13 * S) plus the rounding of v and lambda themselves
        bound = TOL * S + 8 * np.finfo(float).eps * (np.abs(v).max() * 8)
        assert np.all(np.abs(Av - lam * v) <= bound), (p, q)


def test_laplace2d_mode_detects_transpose_and_sign():
    """The sine-mode pin is sensitive: a wrong neighbour sign breaks it."""
    nx = 16
    A = gen.laplace2d(nx)
    bad = gen.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, np.where(A.val < 0, 1.0, A.val))
    x = np.arange(nx)
    s = np.sin(math.pi * (x + 1) / (nx + 1))
    v = (s[:, None] * s[None, :]).reshape(-1)
    lam = 4 - 4 * math.cos(math.pi / (nx + 1))
    assert np.abs(oracle.spmv(A, v) - lam * v).max() < 1e-12
    assert np.abs(oracle.spmv(bad, v) - lam * v).max() > 1e-2


def transpose(A):
    """CSR transpose by counting sort (independent of the library)."""
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    order = np.lexsort((rows, A.col_idx))
    cnt = np.bincount(A.col_idx, minlength=A.n_cols)
    rp = np.zeros(A.n_cols + 1, np.int32)
    rp[1:] = np.cumsum(cnt)
    return gen.CSR(A.n_cols, A.n_rows, rp, rows[order].astype(np.int32), A.val[order])


def test_poisson3d_row_sum_invariant_and_symmetry():
    """Variable-coefficient 7-point stencil: diagonal = sum|off| + 1e-3 with all
    off-diagonals negative, so A*1 = 1e-3 per row; the edge draws make A = A^T."""
    n = 14
    A = gen.poisson3d_var(n, seed=0)
    assert A.n_rows == n ** 3 and A.nnz == 7 * n ** 3 - 6 * n * n
    one = np.ones(A.n_cols)
    r = oracle.spmv(A, one)
    S = oracle.abs_scale(A, one)
    assert np.all(np.abs(r - 1e-3) <= TOL * S)
    T = transpose(A)
    assert np.array_equal(T.row_ptr, A.row_ptr) and np.array_equal(T.col_idx, A.col_idx)
    assert np.array_equal(T.val, A.val)
    rng = np.random.default_rng(3)
    x, y = rng.uniform(-1, 1, A.n_cols), rng.uniform(-1, 1, A.n_cols)
    lhs, rhs = x @ oracle.spmv(A, y), y @ oracle.spmv(A, x)
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(x) @ oracle.abs_scale(A, y))


def test_eigen_shaped_symmetry():
    A = gen.eigen_shaped(20000, seed=0, window=1 << 12)
    T = transpose(A)
    assert np.array_equal(T.row_ptr, A.row_ptr) and np.array_equal(T.col_idx, A.col_idx)
    assert np.array_equal(T.val, A.val)
    rng = np.random.default_rng(4)
    x, y = rng.uniform(-1, 1, A.n_cols), rng.uniform(-1, 1, A.n_cols)
    lhs, rhs = x @ oracle.spmv(A, y), y @ oracle.spmv(A, x)
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(x) @ oracle.abs_scale(A, y))


def test_linearity():
    A = gen.random_csr(300, 250, 0.04, 7)
    rng = np.random.default_rng(7)
    x, y = rng.uniform(-1, 1, 250), rng.uniform(-1, 1, 250)
    a = 0.375  # exact in binary
    lhs = oracle.spmv(A, a * x + y)
    rhs = a * oracle.spmv(A, x) + oracle.spmv(A, y)
    S = oracle.abs_scale(A, np.abs(a * x) + np.abs(y))
    assert np.all(np.abs(lhs - rhs) <= 3 * TOL * S + 1e-300)


@pytest.mark.parametrize("k", [1, 3, 4, 16])
def test_spmm_dense(k):
    A = gen.random_csr(60, 50, 0.2, 11 + k, empty_rows=0.1, duplicates=True)
    rng = np.random.default_rng(k)
    B = rng.uniform(-1, 1, (50, k))
    C = oracle.spmm(A, B)
    ref = (dense_of(A).astype(np.longdouble) @ B.astype(np.longdouble)).astype(np.float64)
    S = oracle.abs_scale(A, B)
    assert oracle.max_err_ratio(C, ref, S, TOL) <= 1.0
    # column c of the block product is the single-vector product of column c
    for c in range(k):
        assert np.array_equal(C[:, c], oracle.spmv(A, np.ascontiguousarray(B[:, c])))


def test_f32val_is_rounded_values():
    """FP32-value form = FP64 loop on values rounded to float (numpy's own RN-even cast)."""
    A = gen.random_csr(200, 180, 0.05, 5)
    A.val = A.val * 3.3e-3 + 1.7  # values with bits below float precision
    rng = np.random.default_rng(5)
    B = rng.uniform(-1, 1, (180, 4))
    A32 = gen.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.val.astype(np.float32).astype(np.float64))
    assert np.array_equal(oracle.spmm(A, B, f32val=True), oracle.spmm(A32, B))
    # and differs from the FP64 product by no more than float rounding of each value
    d = np.abs(oracle.spmm(A, B, f32val=True) - oracle.spmm(A, B))
    assert np.all(d <= 2e-7 * oracle.abs_scale(A, B))
    assert d.max() > 0


def test_abs_scale_dense():
    A = gen.random_csr(40, 30, 0.3, 9)
    B = np.random.default_rng(9).uniform(-1, 1, 30)
    ref = np.abs(dense_of(A)) @ np.abs(B)  # no duplicates here, so |sum| = sum |.|
    assert np.allclose(oracle.abs_scale(A, B), ref, rtol=1e-14, atol=0)


def test_max_err_ratio_semantics():
    assert oracle.max_err_ratio([1.0], [1.0], [0.0], TOL) == 0.0
    assert oracle.max_err_ratio([1.0], [np.nextafter(1.0, 2.0)], [0.0], TOL) == float("inf")
    assert oracle.max_err_ratio([1.0 + 1e-14], [1.0], [1.0], TOL) == pytest.approx(0.1, rel=0.2)


def test_dot2_cancellation_row():
    """A row whose exact sum the plain loop loses completely: 1e16 + 1 - 1e16.
    The compensated evaluation recovers it exactly; the plain loop gives 0."""
    A = gen.CSR(1, 3, np.array([0, 3], np.int32), np.array([0, 1, 2], np.int32), np.array([1e16, 1.0, -1e16]))
    B = np.ones(3)
    assert oracle.spmv(A, B)[0] == 0.0
    assert oracle.spmm_dot2(A, B)[0] == 1.0
    # the rounding error of a product is kept too: (1 + 2^-30)^2 - 1 - 2^-29
    e = 2.0 ** -30
    A2 = gen.CSR(1, 3, np.array([0, 3], np.int32), np.array([0, 1, 2], np.int32), np.array([1.0 + e, -1.0, -2 * e]))
    B2 = np.array([1.0 + e, 1.0, 1.0])
    assert oracle.spmm_dot2(A2, B2)[0] == e * e          # exact: 2^-60


@pytest.mark.parametrize("seed", range(4))
def test_dot2_within_its_error_bound(seed):
    """Against exact rational sums on ill-conditioned random rows (terms that
    cancel to a small fraction of sum|ab|): |dot2 - exact| <= u|exact| +
    gamma_n^2 sum|ab| (Ogita, Rump, Oishi 2005), for every column of a block."""
    rng = np.random.default_rng(300 + seed)
    n, m, k = 40, 60, 3
    rows = [rng.choice(m, size=int(rng.integers(1, 30)), replace=False) for _ in range(n)]
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.concatenate(rows).astype(np.int32)
    va = rng.standard_normal(len(ci)) * 10.0 ** rng.integers(-8, 9, len(ci))
    A = gen.CSR(n, m, rp, ci, va)
    B = rng.standard_normal((m, k))
    got = oracle.spmm_dot2(A, B)
    plain = oracle.spmm(A, B)
    u = 2.0 ** -53
    worse = 0
    for c in range(k):
        ex = exact_product(A, B[:, c])
        for i in range(n):
            L = int(rp[i + 1] - rp[i])
            g = L * u / (1 - L * u)
            s = sum(abs(Fraction(float(A.val[j])) * Fraction(float(B[A.col_idx[j], c])))
                    for j in range(rp[i], rp[i + 1]))
            bound = u * abs(ex[i]) + Fraction(g * g) * s
            assert abs(Fraction(float(got[i, c])) - ex[i]) <= bound
            worse += abs(Fraction(float(plain[i, c])) - ex[i]) > abs(Fraction(float(got[i, c])) - ex[i])
    assert worse > 0   # the plain loop is measurably less accurate on these rows


def test_failed_check_attribution_message():
    """The message a failed GPU parity check carries: the worst entry and the
    distances of both sides from the compensated evaluation (a perturbed copy
    of the oracle's result stands in for a faulty kernel)."""
    from gpu_util import attribution
    A = gen.poisson3d_var(6)
    B = gen.rhs_block(A.n_cols, 2, seed=1)
    ref = oracle.spmm(A, B)
    y = ref.copy()
    y[17, 1] += 1e-6
    msg = attribution(y, ref, A, B, TOL)
    assert msg.startswith("worst entry (17, 1):")
    assert "|y - oracle| = 1.000e-06" in msg and "|oracle - dot2| = " in msg
