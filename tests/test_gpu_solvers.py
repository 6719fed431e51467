"""The iterative consumers of the product (CG and Lanczos on k columns) through
the C ABI against the oracle's restatements: iterates, residual histories,
iteration counts, freezing, breakdown, determinism, the graph and eager paths,
every plan variant, and a full-size run on the 3D Poisson workload."""
import math

import numpy as np
import pytest

import gen
import oracle
from oracle import solvers as osol
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def run_cg(lib, A, B, X0=None, variant=None, **kw):
    import torch
    k = B.shape[1]
    with lib.Plan.from_csr(A, **({} if variant is None else {"variant": variant})) as p, lib.Solver(p, k) as s:
        Bd = dev(np.ascontiguousarray(B))
        Xd = dev(np.zeros_like(B) if X0 is None else np.ascontiguousarray(X0))
        it, rr, summ = s.cg(Bd, Xd, **kw)
        return host(Xd), it, rr, summ


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 8, 13, 16])
def test_cg_fixed_iterations_match_oracle(lib, k):
    """rtol = 0: every column runs all iterations; the iterate and R.R follow
    the oracle's (different rounding: FMA and reduction order).  k covers every
    way the vector kernels walk a block: pairs (1), rows (2, 4), 4-column groups
    (8, 16) and masked scalar rows (3, 6, 13)."""
    A = gen.poisson3d_var(12)
    B = gen.rhs_block(A.n_cols, k, seed=k) if k > 1 else gen.uniform(A.n_cols, seed=1).reshape(-1, 1)
    for iters in (1, 5, 30):
        X, it, rr, _ = run_cg(lib, A, B, max_iter=iters, rtol=0.0, check_every=7)
        Xo, info = osol.cg(A, B, max_iter=iters, rtol=0.0)
        assert np.all(it == iters)
        for c in range(k):
            assert rel(X[:, c], Xo[:, c]) < 1e-10, (iters, c)
            assert abs(rr[c] - info["rr"][c]) <= 1e-8 * info["rr"][c]


def test_cg_converges_to_known_solution(lib):
    """Poisson workload: A * 1 = 1e-3, so b = 1e-3 has the solution 1."""
    A = gen.poisson3d_var(20)
    B = np.full((A.n_rows, 1), 1e-3)
    X, it, rr, summ = run_cg(lib, A, B, max_iter=3000, rtol=1e-10, check_every=16)
    Xo, info = osol.cg(A, B, max_iter=3000, rtol=1e-10)
    assert summ.converged == 1 and summ.breakdown == 0
    assert abs(int(it[0]) - int(info["iterations"][0])) <= 1
    assert np.abs(X[:, 0] - 1.0).max() < 1e-6
    true_r = B[:, 0] - oracle.spmv(A, X[:, 0])
    assert np.linalg.norm(true_r) <= 1.5e-10 * np.linalg.norm(B)


def test_cg_columns_freeze_and_zero_rhs(lib):
    A = gen.poisson3d_var(10)
    rng = np.random.default_rng(2)
    B = np.stack([np.zeros(A.n_rows), rng.standard_normal(A.n_rows), np.full(A.n_rows, 1e-3),
                  rng.standard_normal(A.n_rows)], 1)
    X, it, rr, summ = run_cg(lib, A, B, max_iter=500, rtol=1e-8, check_every=5)
    Xo, info = osol.cg(A, B, max_iter=500, rtol=1e-8)
    assert it[0] == 0 and np.all(X[:, 0] == 0)
    assert np.all(np.abs(it.astype(int) - info["iterations"].astype(int)) <= 1)
    assert summ.converged == 4
    for c in range(1, 4):
        assert rel(X[:, c], Xo[:, c]) < 1e-7


def test_cg_columns_freeze_in_column_groups(lib):
    """k = 8 (4-column groups): zero, fast and slow columns in one group freeze
    independently at the oracle's iteration counts."""
    A = gen.poisson3d_var(10)
    rng = np.random.default_rng(6)
    cols = [np.zeros(A.n_rows), rng.standard_normal(A.n_rows), np.full(A.n_rows, 1e-3),
            rng.standard_normal(A.n_rows), np.zeros(A.n_rows), np.full(A.n_rows, -2e-3),
            rng.standard_normal(A.n_rows), rng.standard_normal(A.n_rows)]
    B = np.stack(cols, 1)
    X, it, rr, summ = run_cg(lib, A, B, max_iter=500, rtol=1e-8, check_every=5)
    Xo, info = osol.cg(A, B, max_iter=500, rtol=1e-8)
    assert it[0] == 0 and it[4] == 0 and np.all(X[:, [0, 4]] == 0)
    assert np.all(np.abs(it.astype(int) - info["iterations"].astype(int)) <= 1)
    assert summ.converged == 8
    for c in (1, 2, 3, 5, 6, 7):
        assert rel(X[:, c], Xo[:, c]) < 1e-7


def test_cg_initial_guess(lib):
    A = gen.poisson3d_var(10)
    B = gen.rhs_block(A.n_cols, 2, seed=3)
    X0 = np.full_like(B, 0.5)
    X, it, rr, _ = run_cg(lib, A, B, X0=X0, max_iter=12, rtol=0.0, check_every=4)
    Xo, info = osol.cg(A, B, X0=X0, max_iter=12, rtol=0.0)
    assert rel(X, Xo) < 1e-10


def test_cg_breakdown_on_indefinite(lib):
    A = gen.CSR(2, 2, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, -1.0]))
    X, it, rr, summ = run_cg(lib, A, np.array([[1.0], [1.0]]), max_iter=10, rtol=1e-12, check_every=1)
    assert summ.breakdown == 1 and summ.converged == 0


def test_cg_deterministic_and_graph_eager_identical(lib):
    """Fixed-order reductions: repeated solves, and any polling interval (graph
    replays vs single iterations), give the same bits."""
    A = gen.eigen_shaped(20_000, window=1 << 12)
    # shift to make it positive definite: A + s I with s above the Gershgorin bound
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    d = rows == A.col_idx
    s = np.bincount(rows, weights=np.abs(A.val), minlength=A.n_rows).max() + 1.0
    val = A.val.copy()
    val[d] += s
    A = gen.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, val)
    for k in (2, 16):
        B = gen.rhs_block(A.n_cols, k, seed=5)
        runs = [run_cg(lib, A, B, max_iter=37, rtol=0.0, check_every=ce)[0] for ce in (1, 7, 37, 100, 7)]
        for r in runs[1:]:
            assert np.array_equal(r, runs[0])
        Xo, _ = osol.cg(A, B, max_iter=37, rtol=0.0)
        assert rel(runs[0], Xo) < 1e-10


@pytest.mark.parametrize("variant", ["SPMV_CRS_STAGED", "SPMV_CRS_L4", "SPMV_SELL", "SPMV_SYM"])
def test_cg_through_every_variant(lib, variant):
    A = gen.poisson3d_var(14)
    B = gen.rhs_block(A.n_cols, 4, seed=8)
    X, it, rr, summ = run_cg(lib, A, B, variant=getattr(lib, variant), max_iter=2000, rtol=1e-9, check_every=10)
    assert summ.converged == 4
    for c in range(4):
        true_r = B[:, c] - oracle.spmv(A, X[:, c])
        assert np.linalg.norm(true_r) <= 2e-9 * np.linalg.norm(B[:, c])


def test_solver_argument_errors(lib):
    A = gen.random_csr(20, 30, 0.2, 1)
    with lib.Plan.from_csr(A) as p:
        with pytest.raises(lib.SpmvError):
            lib.Solver(p, 1)
    A = gen.poisson3d_var(4)
    with lib.Plan.from_csr(A, max_k=4) as p:
        with pytest.raises(lib.SpmvError):
            lib.Solver(p, 5)
        with lib.Solver(p, 2) as s:
            import torch
            Bd = torch.zeros((A.n_rows, 2), dtype=torch.float64, device="cuda")
            with pytest.raises(lib.SpmvError):
                s.cg(Bd, Bd.clone(), check_every=0)
            with pytest.raises(lib.SpmvError):
                s.lanczos(Bd, 0)
            # a block that starts 8 bytes into an allocation is rejected
            big = torch.zeros(A.n_rows * 2 + 1, dtype=torch.float64, device="cuda")
            off = big[1:].view(A.n_rows, 2)
            with pytest.raises(lib.SpmvError) as e:
                s.cg(off, Bd.clone())
            assert "aligned" in str(e.value)


@pytest.mark.parametrize("k", [1, 2, 5, 8, 16])
def test_lanczos_matches_oracle(lib, k):
    import torch
    A = gen.eigen_shaped(20_000, window=1 << 12)
    V0 = gen.rhs_block(A.n_cols, k, seed=10 + k) if k > 1 else gen.uniform(A.n_cols, seed=3).reshape(-1, 1)
    m = 30
    with lib.Plan.from_csr(A) as p, lib.Solver(p, k) as s:
        a, b = s.lanczos(dev(np.ascontiguousarray(V0)), m)
    ao, bo = osol.lanczos(A, V0, m)
    # the recurrence amplifies rounding differences slowly over the first steps
    assert np.abs(a[:10] - ao[:10]).max() < 1e-11 * np.abs(ao[:10]).max()
    assert np.abs(b[:10] - bo[:10]).max() < 1e-11 * np.abs(bo[:10]).max()
    for c in range(k):
        rg, ro = osol.ritz_values(a[:, c], b[:, c]), osol.ritz_values(ao[:, c], bo[:, c])
        assert abs(rg[-1] - ro[-1]) < 1e-9 * abs(ro[-1]) and abs(rg[0] - ro[0]) < 1e-9 * abs(ro[0])


def test_lanczos_laplace_spectrum_and_zero_start(lib):
    A = gen.laplace2d(16)
    V0 = gen.rhs_block(A.n_cols, 3, seed=4)
    V0[:, 1] = 0.0
    with lib.Plan.from_csr(A) as p, lib.Solver(p, 3) as s:
        a, b = s.lanczos(dev(V0), 80)
    assert np.all(a[:, 1] == 0) and np.all(b[:, 1] == 0)
    for c in (0, 2):
        r = osol.ritz_values(a[:, c], b[:, c])
        assert abs(r[-1] - (4 + 4 * math.cos(math.pi / 17))) < 1e-9
        assert abs(r[0] - (4 - 4 * math.cos(math.pi / 17))) < 1e-9


def test_cg_full_size_poisson280(lib):
    """The 280^3 workload, k = 4, 25 iterations through the default plan: the
    recurrence residual equals the true residual |B - A X| (oracle product), and
    the first iterate equals alpha_1 B with alpha_1 = B.B / B.AB (oracle)."""
    import torch
    A = gen.poisson3d_var(280)
    k = 4
    B = gen.rhs_block(A.n_cols, k, seed=0)
    with lib.Plan.from_csr(A) as p, lib.Solver(p, k) as s:
        Bd = dev(B)
        Xd = torch.zeros_like(Bd)
        s.cg(Bd, Xd, max_iter=1, rtol=0.0, check_every=1)
        X1 = host(Xd)
        Xd.zero_()
        it, rr, summ = s.cg(Bd, Xd, max_iter=25, rtol=0.0, check_every=25)
        X = host(Xd)
    assert np.all(it == 25)
    AB = oracle.spmm(A, B)
    alpha1 = np.array([np.dot(B[:, c], B[:, c]) / np.dot(B[:, c], AB[:, c]) for c in range(k)])
    assert rel(X1, alpha1 * B) < 1e-12
    R_true = B - oracle.spmm(A, X)
    for c in range(k):
        nb = np.linalg.norm(B[:, c])
        assert abs(math.sqrt(rr[c]) - np.linalg.norm(R_true[:, c])) <= 1e-9 * nb
        assert math.sqrt(rr[c]) < 0.5 * nb


def test_solvers_on_an_empty_matrix(lib):
    import torch
    A = gen.CSR(0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    with lib.Plan.from_csr(A) as p, lib.Solver(p, 2) as s:
        Bd = torch.zeros((0, 2), dtype=torch.float64, device="cuda")
        it, rr, summ = s.cg(Bd, Bd.clone(), max_iter=10, rtol=1e-8)
        assert np.all(it == 0) and summ.converged == 2
        a, b = s.lanczos(Bd, 3)
        assert np.all(a == 0) and np.all(b == 0)


def test_cg_recaptures_after_the_plan_changes(lib):
    """The iterations replay from a captured graph; switching the plan's kernel
    (here SELL with a new sigma, which rebuilds its arrays) or its tuning makes
    the next solve capture again, so the results follow the oracle."""
    import torch
    A = gen.poisson3d_var(12)
    B = gen.rhs_block(A.n_cols, 2, seed=12)
    Xo, _ = osol.cg(A, B, max_iter=20, rtol=0.0)
    with lib.Plan.from_csr(A, variant=lib.SPMV_SELL, sell_sigma=256) as p, lib.Solver(p, 2) as s:
        Bd = dev(B)
        Xd = torch.zeros_like(Bd)
        for step in range(4):
            if step == 1:
                p.set_variant(lib.SPMV_SELL, 4096)
            elif step == 2:
                p.set_tuning(prefetch_distance=0)
            elif step == 3:
                p.set_variant(lib.SPMV_CRS_STAGED)
            Xd.zero_()
            s.cg(Bd, Xd, max_iter=20, rtol=0.0, check_every=20)
            assert rel(host(Xd), Xo) < 1e-10, step
