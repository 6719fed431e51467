"""Pins of the oracle's reverse Cuthill-McKee reordering and symmetric
permutation: a hand-worked example, a shuffled path (bandwidth 1), the BFS
level structure, components kept contiguous, the bandwidth of a shuffled grid
against SciPy's RCM, and the permuted product against dense indexing."""
import json
import os

import numpy as np
import pytest

import gen
import oracle
from oracle import reorder

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def sym_from_edges(n, edges, seed=0):
    rows, cols = [], []
    for a, b in edges:
        rows += [a, b]
        cols += [b, a]
    rows += list(range(n))
    cols += list(range(n))
    D = np.zeros((n, n))
    D[rows, cols] = 1.0
    r, c = np.nonzero(D)
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum(np.bincount(r, minlength=n))
    vals = np.random.default_rng(seed).integers(1, 9, len(r)).astype(np.float64)
    return gen.CSR(n, n, rp, c.astype(np.int32), vals)


def test_hand_worked_example():
    d = json.load(open(os.path.join(GOLD, "rcm_example.json")))
    A = gen.CSR(d["n"], d["n"], np.array(d["row_ptr"], np.int32), np.array(d["col_idx"], np.int32),
                np.ones(len(d["col_idx"])))
    assert reorder.rcm(A).tolist() == d["perm"]


def test_shuffled_path_gets_bandwidth_one():
    n = 200
    lab = np.random.default_rng(1).permutation(n)
    A = sym_from_edges(n, [(lab[i], lab[i + 1]) for i in range(n - 1)])
    assert reorder.bandwidth(A) > 50
    B = reorder.permute_csr(A, reorder.rcm(A))
    assert reorder.bandwidth(B) == 1


def test_permutation_levels_and_components():
    rng = np.random.default_rng(2)
    n = 300
    edges = [(int(a), int(b)) for a, b in rng.integers(0, 150, (200, 2)) if a != b]
    edges += [(int(a), int(b)) for a, b in rng.integers(150, 300, (200, 2)) if a != b]
    A = sym_from_edges(n, edges)
    perm = reorder.rcm(A)
    assert sorted(perm.tolist()) == list(range(n))
    adj = reorder.adjacency(A)
    order = perm[::-1]                      # Cuthill-McKee order
    pos = np.empty(n, int)
    pos[order] = np.arange(n)
    # each component occupies a contiguous range of the order
    comp = -np.ones(n, int)
    for s in range(n):
        if comp[s] < 0:
            stack = [s]
            comp[s] = s
            while stack:
                u = stack.pop()
                for v in adj[u]:
                    if comp[v] < 0:
                        comp[v] = s
                        stack.append(v)
    seq = comp[order]
    changes = np.flatnonzero(seq[1:] != seq[:-1])
    assert len(changes) == len(set(seq.tolist())) - 1
    # breadth-first: within a component, a node's neighbours are never more than one level away,
    # and the order visits levels in sequence
    for c0 in set(seq.tolist()):
        nodes = order[seq == c0]
        level = {int(nodes[0]): 0}
        for u in nodes:
            for v in adj[u]:
                if v not in level:
                    level[v] = level[int(u)] + 1
        lv = [level[int(u)] for u in nodes]
        assert lv == sorted(lv)
        for u in nodes:
            for v in adj[u]:
                assert abs(level[int(u)] - level[v]) <= 1


def test_grid_bandwidth_close_to_scipy():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    A = gen.laplace2d(24)
    lab = np.random.default_rng(3).permutation(A.n_rows).astype(np.int32)
    S = reorder.permute_csr(A, lab)
    assert reorder.bandwidth(S) > 300
    ours = reorder.bandwidth(reorder.permute_csr(S, reorder.rcm(S)))
    M = sp.csr_matrix((S.val, S.col_idx, S.row_ptr), shape=(S.n_rows, S.n_cols))
    theirs = reorder.bandwidth(reorder.permute_csr(S, csgraph.reverse_cuthill_mckee(M, symmetric_mode=True)))
    assert ours <= 1.25 * theirs + 1 and ours <= 2 * 24


@pytest.mark.parametrize("seed", range(3))
def test_permuted_matrix_and_product(seed):
    A = gen.random_csr(120, 120, 0.05, seed, integer=True, duplicates=True, unsorted=True)
    perm = np.random.default_rng(seed).permutation(120).astype(np.int32)
    B = reorder.permute_csr(A, perm)
    D = np.zeros((120, 120))
    for i in range(120):
        for j in range(A.row_ptr[i], A.row_ptr[i + 1]):
            D[i, A.col_idx[j]] += A.val[j]
    Dp = np.zeros((120, 120))
    for i in range(120):
        for j in range(B.row_ptr[i], B.row_ptr[i + 1]):
            Dp[i, B.col_idx[j]] += B.val[j]
    assert np.array_equal(Dp, D[perm][:, perm])
    for i in range(120):                     # columns sorted inside each row
        c = B.col_idx[B.row_ptr[i]:B.row_ptr[i + 1]]
        assert np.all(c[:-1] <= c[1:])
    x = np.random.default_rng(seed).integers(-100, 100, 120).astype(np.float64)
    assert np.array_equal(oracle.spmv(B, x[perm]), oracle.spmv(A, x)[perm])
