"""ORACLE — test infrastructure only.

Reverse Cuthill-McKee reordering (Sec. 1.3.1 applies it to the Hamiltonian
matrix to make the accesses to B more local), restated in plain Python from
Cuthill and McKee (1969) and George and Liu (1981), with every tie broken in
a fixed way so that the permutation is unique:

* graph: the pattern of A + A^T without self loops; the degree of a node is
  its number of distinct neighbours;
* components are taken in order of their smallest node index; in each, the
  start node comes from the pseudo-peripheral node search: r = the node of
  minimum degree (ties: smallest index); repeat { build the BFS level
  structure from r; among the nodes of its last level take the one of
  minimum degree (ties: smallest index); if its level structure is deeper,
  it becomes r, else stop };
* Cuthill-McKee: breadth-first search from the start node, each dequeued
  node appending its unvisited neighbours in ascending (degree, index);
* the reverse of the whole order is the permutation: perm[new] = old.

``permute_csr`` applies it symmetrically: row r of A' is row perm[r] of A,
its columns relabelled by the inverse permutation and sorted ascending
(stable, so duplicates keep their order).
"""
from __future__ import annotations

from collections import deque

import numpy as np


def adjacency(A) -> list[list[int]]:
    """Sorted distinct neighbours of every node in the pattern of A + A^T (no self loops)."""
    n = A.n_rows
    nb = [set() for _ in range(n)]
    for i in range(n):
        for j in A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]]:
            j = int(j)
            if j != i:
                nb[i].add(j)
                nb[j].add(i)
    return [sorted(s) for s in nb]


def _levels(adj, root, allowed):
    """BFS level structure from root (list of levels)."""
    seen = {root}
    levels = [[root]]
    while True:
        nxt = []
        for u in levels[-1]:
            for v in adj[u]:
                if v not in seen:
                    seen.add(v)
                    nxt.append(v)
        if not nxt:
            return levels
        levels.append(nxt)


def _pseudo_peripheral(adj, deg, component):
    r = min(component, key=lambda u: (deg[u], u))
    levels = _levels(adj, r, None)
    while True:
        cand = min(levels[-1], key=lambda u: (deg[u], u))
        cl = _levels(adj, cand, None)
        if len(cl) > len(levels):
            r, levels = cand, cl
        else:
            return r


def rcm(A) -> np.ndarray:
    """RCM permutation (perm[new] = old) of a square matrix."""
    assert A.n_rows == A.n_cols
    n = A.n_rows
    adj = adjacency(A)
    deg = [len(a) for a in adj]
    visited = [False] * n
    order = []
    for s in range(n):
        if visited[s]:
            continue
        component = [u for lvl in _levels(adj, s, None) for u in lvl]
        start = _pseudo_peripheral(adj, deg, component)
        visited[start] = True
        q = deque([start])
        while q:
            u = q.popleft()
            order.append(u)
            for v in sorted((v for v in adj[u] if not visited[v]), key=lambda v: (deg[v], v)):
                visited[v] = True
                q.append(v)
    return np.array(order[::-1], dtype=np.int32)


def permute_csr(A, perm):
    """A' = P A P^T for perm[new] = old; rows in new order, columns relabelled and sorted (stable)."""
    import gen
    perm = np.asarray(perm, dtype=np.int64)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    rows, cols, vals = [], [], []
    rp = [0]
    for r in range(A.n_rows):
        o = perm[r]
        c = inv[A.col_idx[A.row_ptr[o]:A.row_ptr[o + 1]].astype(np.int64)]
        v = A.val[A.row_ptr[o]:A.row_ptr[o + 1]]
        order = np.argsort(c, kind="stable")
        cols.append(c[order])
        vals.append(v[order])
        rp.append(rp[-1] + len(c))
    ci = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    va = np.concatenate(vals) if vals else np.zeros(0)
    return gen.CSR(A.n_rows, A.n_cols, np.array(rp, np.int32), ci, va)


def bandwidth(A) -> int:
    """max |i - j| over the stored entries (0 for an empty matrix)."""
    if A.nnz == 0:
        return 0
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    return int(np.abs(rows - A.col_idx.astype(np.int64)).max())
