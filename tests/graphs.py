"""Small graph builders and pure-Python checks used by the tests.

Nothing here calls the CUDA library or the oracle; these helpers build CSR
arrays from edge lists and state BFS facts independently (brute-force
relaxation, union-find components, the BFS invariants).
"""
from __future__ import annotations

import numpy as np


def csr_from_edges(n: int, edges, symmetric: bool = True):
    """CSR (int64 row_ptr, int32 col) from (u, v) pairs; both directions when symmetric.

    Keeps self-loops and repeated pairs exactly as given, rows sorted.
    """
    rows = [[] for _ in range(n)]
    for u, v in edges:
        rows[u].append(v)
        if symmetric and u != v:
            rows[v].append(u)
        elif symmetric and u == v:
            rows[u].append(u)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    for i in range(n):
        rows[i].sort()
        row_ptr[i + 1] = row_ptr[i] + len(rows[i])
    col = np.array([v for r in rows for v in r], dtype=np.int32)
    return row_ptr, col


def brute_force_dist(n: int, edges, src: int):
    """Bellman-Ford style fixpoint: repeat d[v] = min(d[v], d[u] + 1) over all arcs."""
    inf = n + 10
    d = [inf] * n
    d[src] = 0
    changed = True
    while changed:
        changed = False
        for u, v in edges:
            for a, b in ((u, v), (v, u)):
                if d[a] + 1 < d[b]:
                    d[b] = d[a] + 1
                    changed = True
    return np.array([x if x < inf else -1 for x in d], dtype=np.int32)


def path_graph(n):
    return csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])


def star_graph(n):
    return csr_from_edges(n, [(0, i) for i in range(1, n)])


def complete_graph(n):
    return csr_from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def cycle_graph(n):
    return csr_from_edges(n, [(i, (i + 1) % n) for i in range(n)])


def components(row_ptr, col):
    """Component label of every vertex: scipy's connected_components when
    the graph is large, the union-find below otherwise."""
    n = len(row_ptr) - 1
    if len(col) > 20000:
        import scipy.sparse as sp
        from scipy.sparse.csgraph import connected_components
        a = sp.csr_matrix((np.ones(len(col), dtype=np.int8), col, row_ptr), shape=(n, n))
        return connected_components(a, directed=False)[1].astype(np.int64)
    return union_find(row_ptr, col)


def union_find(row_ptr, col):
    """Union-find component label of every vertex (smallest id of its component)."""
    n = len(row_ptr) - 1
    parent = np.arange(n, dtype=np.int64)

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    src = np.repeat(np.arange(n), np.diff(row_ptr))
    for u, v in zip(src.tolist(), col.tolist()):
        ru, rv = find(u), find(v)
        if ru != rv:
            parent[max(ru, rv)] = min(ru, rv)
    return np.array([find(x) for x in range(n)], dtype=np.int64)


def check_bfs_invariants(row_ptr, col, src, dist, comp=None):
    """Assert the BFS invariants on ``dist``; returns the reached count.

    d[src] = 0; on every arc with both ends reached |d(u) - d(v)| <= 1 and no
    arc joins a reached and an unreached vertex; every reached v != src has a
    neighbour at d(v) - 1; d = -1 exactly off src's union-find component; the
    level histogram sums to the component size.
    """
    n = len(row_ptr) - 1
    dist = np.asarray(dist)
    assert dist.shape == (n,)
    assert dist[src] == 0
    u = np.repeat(np.arange(n), np.diff(row_ptr))
    v = col.astype(np.int64)
    du, dv = dist[u], dist[v]
    both = (du >= 0) & (dv >= 0)
    assert np.all(np.abs(du[both] - dv[both]) <= 1), "edge spans more than one level"
    assert not np.any((du >= 0) != (dv >= 0)), "edge joins reached and unreached vertex"
    # parent at d-1
    has_parent = np.zeros(n, dtype=bool)
    ok = both & (du == dv - 1)
    has_parent[v[ok]] = True
    reached = dist >= 0
    need = reached.copy()
    need[src] = False
    assert np.all(has_parent[need]), "reached vertex without a neighbour one level closer"
    if comp is None:
        comp = components(row_ptr, col)
    in_comp = comp == comp[src]
    assert np.array_equal(in_comp, reached), "reached set differs from the source's component"
    hist = np.bincount(dist[reached]) if reached.any() else np.zeros(1, dtype=np.int64)
    assert hist.sum() == in_comp.sum()
    assert np.all(hist > 0), "a level between 0 and the eccentricity is empty"
    return int(reached.sum())
