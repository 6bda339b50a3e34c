"""Host replay of a direction policy on known BFS levels (test infrastructure).

Given the graph and the distances (from the oracle), the frontier of every
level is fixed: F_L = {v : dist[v] == L}.  The policy's direction sequence and
the work counters that the library reports (vertices and edges of top-down
levels, unvisited vertices and entries examined up to the first frontier
neighbour in bottom-up levels, conversions) are therefore deterministic and
computed here independently of the GPU code, with numpy.
"""
from __future__ import annotations

import numpy as np

POLICY_FRONTIER, POLICY_EDGES, POLICY_TD_ONLY, POLICY_BU_FROM_1, POLICY_SCRIPT, POLICY_LOCAL = 1, 2, 3, 4, 5, 6
LOCAL_AUTO_MAX_DEGREE = 4096


def resolve(policy, n, m, large_diameter_degree=7, max_degree=0):
    """The policy BFS_POLICY_AUTO stands for: Section 3's large-diameter class (average degree
    below 7) runs top-down only, as the multi-level local kernel unless a list is longer than
    4096 entries; other graphs use the edge-count rule."""
    if policy != 0:
        return policy
    if m < large_diameter_degree * n:
        return POLICY_LOCAL if max_degree <= LOCAL_AUTO_MAX_DEGREE else POLICY_TD_ONLY
    return POLICY_EDGES


def next_top_down(policy, nl, cur_td, nf_next, nf_cur, mf_next, m_unv, n, alpha=14, beta=24, tau_inv=20, script=0):
    if nl == 0:
        return True
    if policy == POLICY_TD_ONLY:
        return True
    if policy == POLICY_BU_FROM_1:
        return False
    if policy == POLICY_SCRIPT:
        return ((script >> min(nl, 63)) & 1) == 0
    if policy == POLICY_FRONTIER:
        return tau_inv * nf_next < n
    if cur_td:
        return not (alpha * mf_next > m_unv)
    return beta * nf_next < n and nf_next < nf_cur


def first_hit_counts(row_ptr, col, rows, in_front):
    """Entries examined by a CSR-order scan of each row in ``rows`` that stops
    at the first neighbour with in_front[nbr] (all entries when none)."""
    deg = (row_ptr[rows + 1] - row_ptr[rows]).astype(np.int64)
    if len(rows) == 0:
        return np.zeros(0, dtype=np.int64)
    idx = np.concatenate([np.arange(row_ptr[r], row_ptr[r + 1]) for r in rows]) if len(rows) < 2000 else \
        _ranges(row_ptr[rows], row_ptr[rows + 1])
    owner = np.repeat(np.arange(len(rows)), deg)
    pos = idx - np.repeat(row_ptr[rows], deg)
    hit = in_front[col[idx]]
    first = deg.copy()
    hp = pos[hit]
    ho = owner[hit]
    # minimum position per owner among hits
    mins = np.full(len(rows), np.iinfo(np.int64).max)
    np.minimum.at(mins, ho, hp)
    got = mins != np.iinfo(np.int64).max
    first[got] = mins[got] + 1
    return first


def _ranges(starts, ends):
    lens = (ends - starts).astype(np.int64)
    tot = int(lens.sum())
    if tot == 0:
        return np.zeros(0, dtype=np.int64)
    offs = np.repeat(starts - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
    return np.arange(tot, dtype=np.int64) + offs


def degree_ordered(row_ptr, col):
    """Each row reordered highest-degree neighbour first, ties by id (the layout of BFS_DEGREE_ORDER)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    deg = np.diff(row_ptr)
    owner = np.repeat(np.arange(len(row_ptr) - 1), deg)
    return col[np.lexsort((col, -deg[col], owner))]


def replay(row_ptr, col, src, dist, policy=0, alpha=14, beta=24, tau_inv=20, script=0, large_diameter_degree=7,
           degree_order=False):
    """Expected bfs_stats totals and per-level records for ``dist``."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    if degree_order:
        col = degree_ordered(row_ptr, col)
    n = len(row_ptr) - 1
    m = int(row_ptr[-1])
    deg = np.diff(row_ptr)
    pol = resolve(policy, n, m, large_diameter_degree, int(deg.max()) if n else 0)
    if pol == POLICY_LOCAL:  # per-level launches of AUTO run the level-synchronous top-down path
        pol = POLICY_TD_ONLY
    ecc = int(dist.max())
    sizes = np.bincount(dist[dist >= 0], minlength=ecc + 2)
    degsum = np.bincount(dist[dist >= 0], weights=deg[dist >= 0], minlength=ecc + 2).astype(np.int64)
    st = dict(levels=0, td_levels=0, bu_levels=0, conversions=0, reached=int((dist >= 0).sum()),
              edges_reached=int(deg[dist >= 0].sum()), td_frontier=0, td_edges=0, bu_unvisited=0, bu_edges=0,
              bu_found=0, conv_frontier=0)
    levels = []
    td = True
    edges_visited = int(deg[src])
    converted = 0
    for L in range(ecc + 1):
        nf = int(sizes[L])
        rec = dict(direction=0 if td else 1, converted=converted, frontier=nf, edges=0, unvisited=0,
                   found=int(sizes[L + 1]))
        if td:
            st["td_levels"] += 1
            st["td_frontier"] += nf
            st["td_edges"] += int(degsum[L])
            rec["edges"] = int(degsum[L])
        else:
            st["bu_levels"] += 1
            unv = np.nonzero(((dist < 0) | (dist > L)) & (deg > 0))[0]
            ex = first_hit_counts(row_ptr, col, unv, dist == L)
            st["bu_unvisited"] += len(unv)
            st["bu_edges"] += int(ex.sum())
            st["bu_found"] += int(sizes[L + 1])
            rec["edges"] = int(ex.sum())
            rec["unvisited"] = len(unv)
        levels.append(rec)
        st["levels"] = L + 1
        nf_next = int(sizes[L + 1])
        if nf_next == 0:
            break
        mf_next = int(degsum[L + 1])
        edges_visited += mf_next
        ntd = next_top_down(pol, L + 1, td, nf_next, nf, mf_next, m - edges_visited, n, alpha, beta, tau_inv, script)
        converted = 1 if ntd != td else 0
        if converted:
            st["conversions"] += 1
            st["conv_frontier"] += nf_next
        td = ntd
    return st, levels
