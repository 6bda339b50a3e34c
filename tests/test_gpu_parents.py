"""GPU parent arrays (BFS trees) from finished distances.

Parents are not unique, so every result is checked by the tree invariants
(the source is its own parent; a reached vertex's parent is one of its
neighbours, one level closer; unreached vertices get -1), and on graphs whose
lists keep the caller's order also against the library's fixed rule (the first
such neighbour in list order) applied to the oracle's distances.
"""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle
from tests import graphs as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bfs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_00430_gb300 as B
    B.load()
    return B


def first_rule(rp, col, d):
    n = len(rp) - 1
    par = np.full(n, -1, dtype=np.int32)
    for v in range(n):
        if d[v] == 0:
            par[v] = v
        elif d[v] > 0:
            nb = col[rp[v]:rp[v + 1]]
            hit = np.nonzero(d[nb] == d[v] - 1)[0]
            par[v] = nb[hit[0]] if len(hit) else -1
    return par


def tree_ok(rp, col, d, par):
    n = len(rp) - 1
    for v in range(n):
        if d[v] < 0:
            if par[v] != -1:
                return False
        elif d[v] == 0:
            if par[v] != v:
                return False
        else:
            p = par[v]
            if p < 0 or d[p] != d[v] - 1 or p not in col[rp[v]:rp[v + 1]]:
                return False
    return True


def run(B, g, n, src, **kw):
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    B.bfs_single_ex(g, int(src), d, params=B.make_params(**kw) if kw else None)
    par = torch.full((n,), 77, dtype=torch.int32, device="cuda")
    B.bfs_parents(g, d, par)
    return d.cpu().numpy(), par.cpu().numpy()


@pytest.mark.parametrize("bits", [32, 64])
def test_first_rule_and_invariants(bfs, bits):
    # A vertex (1) whose parent (200) is entry 100 of its list: the warp-cooperative scan.
    # A star searched from a far leaf: the centre's parent is entry ~2500 of a 2999-entry list, past the
    # warp-scanned part: the chunked scan of long lists.
    edges = [(0, 200), (200, 1)] + [(1, 2 + i) for i in range(100)] + [(300, 301)]
    cases = [(graphgen.rmat(14, seed=51), []), (graphgen.grid2d(20, 30), []), (G.csr_from_edges(310, edges), []),
             (G.star_graph(600), []), (G.star_graph(3000), [2500, 40])]
    for (rp, col), extra in cases:
        g = bfs.bfs_graph_upload(rp.astype(np.int32 if bits == 32 else np.int64), col)
        n = len(rp) - 1
        for src in list(graphgen.sources(rp, 2, 5100)) + [0] + extra:
            want = oracle.bfs(rp, col, int(src))
            d, par = run(bfs, g, n, src)
            assert np.array_equal(d, want)
            assert np.array_equal(par, first_rule(rp, col, want)), int(src)
            assert tree_ok(rp, col, want, par)
        g.free()


def test_degree_ordered_and_renumbered_queries(bfs):
    """Lists stored highest degree first and queries on the renumbered copy: parents are valid trees of
    the caller's ids."""
    rp, col = graphgen.rmat(13, seed=52)
    g = bfs.bfs_graph_upload(rp, col, flags=bfs.BFS_DEGREE_ORDER)
    n = len(rp) - 1
    for src in graphgen.sources(rp, 3, 5200):
        want = oracle.bfs(rp, col, int(src))
        for kw in ({}, {"relabel": 1}):
            d, par = run(bfs, g, n, src, **kw)
            assert np.array_equal(d, want) and tree_ok(rp, col, want, par), (int(src), kw)
    g.free()


def test_invalid(bfs):
    rp, col = G.path_graph(4)
    g = bfs.bfs_graph_upload(rp, col)
    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_parents(g, d, np.zeros(4, dtype=np.int32))
    assert e.value.code == bfs.BFS_EINVAL
    g.free()


def test_calls_on_two_streams_share_the_workspace_safely(bfs):
    """Parent arrays of one graph requested on two streams back to back: the calls share the
    graph's workspace for long lists (more than 1056 entries: chunk records), and the library orders
    them on the device, so both results follow the rule exactly."""
    # Two hubs whose lists are longer than 1056 entries, joined by a path; leaves hang off both.
    n = 6000
    edges = [(0, i) for i in range(2, 3000)] + [(1, i) for i in range(2500, 6000)] + [(0, 5999)]
    rp, col = G.csr_from_edges(n, edges)
    assert np.diff(rp).max() > 1056
    g = bfs.bfs_graph_upload(rp, col)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    srcs = (2, 4000)
    dists = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in srcs]
    for d, s_ in zip(dists, srcs):
        bfs.bfs_single(g, s_, d)
    torch.cuda.synchronize()
    for rep in range(3):
        pars = [torch.full((n,), 77, dtype=torch.int32, device="cuda") for _ in srcs]
        torch.cuda.synchronize()
        bfs.bfs_parents(g, dists[0], pars[0], stream=s1)
        bfs.bfs_parents(g, dists[1], pars[1], stream=s2)
        torch.cuda.synchronize()
        for d, p in zip(dists, pars):
            dd = d.cpu().numpy()
            assert np.array_equal(p.cpu().numpy(), first_rule(rp, col, dd)), rep
    g.free()
