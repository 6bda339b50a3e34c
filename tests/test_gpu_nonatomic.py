"""GPU parity of the non-atomic top-down variant (the paper's BFS-NonAtomic, Section 2).

Distances must equal the oracle's bit for bit (every writer of a level stores
the same value).  The per-level distinct-vertex counts the library reports
must equal the oracle's level histogram, every level's appended entries must be
at least its distinct vertices (duplicates only add), and the list entries read
must equal the degree sum of the level's vertices (duplicates are removed
before a level is expanded).
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


def check(B, rp, col, srcs, bits=64):
    g = B.bfs_graph_upload(rp.astype(np.int32 if bits == 32 else np.int64), col)
    n = len(rp) - 1
    deg = np.diff(rp.astype(np.int64))
    for src in srcs:
        want = oracle.bfs(rp, col, int(src))
        d = torch.full((n,), 77, dtype=torch.int32, device="cuda")
        st, lv = B.bfs_single_nonatomic(g, int(src), d, level_cap=1 << 14)
        got = d.cpu().numpy()
        assert np.array_equal(got, want), (int(src), np.nonzero(got != want)[0][:10])
        hist = np.bincount(want[want >= 0])
        assert [x["unique"] for x in lv] == hist.tolist(), int(src)
        assert st["levels"] == len(hist) and st["unique"] == int((want >= 0).sum())
        for L, x in enumerate(lv):
            assert x["frontier"] >= x["unique"]
            assert x["edges"] == int(deg[want == L].sum()), (int(src), L)
        assert st["frontier_entries"] == sum(x["frontier"] for x in lv)
        assert st["edges"] == sum(x["edges"] for x in lv)
        # Counts off: the same distances.
        d2 = torch.full((n,), 77, dtype=torch.int32, device="cuda")
        none, lv2 = B.bfs_single_nonatomic(g, int(src), d2, stats=False)
        assert none is None and lv2 == [] and torch.equal(d2, d)
    g.free()


@pytest.mark.parametrize("bits", [32, 64])
def test_generated_graphs(bfs, bits):
    for rp, col in (graphgen.rmat(14, seed=41), graphgen.erdos_renyi(6000, 12.0, 42), graphgen.grid2d(30, 50)):
        check(bfs, rp, col, graphgen.sources(rp, 3, 4100), bits)


def test_closed_forms_hubs_and_isolated(bfs):
    edges = [(i, i + 1) for i in range(4)] + [(5 + i, 5 + (i + 1) % 6) for i in range(6)]
    cases = [(G.path_graph(300), [0, 150]), (G.star_graph(2000), [0, 7]),  # the centre's list spans chunks
             (G.complete_graph(300), [3]), (G.csr_from_edges(40, edges), [2, 5, 11, 39])]
    for (rp, col), srcs in cases:
        check(bfs, rp, col, srcs)


def test_invalid(bfs):
    rp, col = G.path_graph(5)
    g = bfs.bfs_graph_upload(rp, col)
    d = torch.empty(5, dtype=torch.int32, device="cuda")
    for src in (-1, 5):
        with pytest.raises(bfs.BfsError) as e:
            bfs.bfs_single_nonatomic(g, src, d)
        assert e.value.code == bfs.BFS_EINVAL
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_single_nonatomic(g, 0, np.zeros(5, dtype=np.int32))  # host memory is not accepted
    assert e.value.code == bfs.BFS_EINVAL
    g.free()


def check_expand(B, rp, col, srcs, must_fit):
    """BFS_DUP_EXPAND (the paper's variant: every appended entry is expanded again).  When the
    copies fit the queues: exact distances, per-level distinct counts equal to the oracle's level
    histogram, the entries expanded at level L+1 equal to those appended at level L, and at least
    the level's degree sum read.  When they do not: BFS_ENOMEM (reported, nothing written out of
    bounds), and the graph stays usable."""
    g = B.bfs_graph_upload(rp, col)
    n = len(rp) - 1
    deg = np.diff(rp.astype(np.int64))
    outcomes = []
    for src in srcs:
        want = oracle.bfs(rp, col, int(src))
        d = torch.full((n,), 77, dtype=torch.int32, device="cuda")
        try:
            st, lv = B.bfs_single_nonatomic(g, int(src), d, level_cap=1 << 14, expand_duplicates=True)
        except B.BfsError as e:
            assert e.code == B.BFS_ENOMEM and not must_fit, int(src)
            outcomes.append("overflow")
            continue
        outcomes.append("fit")
        assert np.array_equal(d.cpu().numpy(), want), int(src)
        hist = np.bincount(want[want >= 0])
        assert [x["unique"] for x in lv] == hist.tolist(), int(src)
        assert lv[0]["frontier"] == 1
        for L, x in enumerate(lv):
            assert x["frontier"] >= x["unique"] and x["edges"] >= int(deg[want == L].sum()), (int(src), L)
        assert st["frontier_entries"] == sum(x["frontier"] for x in lv)
        # the default mode on the same graph afterwards: exact
        B.bfs_single_nonatomic(g, int(src), d)
        assert np.array_equal(d.cpu().numpy(), want)
    g.free()
    return outcomes


def test_expand_duplicates_mode(bfs):
    assert check_expand(bfs, *G.path_graph(300), [0, 150], must_fit=True) == ["fit", "fit"]
    assert check_expand(bfs, *G.star_graph(2000), [0, 7], must_fit=True) == ["fit", "fit"]
    for rp, col in (graphgen.rmat(10, seed=41), graphgen.grid2d(30, 50), graphgen.erdos_renyi(3000, 8.0, 43)):
        check_expand(bfs, rp, col, graphgen.sources(rp, 3, 4100), must_fit=False)


def test_expand_mode_invalid(bfs):
    rp, col = G.path_graph(5)
    g = bfs.bfs_graph_upload(rp, col)
    d = torch.empty(5, dtype=torch.int32, device="cuda")
    rc = bfs.load().bfs_single_nonatomic_ex(g.handle, 0, d.data_ptr(), 7, None, None, 0, None)
    assert rc == bfs.BFS_EINVAL
    g.free()
