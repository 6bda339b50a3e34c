"""GPU parity of the graph-set launch against the oracle (bit-exact, every graph)."""
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


def concat(graphs):
    voff, eoff, rps, cols = [0], [0], [], []
    for rp, col in graphs:
        voff.append(voff[-1] + len(rp) - 1)
        eoff.append(eoff[-1] + len(col))
        rps.append(np.asarray(rp, dtype=np.int64))
        cols.append(np.asarray(col, dtype=np.int32))
    return (np.array(voff), np.array(eoff), np.concatenate(rps), np.concatenate(cols) if cols else np.zeros(0, np.int32))


def check_set(B, gs_voff, gs_eoff, gs_rp, gs_col, srcs, graphs, **kw):
    s = B.bfs_graphset_upload(gs_voff, gs_eoff, gs_rp, gs_col, flags=B.BFS_VALIDATE)
    dist = torch.full((int(gs_voff[-1]),), 99, dtype=torch.int32, device="cuda")
    st = B.bfs_graphset_run(s, srcs, dist, params=B.make_params(**kw) if kw else None)
    got = dist.cpu().numpy()
    for i, (rp, col) in enumerate(graphs):
        want = oracle.bfs(rp, col, int(srcs[i]))
        assert np.array_equal(got[gs_voff[i]:gs_voff[i + 1]], want), i
    s.free()
    return st


def test_generated_set(bfs):
    gs = graphgen.graph_set(300, 1000, 20000, 8.0, seed=4)
    graphs = [gs.graph(i) for i in range(gs.count)]
    st = check_set(bfs, gs.voff, gs.eoff, gs.row_ptr, gs.col, gs.src, graphs)
    assert st["graphs"] == 300 and st["levels"] >= 300


@pytest.mark.parametrize("kw", [dict(threads_per_block=64), dict(threads_per_block=512, blocks_per_sm=1),
                                dict(alpha=1, beta=1), dict(alpha=100000, beta=1)])
def test_parameters(bfs, kw):
    gs = graphgen.graph_set(60, 1000, 8000, 6.0, seed=9)
    graphs = [gs.graph(i) for i in range(gs.count)]
    check_set(bfs, gs.voff, gs.eoff, gs.row_ptr, gs.col, gs.src, graphs, **kw)


def test_mixed_shapes(bfs):
    graphs = [G.path_graph(1), G.path_graph(300), G.star_graph(70), G.complete_graph(40), G.cycle_graph(1001),
              graphgen.grid2d(40, 33), graphgen.rmat(12, seed=5), G.csr_from_edges(64, [(0, 1), (5, 6)]),
              G.star_graph(5000), graphgen.rmat(14, seed=2)]  # long lists: many 32-entry steps per frontier word
    srcs = np.array([0, 150, 3, 7, 500, 600, int(graphgen.sources(graphs[6][0], 1, 3)[0]), 5, 17,
                     int(graphgen.sources(graphs[9][0], 1, 4)[0])], dtype=np.int32)
    check_set(bfs, *concat(graphs), srcs, graphs)


def test_host_output_and_invalid(bfs):
    graphs = [G.path_graph(10), G.cycle_graph(12)]
    voff, eoff, rp, col = concat(graphs)
    s = bfs.bfs_graphset_upload(voff, eoff, rp, col)
    host = np.zeros(22, dtype=np.int32)
    bfs.bfs_graphset_run(s, np.array([0, 3], dtype=np.int32), host)
    assert np.array_equal(host[:10], oracle.bfs(*graphs[0], 0))
    assert np.array_equal(host[10:], oracle.bfs(*graphs[1], 3))
    with pytest.raises(bfs.BfsError):
        bfs.bfs_graphset_run(s, np.array([0, 12], dtype=np.int32), host)
    s.free()
    bad = col.copy()
    bad[0] = 50
    with pytest.raises(bfs.BfsError):
        bfs.bfs_graphset_upload(voff, eoff, rp, bad, flags=bfs.BFS_VALIDATE)
