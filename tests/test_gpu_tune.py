"""Autotuner: returns valid parameters that reproduce the oracle's distances."""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bfs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_00430_gb300 as B
    B.load()
    return B


@pytest.mark.parametrize("make", [lambda: graphgen.rmat(14, seed=41), lambda: graphgen.grid2d(100, 100)])
def test_tune_returns_working_params(bfs, make, tmp_path):
    rp, col = make()
    g = bfs.bfs_graph_upload(rp, col, flags=bfs.BFS_DEGREE_ORDER)
    srcs = graphgen.sources(rp, 3, 4100)
    params, rep = bfs.bfs_tune(g, srcs)
    assert rep["trials"] > 5 and rep["best_ms"] <= rep["start_ms"] * 1.05
    d = torch.empty(len(rp) - 1, dtype=torch.int32, device="cuda")
    for s in graphgen.sources(rp, 3, 4200):
        bfs.bfs_single_ex(g, int(s), d, params=params)
        assert np.array_equal(d.cpu().numpy(), oracle.bfs(rp, col, int(s)))
    path = str(tmp_path / "tune.json")
    entry = bfs.tune_table_update(path, g, srcs)
    p2 = bfs.tuned_params(path, g)
    assert all(getattr(p2, k) == v for k, v in entry["params"].items())
    g.free()


def test_tune_multi_returns_working_params(bfs):
    rp, col = graphgen.rmat(13, seed=42)
    g = bfs.bfs_graph_upload(rp, col, flags=bfs.BFS_DEGREE_ORDER)
    srcs = graphgen.sources(rp, 100, 4300)
    params, rep = bfs.bfs_tune_multi(g, srcs, dist_bits=8)
    assert rep["trials"] > 5 and rep["sources"] == 100 and rep["best_ms"] <= rep["start_ms"] * 1.05
    out = torch.empty((100, len(rp) - 1), dtype=torch.uint8, device="cuda")
    bfs.bfs_multi_ex(g, srcs, out, dist_bits=8, params=params)
    want = oracle.to_uint8(oracle.bfs_many(rp, col, srcs))
    assert np.array_equal(out.cpu().numpy(), want)
    g.free()


def test_tune_graphset_returns_working_params(bfs):
    gs = graphgen.graph_set(300, 100, 5000, 8.0, seed=9)
    s = bfs.bfs_graphset_upload(gs.voff, gs.eoff, gs.row_ptr, gs.col)
    params, rep = bfs.bfs_tune_graphset(s, gs.src)
    assert rep["trials"] > 5 and rep["sources"] == 300
    dist = torch.empty(int(gs.voff[-1]), dtype=torch.int32, device="cuda")
    bfs.bfs_graphset_run(s, gs.src, dist, params=params)
    got = dist.cpu().numpy()
    for i in range(gs.count):
        rp, col = gs.graph(i)
        assert np.array_equal(got[gs.voff[i]:gs.voff[i + 1]], oracle.bfs(rp, col, int(gs.src[i]))), i
    s.free()


def test_committed_table_entries_reproduce_the_oracle(bfs):
    """Every entry of the committed tuning table is a valid parameter set: applied to small graphs
    of both degree classes it reproduces the oracle exactly (single-source, multi-source and
    graph-set entries through their own entry points)."""
    import json
    with open(bfs.TUNED_TABLE) as f:
        table = json.load(f)
    assert table, "the tuning table is empty"
    graphs = [graphgen.rmat(12, seed=43), graphgen.grid2d(60, 40)]
    for key, entry in table.items():
        p = bfs.bfs_params_default()
        for k, v in entry["params"].items():
            setattr(p, k, v)
        if key == "graphset":
            gs = graphgen.graph_set(50, 100, 3000, 8.0, seed=10)
            s = bfs.bfs_graphset_upload(gs.voff, gs.eoff, gs.row_ptr, gs.col)
            dist = torch.empty(int(gs.voff[-1]), dtype=torch.int32, device="cuda")
            bfs.bfs_graphset_run(s, gs.src, dist, params=p)
            got = dist.cpu().numpy()
            for i in range(gs.count):
                rp, col = gs.graph(i)
                assert np.array_equal(got[gs.voff[i]:gs.voff[i + 1]], oracle.bfs(rp, col, int(gs.src[i]))), (key, i)
            s.free()
            continue
        for rp, col in graphs:
            g = bfs.bfs_graph_upload(rp, col, flags=bfs.BFS_DEGREE_ORDER)
            srcs = graphgen.sources(rp, 3, 4400)
            want = oracle.bfs_many(rp, col, srcs)
            if key.startswith("single/"):
                d = torch.empty(len(rp) - 1, dtype=torch.int32, device="cuda")
                for i, s_ in enumerate(srcs):
                    bfs.bfs_single_ex(g, int(s_), d, params=p)
                    assert np.array_equal(d.cpu().numpy(), want[i]), (key, int(s_))
            else:
                out = torch.empty((3, len(rp) - 1), dtype=torch.int32, device="cuda")
                bfs.bfs_multi_ex(g, srcs, out, dist_bits=32, params=p)
                assert np.array_equal(out.cpu().numpy(), want), key
            g.free()
