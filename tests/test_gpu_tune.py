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
