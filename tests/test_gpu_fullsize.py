"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

The oracle runs per sampled source (several in parallel threads); outputs it
cannot afford one by one are checked through properties that hold at any size
(source at 0, unreached exactly -1 / 255, BFS invariants on every edge).
"""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bfs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_00430_gb300 as B
    B.load()
    return B


def edge_invariant(rp, col, d):
    """|d(u) - d(v)| <= 1 on every arc, no arc between reached and unreached (vectorised)."""
    n = len(rp) - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    du, dv = d[src], d[col]
    both = (du >= 0) & (dv >= 0)
    return bool(np.all(np.abs(du[both] - dv[both]) <= 1) and np.all((du >= 0) == (dv >= 0)))


def test_rmat_s25_bench_configuration(bfs):
    """R-MAT scale 25, int64 row pointers, degree-ordered, default (persistent) launch: 3 of the 64
    bench sources against the oracle, all 64 checked by invariants."""
    rp, col = graphgen.rmat(25, 16, 0.57, 0.19, 0.19, 1, 1)
    srcs = graphgen.sources(rp, 64, 1002)
    g = bfs.bfs_graph_upload(rp, col, flags=bfs.BFS_VALIDATE | bfs.BFS_DEGREE_ORDER)
    n = len(rp) - 1
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    want = oracle.bfs_many(rp, col, [int(s) for s in srcs[:3]], threads=3)
    for i in range(3):
        bfs.bfs_single(g, int(srcs[i]), d)
        assert np.array_equal(d.cpu().numpy(), want[i]), i
    reached = int((want[0] >= 0).sum())
    for s in srcs[3::30]:
        bfs.bfs_single(g, int(s), d)
        x = d.cpu().numpy()
        assert x[int(s)] == 0 and int((x >= 0).sum()) == reached  # one giant component
        assert edge_invariant(rp, col, x)
    g.free()


def test_er_2e24_and_large_diameter(bfs):
    for make, bits in ((lambda: graphgen.erdos_renyi(1 << 24, 16.0, 2), 32), (lambda: graphgen.grid2d(4096, 4096), 32),
                       (lambda: graphgen.rgg(1 << 23, graphgen.rgg_radius(1 << 23, 3.0), 3), 32)):
        rp, col = make()
        g = bfs.bfs_graph_upload(rp.astype(np.int32), col, flags=bfs.BFS_VALIDATE)
        srcs = [int(s) for s in graphgen.sources(rp, 2, 1003)]
        want = oracle.bfs_many(rp, col, srcs, threads=2)
        d = torch.empty(len(rp) - 1, dtype=torch.int32, device="cuda")
        for i, s in enumerate(srcs):
            for launch in (0, 2):
                bfs.bfs_single_ex(g, s, d, params=bfs.make_params(launch=launch))
                assert np.array_equal(d.cpu().numpy(), want[i]), (i, launch)
        g.free()


def test_msbfs_rmat_s24_256_sources(bfs):
    rp, col = graphgen.rmat(24, 16, 0.57, 0.19, 0.19, 1, 1)
    n = len(rp) - 1
    srcs = graphgen.sources(rp, 256, 1004)
    g = bfs.bfs_graph_upload(rp, col, flags=bfs.BFS_VALIDATE | bfs.BFS_DEGREE_ORDER)
    out = torch.empty((256, n), dtype=torch.uint8, device="cuda")
    bfs.bfs_multi(g, srcs, out, dist_bits=8)
    rows = [0, 97, 255]
    want = oracle.to_uint8(oracle.bfs_many(rp, col, [int(srcs[i]) for i in rows], threads=3))
    for k, i in enumerate(rows):
        assert np.array_equal(out[i].cpu().numpy(), want[k]), i
    diag = out[torch.arange(256, device="cuda"), torch.from_numpy(srcs.astype(np.int64)).cuda()]
    assert int(diag.max()) == 0  # every row has its own source at distance 0
    del out
    out32 = torch.empty((256, n), dtype=torch.int32, device="cuda")
    bfs.bfs_multi(g, srcs, out32, dist_bits=32)
    x = out32[97].cpu().numpy()
    assert np.array_equal(np.where(x < 0, 255, x).astype(np.uint8), want[1])
    g.free()


def test_graphset_10000(bfs):
    gs = graphgen.graph_set(10000, 1000, 100000, 8.0, seed=4)
    s = bfs.bfs_graphset_upload(gs.voff, gs.eoff, gs.row_ptr, gs.col)
    dist = torch.empty(int(gs.voff[-1]), dtype=torch.int32, device="cuda")
    bfs.bfs_graphset_run(s, gs.src, dist)
    got = dist.cpu().numpy()
    for i in list(range(0, 10000, 97)) + [int(np.argmax(np.diff(gs.voff)))]:
        rp, col = gs.graph(i)
        assert np.array_equal(got[gs.voff[i]:gs.voff[i + 1]], oracle.bfs(rp, col, int(gs.src[i]))), i
    s.free()
