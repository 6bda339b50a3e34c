"""GPU parity of multi-source BFS (bfs_multi) against the oracle, row by row (bit-exact)."""
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


def run_multi(B, g, n, srcs, bits, **kw):
    dt = torch.uint8 if bits == 8 else torch.int32
    out = torch.full((len(srcs), n), 77, dtype=dt, device="cuda")
    st = B.bfs_multi_ex(g, srcs, out, dist_bits=bits, params=B.make_params(**kw) if kw else None)
    return out.cpu().numpy(), st


def expect(rp, col, srcs, bits):
    want = oracle.bfs_many(rp, col, srcs)
    return oracle.to_uint8(want) if bits == 8 else want


@pytest.mark.parametrize("bits", [8, 32])
@pytest.mark.parametrize("k", [1, 5, 64, 100, 256, 300])
def test_rmat_group_sizes(bfs, bits, k):
    rp, col = graphgen.rmat(13, seed=21)
    g = bfs.bfs_graph_upload(rp, col)
    srcs = graphgen.sources(rp, k, 2000 + k)
    got, st = run_multi(bfs, g, len(rp) - 1, srcs, bits)
    assert np.array_equal(got, expect(rp, col, srcs, bits))
    assert st["groups"] == (k + 255) // 256
    g.free()


@pytest.mark.parametrize("kw", [dict(ms_lanes=64), dict(ms_lanes=7, ms_ring=2), dict(ms_heavy_min=0),
                                dict(ms_heavy_min=1 << 30), dict(alpha=1, beta=1), dict(alpha=1000, beta=1000),
                                dict(ms_ring=3, ms_lanes=130), dict(ms_degree_order=1),
                                dict(ms_degree_order=1, ms_heavy_min=0, ms_lanes=64), dict(ms_relabel=0),
                                dict(ms_relabel=0, ms_degree_order=0, ms_lanes=64, ms_ring=2), dict(ms_ring=16)])
def test_parameters(bfs, kw):
    rp, col = graphgen.rmat(12, seed=22)
    g = bfs.bfs_graph_upload(rp, col, flags=bfs.BFS_DEGREE_ORDER)
    srcs = graphgen.sources(rp, 150, 2100)
    got, _ = run_multi(bfs, g, len(rp) - 1, srcs, 32, **kw)
    assert np.array_equal(got, expect(rp, col, srcs, 32))
    g.free()


def test_duplicate_sources_and_disconnected(bfs):
    edges = [(i, i + 1) for i in range(9)] + [(20 + i, 21 + i) for i in range(5)]
    rp, col = G.csr_from_edges(40, edges)
    g = bfs.bfs_graph_upload(rp, col)
    srcs = np.array([0, 0, 5, 20, 39, 5, 25, 9], dtype=np.int32)
    for bits in (8, 32):
        got, _ = run_multi(bfs, g, 40, srcs, bits)
        assert np.array_equal(got, expect(rp, col, srcs, bits))
    g.free()


def test_large_diameter_many_flushes(bfs):
    rp, col = graphgen.grid2d(70, 90)  # eccentricity up to 158: many ring windows
    g = bfs.bfs_graph_upload(rp, col)
    srcs = graphgen.sources(rp, 70, 2200)
    for ring, relabel in ((2, 1), (8, 1), (16, 1), (5, 0)):
        got, st = run_multi(bfs, g, len(rp) - 1, srcs, 8, ms_ring=ring, ms_relabel=relabel)
        assert np.array_equal(got, expect(rp, col, srcs, 8))
    g.free()


@pytest.mark.parametrize("rp_bits", [32, 64])
@pytest.mark.parametrize("degree_order", [False, True])
def test_renumbered_layout(bfs, rp_bits, degree_order):
    """The degree-renumbered copy (lists sorted after renumbering, or already in degree order) against the
    graph as uploaded and the oracle, with isolated vertices among the sources."""
    rp, col = graphgen.rmat(11, seed=24)
    rp64 = rp.astype(np.int64)
    iso = np.flatnonzero(np.diff(rp64) == 0)
    assert len(iso) >= 4
    srcs = np.concatenate([graphgen.sources(rp64, 60, 2400), iso[:3], iso[-1:]]).astype(np.int32)
    g = bfs.bfs_graph_upload(rp.astype(np.int32 if rp_bits == 32 else np.int64), col,
                             flags=bfs.BFS_DEGREE_ORDER if degree_order else 0)
    for bits in (8, 32):
        want = expect(rp64, col, srcs, bits)
        for relabel in (1, 0):
            got, _ = run_multi(bfs, g, len(rp) - 1, srcs, bits, ms_relabel=relabel)
            assert np.array_equal(got, want), (bits, relabel)
    g.free()


def test_uint8_range_error(bfs):
    rp, col = G.path_graph(300)
    g = bfs.bfs_graph_upload(rp, col)
    out = torch.empty((2, 300), dtype=torch.uint8, device="cuda")
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_multi(g, np.array([0, 1], dtype=np.int32), out, dist_bits=8)
    assert e.value.code == bfs.BFS_ERANGE
    out32 = torch.empty((2, 300), dtype=torch.int32, device="cuda")
    bfs.bfs_multi(g, np.array([0, 299], dtype=np.int32), out32, dist_bits=32)
    assert np.array_equal(out32.cpu().numpy(), oracle.bfs_many(rp, col, [0, 299]))
    g.free()


def test_host_output_and_single_agreement(bfs):
    rp, col = graphgen.erdos_renyi(5000, 8, 23)
    g = bfs.bfs_graph_upload(rp, col)
    srcs = graphgen.sources(rp, 40, 2300)
    host = np.zeros((40, 5000), dtype=np.int32)
    bfs.bfs_multi(g, srcs, host, dist_bits=32)
    assert np.array_equal(host, oracle.bfs_many(rp, col, srcs))
    d = torch.empty(5000, dtype=torch.int32, device="cuda")
    for i in (0, 17, 39):
        bfs.bfs_single(g, int(srcs[i]), d)
        assert np.array_equal(d.cpu().numpy(), host[i])
    g.free()


def test_invalid(bfs):
    rp, col = G.path_graph(5)
    g = bfs.bfs_graph_upload(rp, col)
    out = torch.empty((1, 5), dtype=torch.int32, device="cuda")
    for srcs, bits in (([5], 32), ([0], 16), ([-1], 8)):
        with pytest.raises(bfs.BfsError) as e:
            bfs.bfs_multi(g, np.array(srcs, dtype=np.int32), out, dist_bits=bits)
        assert e.value.code == bfs.BFS_EINVAL
    g.free()


def test_counters_against_the_oracle_rows(bfs):
    """The call's counters against facts of its exact output (one group of 256 sources): every
    vertex that a lane reaches (other than at its own source) gains that lane at some level, so
    `found` lies between the most vertices one lane reaches and the sum over lanes; a pull level
    reads at most every vertex of degree > 0, a push level's frontier at most every vertex; the
    output is written once per row."""
    rp, col = graphgen.rmat(13, seed=22)
    n = len(rp) - 1
    g = bfs.bfs_graph_upload(rp, col)
    srcs = graphgen.sources(rp, 256, 2300)
    got, st = run_multi(bfs, g, n, srcs, 32)
    want = oracle.bfs_many(rp, col, srcs)
    assert np.array_equal(got, want)
    reached = (want >= 0).sum(axis=1)
    live = int((np.diff(rp) > 0).sum())
    assert reached.max() - 1 <= st["found"] <= int(reached.sum())
    assert st["pull_active"] <= st["pull_levels"] * live and (st["pull_levels"] == 0 or st["pull_active"] > 0)
    assert st["push_frontier"] <= st["push_levels"] * n and st["push_frontier"] >= (st["push_levels"] > 0)
    assert st["output_bytes"] >= 4 * 256 * n
    assert st["push_levels"] + st["pull_levels"] >= int(want.max()) + 1
    g.free()
