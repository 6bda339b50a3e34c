"""GPU parity of the multi-level local expansion (BFS_POLICY_LOCAL) against the oracle.

The policy relaxes distances with atomicMin while blocks advance several levels
on their own share of the frontier, and stops at the fixpoint; the distances it
returns must still equal the oracle's bit for bit, for any number of local
levels per super-step (1 = level-synchronous), with or without the head
table, on small closed forms, on hub-heavy graphs whose local queues overflow
into the global queue, and on disconnected graphs.  Its counters are checked
against facts of the oracle's result (reached vertices, their degree sum,
eccentricity) and against bounds the method implies.
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


def check(B, rp, col, srcs, ks=(1, 2, 16, 64), rp_bits=64, head=True, extra=None):
    flags = B.BFS_VALIDATE | (0 if head else B.BFS_NO_HEAD)
    g = B.bfs_graph_upload(rp, col, flags=flags, row_ptr_bits=rp_bits)
    n = len(rp) - 1
    deg = np.diff(np.asarray(rp, dtype=np.int64))
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    for src in srcs:
        want = oracle.bfs(rp, col, int(src))
        for k in ks:
            p = B.make_params(policy=B.BFS_POLICY_LOCAL, local_levels=k, **(extra or {}))
            d.fill_(12345)
            st, lv = B.bfs_single_ex(g, int(src), d, params=p, stats=True, level_cap=1 << 14)
            got = d.cpu().numpy()
            assert np.array_equal(got, want), (k, int(src), np.nonzero(got != want)[0][:10])
            reached = int((want >= 0).sum())
            assert st["reached"] == reached
            assert st["edges_reached"] == int(deg[want >= 0].sum())
            assert st["levels"] == int(want.max()) + 1 and st["td_levels"] == st["levels"]
            assert st["bu_levels"] == 0
            assert st["improved"] >= reached - 1  # every reached vertex but the source is lowered at least once
            assert st["td_frontier"] >= reached   # and expanded at least once
            assert st["supersteps"] >= 1 and len(lv) == min(st["supersteps"], 1 << 14)
            # a super-step advances at most k levels
            assert st["supersteps"] * k >= st["levels"] - 1 or st["supersteps"] >= st["levels"]
            assert all(x["direction"] == 2 for x in lv)
            assert lv[0]["frontier"] == 1 and lv[-1]["found"] == 0
            # without the counting variant the same distances come back
            d.fill_(-7)
            B.bfs_single_ex(g, int(src), d, params=p)
            assert np.array_equal(d.cpu().numpy(), want), (k, int(src), "production kernel")
    g.free()


@pytest.mark.parametrize("head", [True, False])
def test_closed_forms(bfs, head):
    cases = [G.path_graph(1), G.path_graph(2), G.path_graph(300), G.star_graph(40), G.complete_graph(9),
             G.cycle_graph(33), graphgen.grid2d(7, 45), graphgen.grid2d(64, 64)]
    for rp, col in cases:
        n = len(rp) - 1
        check(bfs, rp, col, sorted({0, n // 2, n - 1}), head=head)


def test_disjoint_union_isolated_source(bfs):
    edges = [(i, i + 1) for i in range(4)] + [(5 + i, 5 + (i + 1) % 6) for i in range(6)]
    rp, col = G.csr_from_edges(70, edges)  # vertices 11..69 isolated
    check(bfs, rp, col, [2, 5, 11, 69])


@pytest.mark.parametrize("bits,head", [(32, True), (64, False)])
def test_rmat_hubs_overflow_local_queues(bfs, bits, head):
    """Hub-heavy graph: a block's share expands into far more than its shared-memory queue holds."""
    rp, col = graphgen.rmat(14, seed=7)
    check(bfs, rp, col, graphgen.sources(rp, 3, 1002), ks=(1, 4, 16), rp_bits=bits, head=head)


def test_large_diameter_graphs(bfs):
    for rp, col in (graphgen.grid2d(300, 211), graphgen.rgg(40000, graphgen.rgg_radius(40000, 6.0), 3),
                    G.path_graph(5000)):
        check(bfs, rp, col, graphgen.sources(rp, 2, 1003), ks=(3, 16, 200), rp_bits=32)


def test_block_shapes(bfs):
    rp, col = graphgen.grid2d(120, 97)
    for extra in (dict(local_threads=64), dict(local_threads=512, blocks_per_sm=1),
                  dict(local_threads=128, blocks_per_sm=1), dict(local_threads=96, blocks_per_sm=3)):
        check(bfs, rp, col, [0, 5000], ks=(8,), rp_bits=32, extra=extra)


def test_hub_row_longer_than_a_window(bfs):
    """A star with more than 2^20 leaves: the centre's row is taken in several windows."""
    n = (1 << 20) + 300
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1] = n - 1
    rp[2:] = n - 1 + np.arange(1, n, dtype=np.int64)
    col = np.concatenate([np.arange(1, n, dtype=np.int32), np.zeros(n - 1, dtype=np.int32)])
    check(bfs, rp, col, [0, 7], ks=(1, 16))


def test_other_launch_modes(bfs):
    rp, col = graphgen.grid2d(40, 40)
    g = bfs.bfs_graph_upload(rp, col)
    d = torch.empty(1600, dtype=torch.int32, device="cuda")
    want = oracle.bfs(rp, col, 3)
    bfs.bfs_single_ex(g, 3, d, params=bfs.make_params(policy=bfs.BFS_POLICY_LOCAL, launch=bfs.BFS_LAUNCH_GRAPH))
    assert np.array_equal(d.cpu().numpy(), want)
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_single_ex(g, 3, d, params=bfs.make_params(policy=bfs.BFS_POLICY_LOCAL,
                                                         launch=bfs.BFS_LAUNCH_PER_LEVEL))
    assert e.value.code == bfs.BFS_EINVAL
    for bad in (dict(local_levels=0), dict(local_levels=5000), dict(local_threads=32), dict(local_threads=100),
                dict(local_threads=1024)):
        with pytest.raises(bfs.BfsError) as e:
            bfs.bfs_single_ex(g, 3, d, params=bfs.make_params(policy=bfs.BFS_POLICY_LOCAL, **bad))
        assert e.value.code == bfs.BFS_EINVAL
    # relabel is ignored: same distances
    bfs.bfs_single_ex(g, 3, d, params=bfs.make_params(policy=bfs.BFS_POLICY_LOCAL, relabel=1))
    assert np.array_equal(d.cpu().numpy(), want)
    g.free()


def test_auto_policy_picks_local_for_large_diameter(bfs):
    """Average degree below 7 and no list longer than 4096: AUTO runs the local kernel (its
    counters report super-steps); a star with a longer list stays level-synchronous."""
    rp, col = graphgen.grid2d(64, 64)
    g = bfs.bfs_graph_upload(rp, col)
    d = torch.empty(4096, dtype=torch.int32, device="cuda")
    st, _ = bfs.bfs_single_ex(g, 0, d, stats=True)
    assert st["supersteps"] > 0 and np.array_equal(d.cpu().numpy(), oracle.bfs(rp, col, 0))
    g.free()
    rp, col = G.star_graph(5000)
    g = bfs.bfs_graph_upload(rp, col)
    d = torch.empty(5000, dtype=torch.int32, device="cuda")
    st, _ = bfs.bfs_single_ex(g, 3, d, stats=True)
    assert st["supersteps"] == 0 and np.array_equal(d.cpu().numpy(), oracle.bfs(rp, col, 3))
    g.free()


def test_barrier_timeout_reports_status(bfs):
    """A grid barrier told to wait for one block more than launched runs out of time: BFS_ETIMEOUT,
    and the next query on the same graph still succeeds."""
    rp, col = graphgen.grid2d(50, 50)
    g = bfs.bfs_graph_upload(rp, col)
    d = torch.empty(2500, dtype=torch.int32, device="cuda")
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_single_ex(g, 0, d, params=bfs.make_params(policy=bfs.BFS_POLICY_LOCAL, test_barrier_extra=1,
                                                         timeout_ms=50))
    assert e.value.code == bfs.BFS_ETIMEOUT
    bfs.bfs_single_ex(g, 0, d, params=bfs.make_params(policy=bfs.BFS_POLICY_LOCAL))
    assert np.array_equal(d.cpu().numpy(), oracle.bfs(rp, col, 0))
    g.free()
