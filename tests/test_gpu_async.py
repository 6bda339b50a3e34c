"""GPU parity of the asynchronous single-source entry points (bfs_single_async /
bfs_single_wait) against the oracle, and their status reporting.

Queries are enqueued back to back without waiting; every output buffer must
equal the oracle's distances exactly once bfs_single_wait has returned, in
every launch form, across streams, and mixed with synchronous calls.  A query
whose grid barrier runs out (a barrier that waits for one block more than
launched) is reported by the next wait, once, and the graph stays usable.
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


def _enqueue_all(B, g, srcs, n, params=None, streams=(None,)):
    outs = []
    for i, src in enumerate(srcs):
        d = torch.full((n,), 77, dtype=torch.int32, device="cuda")
        B.bfs_single_async(g, int(src), d, params=params, stream=streams[i % len(streams)])
        outs.append(d)
    return outs


@pytest.mark.parametrize("kw", [dict(), dict(relabel=1), dict(launch=2), dict(launch=1), dict(policy=3),
                                dict(policy=4, launch=2, relabel=1)])
def test_back_to_back_queries_match_the_oracle(bfs, kw):
    rp, col = graphgen.rmat(15, seed=3)
    g = bfs.bfs_graph_upload(rp, col, flags=bfs.BFS_VALIDATE | bfs.BFS_DEGREE_ORDER)
    n = len(rp) - 1
    srcs = graphgen.sources(rp, 12, 21)
    outs = _enqueue_all(bfs, g, srcs, n, params=bfs.make_params(**kw))
    bfs.bfs_single_wait(g)
    for src, d in zip(srcs, outs):
        assert np.array_equal(d.cpu().numpy(), oracle.bfs(rp, col, int(src))), (kw, int(src))
    g.free()


def test_queries_on_two_streams_run_in_submission_order(bfs):
    """Alternating streams share the graph's workspace: each query waits for the previous one."""
    rp, col = graphgen.erdos_renyi(1 << 14, 6.0, 5)
    g = bfs.bfs_graph_upload(rp, col)
    n = len(rp) - 1
    srcs = graphgen.sources(rp, 10, 4)
    streams = (torch.cuda.Stream(), torch.cuda.Stream())
    outs = _enqueue_all(bfs, g, srcs, n, streams=streams)
    bfs.bfs_single_wait(g)
    torch.cuda.synchronize()
    for src, d in zip(srcs, outs):
        assert np.array_equal(d.cpu().numpy(), oracle.bfs(rp, col, int(src)))
    g.free()


def test_local_expansion_and_deep_paths(bfs):
    """Large-diameter graphs: the multi-level local kernel (AUTO) and a path deeper than 254
    levels, where distances are written during the levels."""
    for (rp, col), kw in ((graphgen.grid2d(96, 80), dict()), (G.path_graph(700), dict(policy=3)),
                          (G.path_graph(700), dict())):
        g = bfs.bfs_graph_upload(rp, col)
        n = len(rp) - 1
        srcs = [0, n // 2, n - 1]
        outs = _enqueue_all(bfs, g, srcs, n, params=bfs.make_params(**kw))
        bfs.bfs_single_wait(g)
        for src, d in zip(srcs, outs):
            assert np.array_equal(d.cpu().numpy(), oracle.bfs(rp, col, int(src))), (n, kw, src)
        g.free()


def test_pinned_host_output_and_pageable_rejected(bfs):
    rp, col = graphgen.rmat(13, seed=9)
    g = bfs.bfs_graph_upload(rp, col)
    n = len(rp) - 1
    srcs = graphgen.sources(rp, 4, 2)
    hosts = [torch.full((n,), 77, dtype=torch.int32).pin_memory().numpy() for _ in srcs]
    for src, h in zip(srcs, hosts):
        bfs.bfs_single_async(g, int(src), h)
    bfs.bfs_single_wait(g)
    for src, h in zip(srcs, hosts):
        assert np.array_equal(h, oracle.bfs(rp, col, int(src)))
    pageable = np.zeros(n, dtype=np.int32)
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_single_async(g, int(srcs[0]), pageable)
    assert e.value.code == bfs.BFS_EINVAL
    g.free()


def test_invalid_arguments(bfs):
    rp, col = G.path_graph(8)
    g = bfs.bfs_graph_upload(rp, col)
    d = torch.empty(8, dtype=torch.int32, device="cuda")
    for src in (-1, 8):
        with pytest.raises(bfs.BfsError) as e:
            bfs.bfs_single_async(g, src, d)
        assert e.value.code == bfs.BFS_EINVAL
    with pytest.raises(bfs.BfsError):
        bfs.bfs_single_async(g, 0, d, params=bfs.make_params(chunk=10))
    bfs.bfs_single_wait(g)  # nothing enqueued yet: returns at once
    g.free()


@pytest.mark.parametrize("launch", [0, 2])
def test_failed_query_is_reported_once_by_the_next_wait(bfs, launch):
    """One query among several runs out of its barrier wait: the wait raises BFS_ETIMEOUT, the
    following wait is clean, the other queries are exact, and the graph keeps working."""
    rp, col = graphgen.rmat(12, seed=4)
    g = bfs.bfs_graph_upload(rp, col)
    n = len(rp) - 1
    srcs = graphgen.sources(rp, 5, 6)
    ok = bfs.make_params(launch=launch)
    bad = bfs.make_params(launch=launch, test_barrier_extra=1, timeout_ms=50)
    outs = []
    for i, src in enumerate(srcs):
        d = torch.empty(n, dtype=torch.int32, device="cuda")
        bfs.bfs_single_async(g, int(src), d, params=bad if i == 1 else ok)
        outs.append(d)
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_single_wait(g)
    assert e.value.code == bfs.BFS_ETIMEOUT
    bfs.bfs_single_wait(g)
    for i, (src, d) in enumerate(zip(srcs, outs)):
        if i != 1:
            assert np.array_equal(d.cpu().numpy(), oracle.bfs(rp, col, int(src)))
    # the last query fails: its status is still in the control block when the wait runs
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    bfs.bfs_single_async(g, int(srcs[0]), d, params=ok)
    bfs.bfs_single_async(g, int(srcs[0]), d, params=bad)
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_single_wait(g)
    assert e.value.code == bfs.BFS_ETIMEOUT
    bfs.bfs_single_wait(g)
    bfs.bfs_single(g, int(srcs[2]), d)
    assert np.array_equal(d.cpu().numpy(), oracle.bfs(rp, col, int(srcs[2])))
    g.free()


def test_mixed_with_synchronous_calls(bfs):
    """A synchronous call returns its own failure, and the next wait does not repeat it; its
    statistics and the enqueued queries around it stay exact."""
    rp, col = graphgen.rmat(13, seed=11)
    g = bfs.bfs_graph_upload(rp, col)
    n = len(rp) - 1
    srcs = graphgen.sources(rp, 3, 7)
    a = torch.empty(n, dtype=torch.int32, device="cuda")
    b = torch.empty(n, dtype=torch.int32, device="cuda")
    bfs.bfs_single_async(g, int(srcs[0]), a)
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_single_ex(g, int(srcs[1]), b, params=bfs.make_params(test_barrier_extra=1, timeout_ms=50))
    assert e.value.code == bfs.BFS_ETIMEOUT
    st, _ = bfs.bfs_single_ex(g, int(srcs[1]), b, stats=True)
    want_b = oracle.bfs(rp, col, int(srcs[1]))
    assert st["reached"] == int((want_b >= 0).sum())
    c = torch.empty(n, dtype=torch.int32, device="cuda")
    bfs.bfs_single_async(g, int(srcs[2]), c)
    bfs.bfs_single_wait(g)
    for src, d in zip(srcs, (a, b, c)):
        assert np.array_equal(d.cpu().numpy(), oracle.bfs(rp, col, int(src)))
    g.free()
