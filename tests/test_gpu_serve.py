"""Serving loop: every query's distances equal the oracle's, alone or in a mix
(bit-exact: the tolerance for serving is zero differences)."""
from __future__ import annotations

import time

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


@pytest.fixture(scope="module")
def graphs(bfs):
    gs = [graphgen.rmat(12, seed=31), graphgen.grid2d(40, 60), graphgen.erdos_renyi(3000, 10, 32),
          G.csr_from_edges(50, [(i, i + 1) for i in range(20)])]
    handles = [bfs.bfs_graph_upload(rp, col) for rp, col in gs]
    yield gs, handles
    for h in handles:
        h.free()


def run_mix(bfs, gs, handles, queries, budget=1 << 32, device_out=True, stagger=0.0, **kw):
    srv = bfs.bfs_serve_create(budget, bfs.make_params(**kw) if kw else None)
    ids = [srv.add_graph(h) for h in handles]
    outs, tickets = [], []
    for k, (gi, src) in enumerate(queries):
        n = len(gs[gi][0]) - 1
        out = (torch.full((n,), 77, dtype=torch.int32, device="cuda") if device_out
               else torch.full((n,), 77, dtype=torch.int32).pin_memory().numpy() if k % 2 else np.full(n, 77, np.int32))
        outs.append(out)
        if device_out:
            torch.cuda.synchronize()  # the fill must not be pending when the server starts writing the row
        tickets.append(srv.submit(ids[gi], src, out))
        if stagger:
            time.sleep(stagger)
    stats = [srv.wait(t, 60_000_000) for t in tickets]
    for (gi, src), out in zip(queries, outs):
        got = out.cpu().numpy() if hasattr(out, "cpu") else out
        assert np.array_equal(got, oracle.bfs(*gs[gi], src)), (gi, src)
    srv.destroy()
    return stats


def mix(gs, k, seed):
    rng = np.random.default_rng(seed)
    q = []
    for _ in range(k):
        gi = int(rng.integers(len(gs)))
        q.append((gi, int(graphgen.sources(gs[gi][0], 1, int(rng.integers(1 << 30)))[0])))
    return q


def test_single_queries_alone(bfs, graphs):
    gs, handles = graphs
    for gi in range(len(gs)):
        run_mix(bfs, gs, handles, [(gi, int(graphgen.sources(gs[gi][0], 1, 5)[0]))])


def test_mix_many_queries_lane_reuse(bfs, graphs):
    gs, handles = graphs
    stats = run_mix(bfs, gs, handles, mix(gs, 300, 1))  # > 64 per graph: lanes are reused
    assert all(s["status"] == 0 and s["done_ns"] >= s["start_ns"] >= s["submit_ns"] for s in stats)


def test_staggered_arrivals_join_running_groups(bfs, graphs):
    gs, handles = graphs
    stats = run_mix(bfs, gs, handles, mix(gs, 120, 2), stagger=0.0005)
    assert max(s["lane"] for s in stats) < 64


def test_host_outputs_and_tight_budget(bfs, graphs):
    gs, handles = graphs
    # Budget: the groups plus only a few staging buffers, so host-output queries queue for memory.
    run_mix(bfs, gs, handles, mix(gs, 40, 3), device_out=False, budget=80 << 20)


@pytest.mark.parametrize("kw", [dict(ms_ring=2), dict(tau_inv=1), dict(tau_inv=100000), dict(ms_heavy_min=8)])
def test_parameters(bfs, graphs, kw):
    gs, handles = graphs
    run_mix(bfs, gs, handles, mix(gs, 100, 4), **kw)


def test_errors(bfs, graphs):
    gs, handles = graphs
    srv = bfs.bfs_serve_create(1 << 30)
    gid = srv.add_graph(handles[3])
    out = torch.empty(50, dtype=torch.int32, device="cuda")
    with pytest.raises(bfs.BfsError) as e:
        srv.submit(gid + 1, 0, out)
    assert e.value.code == bfs.BFS_ENOTFOUND
    with pytest.raises(bfs.BfsError) as e:
        srv.submit(gid, 50, out)
    assert e.value.code == bfs.BFS_EINVAL
    t = srv.submit(gid, 3, out)
    srv.wait(t)
    with pytest.raises(bfs.BfsError) as e:
        srv.poll(t)
    assert e.value.code == bfs.BFS_ENOTFOUND
    srv.destroy()


@pytest.mark.parametrize("ring", [16, 3])
def test_persistent_push_levels_large_diameter(bfs, ring):
    """A large-diameter graph runs many push levels per persistent launch (every level a push with
    tau_inv=1); lanes retire and join between launches; every query's distances are the oracle's."""
    rp, col = graphgen.grid2d(30, 90)
    g = bfs.bfs_graph_upload(rp, col)
    gs = [(rp, col)]
    for rep in range(2):
        qs = [(0, int(s)) for s in graphgen.sources(rp, 200, 4000 + rep)]
        run_mix(bfs, gs, [g], qs, tau_inv=1, ms_ring=ring)
    g.free()


def _group_budget_for_one(n):
    """A budget that holds the lane group of one graph with n vertices (at most about 193 bytes per
    vertex plus a few KB with the default 16-level ring) but not two (at least 160 bytes per vertex each)."""
    return 200 * n + 8192


def test_budget_for_one_group_serves_two_busy_graphs(bfs):
    """Two graphs with traffic and a budget that fits one group at a time: the group holding the
    memory drains and releases it when the other graph waits, so every query completes, exactly."""
    gs = [graphgen.rmat(12, seed=41), graphgen.rmat(12, seed=42)]
    handles = [bfs.bfs_graph_upload(rp, col) for rp, col in gs]
    qs = mix(gs, 160, 7)
    assert {gi for gi, _ in qs} == {0, 1}
    stats = run_mix(bfs, gs, handles, qs, budget=_group_budget_for_one(4096))
    assert all(s["status"] == 0 for s in stats)
    for h in handles:
        h.free()


def test_group_larger_than_budget_fails_with_enomem(bfs):
    rp, col = graphgen.rmat(12, seed=43)
    g = bfs.bfs_graph_upload(rp, col)
    srv = bfs.bfs_serve_create(10 * 4096)
    gid = srv.add_graph(g)
    out = torch.empty(4096, dtype=torch.int32, device="cuda")
    t = srv.submit(gid, 5, out)
    with pytest.raises(bfs.BfsError) as e:
        srv.wait(t, 30_000_000)
    assert e.value.code == bfs.BFS_ENOMEM
    srv.destroy()
    g.free()


def test_serving_loop_timeout_fails_only_that_group(bfs):
    """The persistent push loop of a large-diameter group waits at a grid barrier for one block more
    than launched: the wait runs out after 50 ms, the query ends with BFS_ETIMEOUT, and the server
    keeps serving (another graph's query completes exactly; the next grid query times out again
    instead of hanging)."""
    grid = graphgen.grid2d(40, 60)
    rm = graphgen.rmat(12, seed=44)
    hg, hr = bfs.bfs_graph_upload(*grid), bfs.bfs_graph_upload(*rm)
    srv = bfs.bfs_serve_create(1 << 30, bfs.make_params(test_barrier_extra=1, timeout_ms=50))
    ig, ir = srv.add_graph(hg), srv.add_graph(hr)
    og = torch.empty(2400, dtype=torch.int32, device="cuda")
    orr = torch.empty(4096, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    for rep in range(2):
        t = srv.submit(ig, 7 + rep, og)
        with pytest.raises(bfs.BfsError) as e:
            srv.wait(t, 60_000_000)
        assert e.value.code == bfs.BFS_ETIMEOUT
        with pytest.raises(bfs.BfsError) as e:  # the query itself ended (reported once), not the wait
            srv.poll(t)
        assert e.value.code == bfs.BFS_ENOTFOUND
        src = int(graphgen.sources(rm[0], 1, 50 + rep)[0])
        st = srv.wait(srv.submit(ir, src, orr), 60_000_000)
        assert st["status"] == 0
        assert np.array_equal(orr.cpu().numpy(), oracle.bfs(*rm, src))
    srv.destroy()
    hg.free()
    hr.free()


def test_full_queue_returns_eagain(bfs):
    """At most serve_queue submitted queries wait for admission; beyond that bfs_serve_submit returns
    BFS_EAGAIN and accepts again once the backlog drains.  Accepted queries are exact."""
    rp, col = graphgen.grid2d(256, 256)  # ~500 levels per query: submissions outrun completions
    g = bfs.bfs_graph_upload(rp, col)
    srv = bfs.bfs_serve_create(1 << 30, bfs.make_params(serve_queue=4))
    gid = srv.add_graph(g)
    srcs = [int(s) for s in graphgen.sources(rp, 200, 61)]
    outs = [torch.empty(len(rp) - 1, dtype=torch.int32, device="cuda") for _ in srcs]
    torch.cuda.synchronize()
    accepted, rejected = [], 0
    for s, o in zip(srcs, outs):
        try:
            accepted.append((s, o, srv.submit(gid, s, o)))
        except bfs.BfsError as e:
            assert e.code == bfs.BFS_EAGAIN
            rejected += 1
    assert rejected > 0 and len(accepted) <= 64 + 4 + 64  # lanes + queue (+ lanes freed meanwhile)
    for s, o, t in accepted:
        assert srv.wait(t, 120_000_000)["status"] == 0
        assert np.array_equal(o.cpu().numpy(), oracle.bfs(rp, col, s)), s
    t = srv.submit(gid, srcs[0], outs[0])
    srv.wait(t, 120_000_000)
    assert np.array_equal(outs[0].cpu().numpy(), oracle.bfs(rp, col, srcs[0]))
    srv.destroy()
    g.free()
