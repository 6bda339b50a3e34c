"""GPU parity of single-source BFS against the oracle (bit-exact).

Distances are unique (the shortest-path hop count), so every policy, launch
mode and parameter set must reproduce the oracle's int32 array exactly.  The
work counters the library reports are compared with the host replay of the
same policy on the oracle's levels.
"""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle
from tests import graphs as G
from tests.replay import POLICY_LOCAL, replay, resolve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bfs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_00430_gb300 as B
    B.load()
    return B


POLICIES = {
    "auto": dict(policy=0),
    "frontier": dict(policy=1),
    "edges": dict(policy=2),
    "td_only": dict(policy=3),
    "bu_from_1": dict(policy=4),
    "script_alt": dict(policy=5, script=0xAAAAAAAAAAAAAAAA),
    "script_rand": dict(policy=5, script=0x9D3F5A61C2E4B807),
}


def run(B, g, src, n, stream=None, **kw):
    dist = torch.empty(n, dtype=torch.int32, device="cuda")
    p = B.make_params(**kw)
    st, lv = B.bfs_single_ex(g, int(src), dist, params=p, stats=True, level_cap=4096, stream=stream)
    return dist.cpu().numpy(), st, lv


def check(B, rp, col, srcs, rp_bits=64, policies=POLICIES, launches=(0, 1), extra=None, check_stats=True,
          degree_order=False, head=True):
    flags = B.BFS_VALIDATE | B.BFS_VALIDATE_SYMMETRY | (B.BFS_DEGREE_ORDER if degree_order else 0)
    flags |= 0 if head else B.BFS_NO_HEAD
    g = B.bfs_graph_upload(rp, col, flags=flags, row_ptr_bits=rp_bits)
    n = len(rp) - 1
    for src in srcs:
        want = oracle.bfs(rp, col, int(src))
        for name, kw in policies.items():
            for launch in launches:
                kw2 = dict(kw, launch=launch, **(extra or {}))
                got, st, lv = run(B, g, src, n, **kw2)
                assert np.array_equal(got, want), (name, launch, int(src), np.nonzero(got != want)[0][:10])
                deg = np.diff(np.asarray(rp, dtype=np.int64))
                local = launch != 1 and resolve(kw.get("policy", 0), n, len(col),
                                                max_degree=int(deg.max())) == POLICY_LOCAL
                if local:  # AUTO on a large-diameter graph: the local kernel (its counters: test_gpu_local.py)
                    assert st["supersteps"] > 0
                if check_stats and not local:
                    est, elv = replay(rp, col, int(src), want, policy=kw.get("policy", 0), script=kw.get("script", 0),
                                      degree_order=degree_order)
                    for k, v in est.items():
                        assert st[k] == v, (name, launch, k, st[k], v)
                    got_lv = [{k: v for k, v in x.items() if k != "ns"} for x in lv]
                    assert got_lv == elv, (name, launch)
    g.free()


@pytest.mark.parametrize("head", [True, False])
def test_closed_form_graphs(bfs, head):
    cases = [G.path_graph(1), G.path_graph(2), G.path_graph(100), G.star_graph(40), G.complete_graph(9),
             G.cycle_graph(33), graphgen.grid2d(7, 45)]
    for rp, col in cases:
        n = len(rp) - 1
        check(bfs, rp, col, sorted({0, n // 2, n - 1}), head=head)


def test_disjoint_union_and_isolated(bfs):
    edges = [(i, i + 1) for i in range(4)] + [(5 + i, 5 + (i + 1) % 6) for i in range(6)]
    rp, col = G.csr_from_edges(70, edges)  # vertices 11..69 isolated
    check(bfs, rp, col, [2, 5, 11, 69])


def test_rmat_s16_td(bfs):
    """R-MAT scale 16, plain top-down, 8 sources, int32 row pointers."""
    rp, col = graphgen.rmat(16)
    srcs = graphgen.sources(rp, 8, 1001)
    check(bfs, rp, col, srcs, rp_bits=32, policies={"td_only": dict(policy=3)}, launches=(0, 1, 2))


@pytest.mark.parametrize("bits,head", [(32, True), (64, True), (32, False), (64, False)])
def test_rmat_s14_all_policies(bfs, bits, head):
    rp, col = graphgen.rmat(14, seed=7)
    check(bfs, rp, col, graphgen.sources(rp, 3, 1002), rp_bits=bits, head=head)


def test_er_and_rgg_and_grid(bfs):
    for rp, col in (graphgen.erdos_renyi(20000, 16, 2), graphgen.rgg(30000, graphgen.rgg_radius(30000, 6.0), 3),
                    graphgen.grid2d(150, 131)):
        check(bfs, rp, col, graphgen.sources(rp, 2, 1003), rp_bits=32,
              policies={k: POLICIES[k] for k in ("auto", "frontier", "edges", "script_rand")})


@pytest.mark.parametrize("params", [
    dict(small_max=1, chunk=256, bu_warp_min=0, threads_per_block=128),
    dict(small_max=8, chunk=300, bu_warp_min=4, threads_per_block=1024, blocks_per_sm=1),
    dict(small_max=32, chunk=65535, bu_warp_min=1000000, threads_per_block=256, blocks_per_sm=2),
    dict(bu_chunk=0),
    dict(bu_chunk=1, threads_per_block=64),
    dict(bu_chunk=4096),
    dict(bu_thread_max=0),
    dict(bu_thread_max=4, bu_warp_min=0),
    dict(bu_thread_max=1 << 20, bu_warp_min=1 << 24),
])
@pytest.mark.parametrize("head", [True, False])
def test_parameter_extremes(bfs, params, head):
    rp, col = graphgen.rmat(13, seed=9)
    check(bfs, rp, col, graphgen.sources(rp, 2, 1004), extra=params, head=head,
          policies={k: POLICIES[k] for k in ("edges", "bu_from_1", "script_rand")})


def test_hub_split_over_chunks(bfs):
    """A star with 200,000 leaves: the hub's adjacency exceeds 65,535 and is split into chunks."""
    rp, col = G.star_graph(200001)
    check(bfs, rp, col, [0, 7], policies={k: POLICIES[k] for k in ("td_only", "edges", "bu_from_1")})


def test_host_output_buffer(bfs):
    rp, col = graphgen.rmat(12)
    g = bfs.bfs_graph_upload(rp, col)
    src = int(graphgen.sources(rp, 1, 5)[0])
    host = np.full(len(rp) - 1, 77, dtype=np.int32)
    bfs.bfs_single(g, src, host)
    assert np.array_equal(host, oracle.bfs(rp, col, src))
    g.free()


def test_stream_and_repeated_queries(bfs):
    rp, col = graphgen.rmat(13)
    g = bfs.bfs_graph_upload(rp, col)
    s = torch.cuda.Stream()
    srcs = graphgen.sources(rp, 5, 8)
    outs = []
    for src in srcs:
        d = torch.empty(len(rp) - 1, dtype=torch.int32, device="cuda")
        bfs.bfs_single(g, int(src), d, stream=s)
        outs.append(d)
    torch.cuda.synchronize()
    for src, d in zip(srcs, outs):
        assert np.array_equal(d.cpu().numpy(), oracle.bfs(rp, col, int(src)))
    g.free()


def test_invalid_arguments(bfs):
    rp, col = G.path_graph(5)
    g = bfs.bfs_graph_upload(rp, col)
    d = torch.empty(5, dtype=torch.int32, device="cuda")
    for src in (-1, 5):
        with pytest.raises(bfs.BfsError) as e:
            bfs.bfs_single(g, src, d)
        assert e.value.code == bfs.BFS_EINVAL
    with pytest.raises(bfs.BfsError):
        bfs.bfs_single_ex(g, 0, d, params=bfs.make_params(chunk=10))
    g.free()
    bad = col.copy()
    bad[0] = 9
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_graph_upload(rp, bad, flags=bfs.BFS_VALIDATE)
    assert e.value.code == bfs.BFS_EINVAL
    rp2, col2 = G.csr_from_edges(4, [(0, 1), (1, 2)], symmetric=False)
    with pytest.raises(bfs.BfsError):
        bfs.bfs_graph_upload(rp2, col2, flags=bfs.BFS_VALIDATE_SYMMETRY)
    rp3 = rp.copy()
    rp3[2], rp3[3] = rp3[3], rp3[2]
    with pytest.raises(bfs.BfsError):
        bfs.bfs_graph_upload(rp3, col, flags=bfs.BFS_VALIDATE)


def test_barrier_timeout_reports_status(bfs):
    """The grid barrier waits for one block more than launched: the bounded wait
    runs out, the query returns BFS_ETIMEOUT, and the context stays usable."""
    rp, col = G.path_graph(64)
    g = bfs.bfs_graph_upload(rp, col)
    d = torch.empty(64, dtype=torch.int32, device="cuda")
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_single_ex(g, 0, d, params=bfs.make_params(test_barrier_extra=1, timeout_ms=50))
    assert e.value.code == bfs.BFS_ETIMEOUT
    bfs.bfs_single(g, 3, d)
    assert np.array_equal(d.cpu().numpy(), oracle.bfs(rp, col, 3))
    g.free()


def test_graph_info(bfs):
    rp, col = G.csr_from_edges(10, [(0, 1), (0, 2), (0, 3)])
    g = bfs.bfs_graph_upload(rp, col)
    assert g.info() == {"n": 10, "m": 6, "max_degree": 3, "isolated": 6}
    g.free()


@pytest.mark.parametrize("bits", [32, 64])
def test_degree_ordered_layout(bfs, bits):
    """BFS_DEGREE_ORDER changes only the scan order: same distances, counters of the reordered CSR."""
    rp, col = graphgen.rmat(14, seed=11)
    check(bfs, rp, col, graphgen.sources(rp, 3, 1006), rp_bits=bits, degree_order=True)
    rp, col = G.star_graph(3000)
    check(bfs, rp, col, [0, 5], rp_bits=bits, degree_order=True,
          policies={k: POLICIES[k] for k in ("edges", "bu_from_1")})


@pytest.mark.parametrize("launch", [0, 1, 2])
def test_level_records_without_counters(bfs, launch):
    """Level records from the non-counting kernel match the counting kernel's (ns aside)."""
    rp, col = graphgen.rmat(13, seed=21)
    g = bfs.bfs_graph_upload(rp, col, flags=bfs.BFS_DEGREE_ORDER)
    n = len(rp) - 1
    for src in graphgen.sources(rp, 2, 1010):
        want = oracle.bfs(rp, col, int(src))
        d0 = torch.empty(n, dtype=torch.int32, device="cuda")
        st, lv = bfs.bfs_single_ex(g, int(src), d0, params=bfs.make_params(launch=launch), stats=True, level_cap=64)
        d1 = torch.empty(n, dtype=torch.int32, device="cuda")
        none, lv1 = bfs.bfs_single_ex(g, int(src), d1, params=bfs.make_params(launch=launch), level_cap=64)
        assert none is None
        assert np.array_equal(d1.cpu().numpy(), want)
        keys = ("direction", "converted", "frontier", "found")
        assert [{k: x[k] for k in keys} for x in lv1] == [{k: x[k] for k in keys} for x in lv]
        assert all(x["edges"] == 0 and x["unvisited"] == 0 for x in lv1)
        if launch != 1:
            assert all(x["ns"] > 0 for x in lv1)
    g.free()


@pytest.mark.parametrize("bits", [32, 64])
def test_renumbered_copy(bfs, bits):
    """params.relabel: the search runs on the degree-renumbered copy (lists highest degree first), so the
    distances are the oracle's and the counters those of the degree-ordered layout, in every launch mode;
    a graph uploaded in caller order (lists sorted after renumbering) and isolated sources too."""
    rp, col = graphgen.rmat(14, seed=12)
    iso = [int(v) for v in np.flatnonzero(np.diff(rp) == 0)[:1]]
    srcs = [int(s) for s in graphgen.sources(rp, 3, 1011)] + iso
    check(bfs, rp, col, srcs, rp_bits=bits, degree_order=True, launches=(0, 1, 2), extra=dict(relabel=1))
    g = bfs.bfs_graph_upload(rp, col, row_ptr_bits=bits)
    n = len(rp) - 1
    for src in srcs:
        got, _, _ = run(bfs, g, src, n, relabel=1)
        assert np.array_equal(got, oracle.bfs(rp, col, src)), src
    g.free()


def test_renumbered_copy_deep_search(bfs):
    """More than 254 levels on the renumbered copy: distances past the level bytes are written through the
    new-to-caller id map."""
    for rp, col in (G.path_graph(600), graphgen.grid2d(3, 400)):
        n = len(rp) - 1
        check(bfs, rp, col, [0, n // 3, n - 1], policies={k: POLICIES[k] for k in ("auto", "edges")},
              launches=(0, 1), extra=dict(relabel=1), check_stats=False)


def _big_star():
    """Centre 0 with 2^20 + 300 leaves: one list longer than 2^20 entries (a hub record of
    more than 4096 chunk tickets in top-down levels, a whole-warp scan in bottom-up ones)."""
    n = (1 << 20) + 301
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1] = n - 1
    rp[2:] = n - 1 + np.arange(1, n, dtype=np.int64)
    col = np.concatenate([np.arange(1, n, dtype=np.int32), np.zeros(n - 1, dtype=np.int32)])
    return rp, col


def test_hub_longer_than_2_pow_20(bfs):
    rp, col = _big_star()
    pol = {k: POLICIES[k] for k in ("td_only", "edges", "bu_from_1", "frontier")}
    check(bfs, rp, col, [0, 7, len(rp) - 2], policies=pol)
    check(bfs, rp, col, [0, 7], policies=pol, launches=(0,), extra=dict(relabel=1), check_stats=False)


def _fan(n, k):
    """Source 0 joined to vertices 1..k; every other vertex hangs off one of them (round robin)."""
    edges = [(0, i) for i in range(1, k + 1)] + [(1 + (v - k - 1) % k, v) for v in range(k + 1, n)]
    return G.csr_from_edges(n, edges)


@pytest.mark.parametrize("k,bottom_up", [(20, True), (19, False)])
def test_frontier_rule_at_exactly_n_over_20(bfs, k, bottom_up):
    """n = 400 (divisible by 20) and |F_1| = k: the paper's rule (top-down while |F| is below 5 % of
    n, read as the integer test 20 |F| < n) sends level 1 bottom-up at |F_1| = n/20 = 20 exactly and
    keeps it top-down at 19; distances are the oracle's either way."""
    rp, col = _fan(400, k)
    check(bfs, rp, col, [0], policies={"frontier": dict(policy=1)})
    g = bfs.bfs_graph_upload(rp, col)
    d = torch.empty(400, dtype=torch.int32, device="cuda")
    for launch in (0, 1):
        _, lv = bfs.bfs_single_ex(g, 0, d, params=bfs.make_params(policy=1, launch=launch), level_cap=8)
        assert lv[1]["frontier"] == k and lv[1]["direction"] == (1 if bottom_up else 0), (launch, lv[1])
    g.free()


def test_pinned_host_output_written_directly(bfs):
    """Pinned host output is written by the kernel through its device alias: exact on a hybrid
    search, on the renumbered copy, and on a path deeper than 254 levels (where distances are
    written during the levels instead of by the final expansion)."""
    for (rp, col), kw in ((graphgen.rmat(14, seed=7), dict()), (graphgen.rmat(14, seed=7), dict(relabel=1)),
                          (G.path_graph(600), dict(policy=3)), (G.path_graph(600), dict(policy=3, launch=1)),
                          (G.path_graph(600), dict())):  # AUTO: the local kernel, staged
        g = bfs.bfs_graph_upload(rp, col)
        n = len(rp) - 1
        host = torch.full((n,), 77, dtype=torch.int32).pin_memory().numpy()
        for src in (0, n // 3):
            bfs.bfs_single_ex(g, src, host, params=bfs.make_params(**kw))
            assert np.array_equal(host, oracle.bfs(rp, col, src)), (n, kw, src)
        g.free()
