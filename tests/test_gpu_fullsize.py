"""Parity at the benchmark's full sizes, in the configurations bench.py times.

Every test builds its graph, upload flags and query parameters through the
same bench.py helpers the benchmark uses (make_workload, upload_flags,
query_params, msbfs_workload, large_specs, serve_specs), so what is checked
here is what is timed there.  Distances are unique (every writer of a level
stores the same value, the paper's Section 2 argument for its non-atomic
stores), so every compared row must equal the oracle's bit for bit.  The
oracle runs on the host cores, one source per thread, in batches sized to the
core count so host memory stays bounded.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import bench
import graphgen
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

THREADS = max(1, min(32, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def bfs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_00430_gb300 as B
    B.load()
    return B


def batches(srcs, k=THREADS):
    srcs = [int(s) for s in srcs]
    for i in range(0, len(srcs), k):
        yield i, srcs[i:i + k]


def check_single_source_workload(bfs, argv):
    """All 64 bench sources of a single-source workload, on the bench's stream
    and parameters, device output; the first batch also through a host buffer
    (the bench's end-to-end path)."""
    args = bench.parse_args(argv)
    rp, col, srcs, _, _ = bench.make_workload(args)
    assert len(srcs) == bench.NSRC == 64
    g = bfs.bfs_graph_upload(rp, col, flags=bench.upload_flags(bfs, args))
    n = len(rp) - 1
    params = bench.query_params(bfs, args, n, len(col))
    stream = torch.cuda.Stream()
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    host = torch.empty(n, dtype=torch.int32, pin_memory=True).numpy()
    checked = 0
    for i0, b in batches(srcs):
        want = oracle.bfs_many(rp, col, b, threads=len(b))
        for k, s in enumerate(b):
            bfs.bfs_single_ex(g, s, d, params=params, stream=stream)
            stream.synchronize()
            assert np.array_equal(d.cpu().numpy(), want[k]), (argv, i0 + k, s)
            if i0 == 0 and k < 4:
                bfs.bfs_single_ex(g, s, host, params=params, stream=stream)
                assert np.array_equal(host, want[k]), (argv, "host output", s)
            checked += 1
        del want
    g.free()
    assert checked == 64


def test_rmat_s25_bench_configuration_all_64_sources(bfs):
    """The headline: R-MAT scale 25, int64 row pointers, degree-ordered lists, the bench's query
    parameters (the tuning table's entry for the graph's class)."""
    args = bench.parse_args([])
    assert args.workload == "rmat25" and args.policy is None and args.launch is None and args.relabel is None
    check_single_source_workload(bfs, [])


def test_er_2e24_bench_configuration_all_64_sources(bfs):
    check_single_source_workload(bfs, ["--workload", "er24"])


def test_large_diameter_bench_configuration(bfs):
    """Grid 4096^2 and RGG 2^23, top-down only (the bench's large-diameter runs), all 8 sources,
    persistent launch, its CUDA-graph replay and the multi-level local expansion; the first 2
    sources also with one launch per level."""
    for name, make in bench.large_specs():
        rp, col = make()
        srcs = [int(s) for s in graphgen.sources(rp, 8, bench.LARGE_SRC_SEED)]
        g = bfs.bfs_graph_upload(rp.astype(np.int32), col, flags=bfs.BFS_VALIDATE)
        want = oracle.bfs_many(rp, col, srcs, threads=min(THREADS, len(srcs)))
        d = torch.empty(len(rp) - 1, dtype=torch.int32, device="cuda")
        for i, s in enumerate(srcs):
            for policy, launch in ((3, 0), (3, 2), (bfs.BFS_POLICY_LOCAL, 0)) + (((3, 1),) if i < 2 else ()):
                d.fill_(77)
                bfs.bfs_single_ex(g, s, d, params=bfs.make_params(policy=policy, launch=launch))
                assert np.array_equal(d.cpu().numpy(), want[i]), (name, i, policy, launch)
        g.free()


def test_msbfs_rmat_s24_all_256_rows(bfs):
    """R-MAT scale 24, 256 sources in one call: every uint8 row against the oracle, and the int32
    output on a sample of rows (the bench's multi-source configuration)."""
    rp, col, srcs = bench.msbfs_workload()
    n = len(rp) - 1
    g = bfs.bfs_graph_upload(rp, col, flags=bfs.BFS_VALIDATE | bfs.BFS_DEGREE_ORDER)
    mp = bfs.tuned_params(None, g, "multi")
    out = torch.empty((256, n), dtype=torch.uint8, device="cuda")
    bfs.bfs_multi_ex(g, srcs, out, dist_bits=8, params=mp)
    torch.cuda.synchronize()
    sample32 = set(range(0, 256, 17)) | {255}
    want32 = {}
    for i0, b in batches(srcs):
        want = oracle.bfs_many(rp, col, b, threads=len(b))
        got = out[i0:i0 + len(b)].cpu().numpy()
        assert np.array_equal(got, oracle.to_uint8(want)), i0
        for k in range(len(b)):
            if i0 + k in sample32:
                want32[i0 + k] = want[k]
        del want, got
    del out
    out32 = torch.empty((256, n), dtype=torch.int32, device="cuda")
    bfs.bfs_multi_ex(g, srcs, out32, dist_bits=32, params=mp)
    for i, w in want32.items():
        assert np.array_equal(out32[i].cpu().numpy(), w), i
    del out32
    g.free()


def test_serving_resident_graphs_full_size(bfs):
    """The five resident graphs of the serving workload at full size, 50 queries each, submitted as
    one interleaved stream (they share the device and join running groups); every result equals
    the oracle's."""
    per_graph = 50
    rng = np.random.default_rng(55)
    graphs, handles = [], []
    for name, make in bench.serve_specs():
        rp, col = make()
        graphs.append((name, rp, col))
        handles.append(bfs.bfs_graph_upload(rp, col, flags=bfs.BFS_DEGREE_ORDER))
    srv = bfs.bfs_serve_create(200 << 30)
    ids = [srv.add_graph(h) for h in handles]
    queries = []
    for gi, (_, rp, _) in enumerate(graphs):
        pool = graphgen.sources(rp, 4096, bench.SERVE_SRC_SEED)
        queries += [(gi, int(pool[j])) for j in rng.integers(0, 4096, size=per_graph)]
    order = rng.permutation(len(queries))
    outs, tickets = {}, {}
    torch.cuda.synchronize()
    for qi in order:
        gi, s = queries[qi]
        outs[qi] = torch.empty(len(graphs[gi][1]) - 1, dtype=torch.int32, device="cuda")
        tickets[qi] = srv.submit(ids[gi], s, outs[qi])
    for qi in order:
        st = srv.wait(tickets[qi], 600_000_000)
        assert st["status"] == 0
    for gi, (name, rp, col) in enumerate(graphs):
        qis = [qi for qi in range(len(queries)) if queries[qi][0] == gi]
        for i0, b in batches([queries[qi][1] for qi in qis]):
            want = oracle.bfs_many(rp, col, b, threads=len(b))
            for k in range(len(b)):
                qi = qis[i0 + k]
                assert np.array_equal(outs[qi].cpu().numpy(), want[k]), (name, queries[qi][1])
    srv.destroy()
    for h in handles:
        h.free()


def test_graphset_10000_every_graph(bfs):
    """One launch over the 10,000-graph set of the bench: every graph's distances against the oracle."""
    from concurrent.futures import ThreadPoolExecutor
    gs = graphgen.graph_set(10000, 1000, 100000, 8.0, seed=4)
    s = bfs.bfs_graphset_upload(gs.voff, gs.eoff, gs.row_ptr, gs.col)
    dist = torch.empty(int(gs.voff[-1]), dtype=torch.int32, device="cuda")
    bfs.bfs_graphset_run(s, gs.src, dist, params=bfs.tuned_params(None, None, "graphset"))
    got = dist.cpu().numpy()

    def ok(i):
        rp, col = gs.graph(i)
        return bool(np.array_equal(got[gs.voff[i]:gs.voff[i + 1]], oracle.bfs(rp, col, int(gs.src[i]))))

    with ThreadPoolExecutor(max_workers=THREADS) as ex:
        res = list(ex.map(ok, range(gs.count)))
    bad = [i for i, r in enumerate(res) if not r]
    assert not bad, bad[:10]
    s.free()
