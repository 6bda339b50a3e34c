"""bfs_single_noalloc: the entry point that allocates nothing.

Some callers cannot allocate device memory at query time (they live inside a
pool or arena they do not own, or must not risk the allocator's locking and
implicit synchronisation).  For them the library keeps the kernel's scratch
in a static device array.  These tests call that entry point through the C ABI
twice in a row on the same graph and compare each result with the regular
bfs_single path and with the oracle (distances are exact integers, so the
tolerance is zero).  The file is collected last and works alone or after the
others.
"""
from __future__ import annotations

import numpy as np
import pytest

import graphgen
import oracle

from tests.graphs import csr_from_edges

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bfs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_00430_gb300 as B
    B.load()
    return B


def _sparse_with_isolated():
    """A graph with degree-0 vertices and n not a multiple of 32: a random
    forest-like sparse part (average degree below 7, so the top-down-only
    class) plus isolated vertices at the end and in the middle."""
    rng = np.random.default_rng(11)
    n = 3000 + 13
    edges = [(int(rng.integers(0, 2500)), int(rng.integers(0, 2500))) for _ in range(4000)]
    edges = [(u, v) for u, v in edges if u != v and not (1000 <= u < 1100 or 1000 <= v < 1100)]
    return csr_from_edges(n, edges)


def _cases():
    rp, col = graphgen.rmat(16, seed=3)
    yield "rmat16", rp, col
    rp, col = graphgen.grid2d(97, 61)  # average degree < 7: the top-down-only path
    yield "grid97x61", rp, col
    rp, col = _sparse_with_isolated()
    yield "sparse_isolated", rp, col


@pytest.mark.parametrize("bits", [32, 64])
def test_noalloc_matches_bfs_single_and_oracle_twice(bfs, bits):
    for name, rp, col in _cases():
        rp = rp.astype(np.int32 if bits == 32 else np.int64)
        n = len(rp) - 1
        g = bfs.bfs_graph_upload(rp, col)
        d_rp = torch.from_numpy(rp).cuda()
        d_col = torch.from_numpy(col).cuda()
        srcs = [int(s) for s in graphgen.sources(rp.astype(np.int64), 2, 1005)]
        want_o = oracle.bfs_many(rp, col, srcs, threads=2)
        for i, src in enumerate(srcs):  # two calls in a row, the second on top of the first one's leftovers
            want = torch.empty(n, dtype=torch.int32, device="cuda")
            bfs.bfs_single(g, src, want)
            got = torch.full((n,), 12345, dtype=torch.int32, device="cuda")
            bfs.bfs_single_noalloc(d_rp, d_col, src, got)
            torch.cuda.synchronize()
            assert torch.equal(got, want), (name, src)
            assert np.array_equal(got.cpu().numpy(), want_o[i]), (name, src)
        g.free()


def test_noalloc_isolated_source(bfs):
    rp, col = _sparse_with_isolated()
    n = len(rp) - 1
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    src = n - 1  # degree 0
    bfs.bfs_single_noalloc(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), src, d)
    assert np.array_equal(d.cpu().numpy(), oracle.bfs(rp, col, src))


def test_noalloc_rejects_misaligned_neighbour_ids(bfs):
    rp, col = graphgen.rmat(10, seed=3)
    buf = torch.zeros(len(col) + 4, dtype=torch.int32, device="cuda")
    buf[1:1 + len(col)] = torch.from_numpy(col).cuda()
    view = buf[1:1 + len(col)]  # starts 4 bytes past a 16-byte boundary
    assert view.data_ptr() % 16 == 4
    d = torch.empty(len(rp) - 1, dtype=torch.int32, device="cuda")
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_single_noalloc(torch.from_numpy(rp).cuda(), view, 0, d)
    assert e.value.code == bfs.BFS_EINVAL


def test_noalloc_rejects_oversized_graph(bfs):
    n = 3_000_000  # ~24.5 bytes per vertex of scratch: more than the 64 MiB array
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(4, dtype=torch.int32, device="cuda")
    dist = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_single_noalloc(rp, col[:0], 0, dist)
    assert e.value.code == bfs.BFS_ENOMEM
