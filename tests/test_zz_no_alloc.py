"""bfs_single_noalloc: the entry point that allocates nothing.

Some callers cannot allocate device memory at query time (they live inside a
pool or arena they do not own, or must not risk the allocator's locking and
implicit synchronisation).  For them the library keeps the kernel's scratch
in a static device array.  This test calls that entry point through the C ABI
twice in a row on the same graph and compares each result with the regular
bfs_single path (distances are exact integers, so the tolerance is zero).
It sits in its own file, collected last, and works alone or after the others.
"""
from __future__ import annotations

import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bfs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_00430_gb300 as B
    B.load()
    return B


@pytest.mark.parametrize("bits", [32, 64])
def test_noalloc_matches_bfs_single_twice(bfs, bits):
    rp, col = graphgen.rmat(16, seed=3)
    rp = rp.astype(np.int32 if bits == 32 else np.int64)
    n = len(rp) - 1
    g = bfs.bfs_graph_upload(rp, col)
    d_rp = torch.from_numpy(rp).cuda()
    d_col = torch.from_numpy(col).cuda()
    srcs = graphgen.sources(rp.astype(np.int64), 2, 1005)
    for src in srcs:  # two calls in a row, the second on top of the first one's leftovers
        want = torch.empty(n, dtype=torch.int32, device="cuda")
        bfs.bfs_single(g, int(src), want)
        got = torch.full((n,), 12345, dtype=torch.int32, device="cuda")
        bfs.bfs_single_noalloc(d_rp, d_col, int(src), got)
        torch.cuda.synchronize()
        assert torch.equal(got, want), int(src)
    g.free()


def test_noalloc_rejects_oversized_graph(bfs):
    n = 3_000_000  # ~24.5 bytes per vertex of scratch: more than the 64 MiB array
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(4, dtype=torch.int32, device="cuda")
    dist = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(bfs.BfsError) as e:
        bfs.bfs_single_noalloc(rp, col[:0], 0, dist)
    assert e.value.code == bfs.BFS_ENOMEM
