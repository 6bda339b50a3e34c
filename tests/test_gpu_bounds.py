"""The small parity cases again, on the bounds-checked build of the library.

The bounds-checked variant (compiled with GBFS_DEBUG_BOUNDS) checks every
data-dependent global index of the single-source kernels - level-synchronous
hybrid, top-down only, bottom-up from level 1, scripted switches, the
renumbered copy, graphs without the head table, the no-allocation entry point
and the multi-level local kernel - against its array and records the first
violation.  The cases run in a child process (the binding holds one library
per process); every distance array must equal the oracle's and no index may
have left its array.
"""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, ROOT)
import numpy as np, torch
import graphgen, oracle
from tests import graphs as G
import paper_2503_00430_gb300 as bfs
from paper_2503_00430_gb300 import build
bfs.load(build.build(debug_bounds=True))
first, checked = bfs.bfs_debug_bounds(reset=True)
assert checked, "the library was built without bounds checks"
cases = [G.path_graph(1), G.path_graph(300), G.star_graph(2000), G.complete_graph(9), G.cycle_graph(33),
         graphgen.grid2d(37, 45), graphgen.rmat(12, seed=5), graphgen.rmat(14, seed=7),
         graphgen.erdos_renyi(5000, 12, 3), G.csr_from_edges(70, [(i, i + 1) for i in range(4)])]
policies = [dict(policy=0), dict(policy=1), dict(policy=2), dict(policy=3), dict(policy=4),
            dict(policy=5, script=0x9D3F5A61C2E4B807), dict(policy=2, relabel=1), dict(policy=6, local_levels=4),
            dict(policy=2, launch=1), dict(policy=3, launch=2)]
runs = 0
for rp, col in cases:
    n = len(rp) - 1
    srcs = sorted({0, n // 2, n - 1})
    for flags in (bfs.BFS_DEGREE_ORDER, bfs.BFS_NO_HEAD):
        g = bfs.bfs_graph_upload(rp, col, flags=flags)
        d = torch.empty(n, dtype=torch.int32, device="cuda")
        for s in srcs:
            want = oracle.bfs(rp, col, s)
            for kw in policies:
                d.fill_(77)
                bfs.bfs_single_ex(g, s, d, params=bfs.make_params(**kw))
                assert np.array_equal(d.cpu().numpy(), want), (n, flags, s, kw)
                runs += 1
            d.fill_(77)
            bfs.bfs_single_noalloc(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), s, d)
            assert np.array_equal(d.cpu().numpy(), want), (n, "noalloc", s)
        g.free()
first, checked = bfs.bfs_debug_bounds()
assert first == 0, "out-of-range index recorded: site %d index %d" % ((first >> 48) & 0x7fff, first & 0xffffffffffff)
print("bounds ok", runs)
""".replace("ROOT", repr(ROOT))


def test_small_parity_cases_stay_in_bounds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "-c", CHILD], capture_output=True, text=True, timeout=1200, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "bounds ok" in r.stdout
