"""Checks of the seeded input generators (CPU only)."""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

import graphgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "graphs.json")


def _well_formed(rp, col):
    n = len(rp) - 1
    assert rp[0] == 0 and rp[-1] == len(col)
    assert np.all(np.diff(rp) >= 0)
    assert col.min(initial=0) >= 0 and col.max(initial=-1) < n
    src = np.repeat(np.arange(n), np.diff(rp))
    assert not np.any(src == col), "self-loop"
    # rows sorted strictly ascending (no duplicates)
    d = np.diff(col.astype(np.int64))
    same_row = np.diff(src) == 0
    assert np.all(d[same_row] > 0), "row not strictly ascending"
    # symmetric: the sorted arc list equals its transpose
    a = np.sort(src.astype(np.int64) * n + col)
    b = np.sort(col.astype(np.int64) * n + src)
    assert np.array_equal(a, b), "not symmetric"


@pytest.mark.parametrize("make", [
    lambda: graphgen.rmat(11, seed=2),
    lambda: graphgen.erdos_renyi(5000, 16, 2),
    lambda: graphgen.grid2d(33, 17),
    lambda: graphgen.rgg(6000, graphgen.rgg_radius(6000, 3.0), 3),
])
def test_well_formed_and_deterministic(make):
    rp, col = make()
    _well_formed(rp, col)
    rp2, col2 = make()
    assert graphgen.csr_sha256(rp, col) == graphgen.csr_sha256(rp2, col2)


def test_grid_edge_count_closed_form():
    for r, c in ((1, 1), (2, 3), (64, 64), (7, 40)):
        rp, col = graphgen.grid2d(r, c)
        assert len(col) == 2 * (r * (c - 1) + c * (r - 1))


def test_rmat_heavy_tail_and_bounds():
    rp, col = graphgen.rmat(14)
    deg = np.diff(rp)
    n = 1 << 14
    assert len(col) <= 2 * 16 * n
    assert deg.max() > 20 * deg.mean()
    assert (deg == 0).sum() > 0  # R-MAT leaves isolated vertices


def test_rgg_mean_degree_near_target():
    n = 1 << 16
    rp, col = graphgen.rgg(n, graphgen.rgg_radius(n, 3.0), 11)
    assert 2.8 < len(col) / n < 3.05  # border effects pull it slightly below 3


def test_sources_have_degree():
    rp, col = graphgen.rmat(12)
    s = graphgen.sources(rp, 200, 9)
    assert np.all(np.diff(rp)[s] > 0)
    assert np.array_equal(s, graphgen.sources(rp, 200, 9))


def test_graph_set_shapes():
    gs = graphgen.graph_set(40, 1000, 100000, 8.0, 4)
    sizes = np.diff(gs.voff)
    assert sizes.min() >= 1000 and sizes.max() <= 100000
    for i in range(0, 40, 7):
        rp, col = gs.graph(i)
        _well_formed(rp, col)
        assert 0 <= gs.src[i] < len(rp) - 1
        assert rp[gs.src[i] + 1] > rp[gs.src[i]]


def test_thread_count_independent():
    """Same graph whatever the OpenMP thread count (run in a child process)."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r); import graphgen; "
            "print(graphgen.csr_sha256(*graphgen.rmat(13, seed=5)))" % root)
    outs = set()
    for t in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=t)
        outs.add(subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                                check=True).stdout.strip())
    outs.add(graphgen.csr_sha256(*graphgen.rmat(13, seed=5)))
    assert len(outs) == 1


def test_golden_hashes():
    """Hashes written by tests/golden/make_golden.py: same graphs on every machine."""
    with open(GOLDEN) as f:
        gold = json.load(f)
    for name, rec in gold["graphs"].items():
        rp, col = eval("graphgen." + rec["call"])  # noqa: S307 - fixed calls from the fixture
        assert graphgen.csr_sha256(rp, col) == rec["csr_sha256"], name
        assert len(rp) - 1 == rec["n"] and len(col) == rec["m"], name
