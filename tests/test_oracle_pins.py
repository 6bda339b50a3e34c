"""Pins for the oracle (CPU only).

The oracle (serial queue BFS, ``oracle/bfs_oracle.c``) is checked here against
facts that do not come from it: brute-force repeated relaxation, closed-form
distances and the BFS invariants.  A final test plants plausible mistakes in
a copy of the oracle source and checks that every one of them trips a pin.
"""
from __future__ import annotations

import itertools
import os
import random
import subprocess
import sys

import numpy as np
import pytest

import graphgen
import oracle
from tests import graphs as G


# ---- pin suite (parameterised by an oracle library so mutants can be run) ----

def pin_bruteforce_exhaustive(lib, max_n=5):
    """Every simple undirected graph on n <= max_n labelled vertices, every source."""
    for n in range(1, max_n + 1):
        pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(pairs)):
            edges = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
            rp, col = G.csr_from_edges(n, edges)
            for s in range(n):
                got = oracle.bfs(rp, col, s, lib)
                want = G.brute_force_dist(n, edges, s)
                if not np.array_equal(got, want):
                    return False, (n, edges, s, got.tolist(), want.tolist())
    return True, None


def pin_bruteforce_atlas(lib):
    """Every graph on up to 7 vertices up to isomorphism (the 1,253 graphs of networkx's graph
    atlas), every source: distances are equivariant under relabelling, so together with the
    labelled exhaustive pin above this covers every graph of <= 7 vertices."""
    try:
        import networkx as nx
    except ImportError:  # pragma: no cover - networkx is part of the image
        return True, "networkx missing: skipped"
    for h in nx.graph_atlas_g():
        n = h.number_of_nodes()
        if n == 0:
            continue
        edges = [(int(a), int(b)) for a, b in h.edges()]
        rp, col = G.csr_from_edges(n, edges)
        for s in range(n):
            got = oracle.bfs(rp, col, s, lib)
            want = G.brute_force_dist(n, edges, s)
            if not np.array_equal(got, want):
                return False, (n, edges, s, got.tolist(), want.tolist())
    return True, None


def pin_bruteforce_random(lib, cases=300, seed=12345):
    """Random multigraphs (self-loops and repeated pairs included) on up to 64 vertices."""
    rng = random.Random(seed)
    for _ in range(cases):
        n = rng.randint(1, 64)
        k = rng.randint(0, 3 * n)
        edges = [(rng.randrange(n), rng.randrange(n)) for _ in range(k)]
        rp, col = G.csr_from_edges(n, edges)
        s = rng.randrange(n)
        got = oracle.bfs(rp, col, s, lib)
        want = G.brute_force_dist(n, edges, s)
        if not np.array_equal(got, want):
            return False, (n, edges, s)
    return True, None


def pin_closed_forms(lib):
    """Paths, stars, complete graphs, cycles, grids, disjoint unions."""
    for n in (1, 2, 3, 7, 50):
        rp, col = G.path_graph(n)
        for s in {0, n // 2, n - 1}:
            want = np.abs(np.arange(n) - s)
            if not np.array_equal(oracle.bfs(rp, col, s, lib), want):
                return False, ("path", n, s)
    for n in (2, 3, 10):
        rp, col = G.star_graph(n)
        want = np.ones(n, dtype=np.int32)
        want[0] = 0
        if not np.array_equal(oracle.bfs(rp, col, 0, lib), want):
            return False, ("star centre", n)
        want = np.full(n, 2, dtype=np.int32)
        want[0], want[n - 1] = 1, 0
        if not np.array_equal(oracle.bfs(rp, col, n - 1, lib), want):
            return False, ("star leaf", n)
    for n in (1, 2, 6):
        rp, col = G.complete_graph(n)
        for s in range(n):
            want = np.ones(n, dtype=np.int32)
            want[s] = 0
            if not np.array_equal(oracle.bfs(rp, col, s, lib), want):
                return False, ("complete", n, s)
    for n in (3, 4, 9, 10):
        rp, col = G.cycle_graph(n)
        for s in (0, n // 3):
            i = np.arange(n)
            want = np.minimum(np.abs(i - s), n - np.abs(i - s))
            if not np.array_equal(oracle.bfs(rp, col, s, lib), want):
                return False, ("cycle", n, s)
    for r, c in ((1, 1), (1, 6), (5, 4), (17, 23)):
        rp, col = graphgen.grid2d(r, c)
        for s in (0, (r // 2) * c + c // 3, r * c - 1):
            rr, cc = np.divmod(np.arange(r * c), c)
            want = np.abs(rr - s // c) + np.abs(cc - s % c)
            if not np.array_equal(oracle.bfs(rp, col, s, lib), want):
                return False, ("grid", r, c, s)
    # disjoint union of a path (0..4) and a cycle (5..10) plus an isolated vertex 11
    edges = [(i, i + 1) for i in range(4)] + [(5 + i, 5 + (i + 1) % 6) for i in range(6)]
    rp, col = G.csr_from_edges(12, edges)
    want = np.array([2, 1, 0, 1, 2] + [-1] * 7, dtype=np.int32)
    if not np.array_equal(oracle.bfs(rp, col, 2, lib), want):
        return False, ("union path",)
    want = np.array([-1] * 5 + [0, 1, 2, 3, 2, 1, -1], dtype=np.int32)
    if not np.array_equal(oracle.bfs(rp, col, 5, lib), want):
        return False, ("union cycle",)
    want = np.array([-1] * 11 + [0], dtype=np.int32)
    if not np.array_equal(oracle.bfs(rp, col, 11, lib), want):
        return False, ("isolated",)
    return True, None


def pin_invariants(lib):
    """BFS invariants on seeded generator graphs (R-MAT, uniform random, RGG)."""
    cases = [graphgen.rmat(10, seed=3), graphgen.erdos_renyi(3000, 3.0, 5),
             graphgen.rgg(4000, graphgen.rgg_radius(4000, 3.0), 6)]
    for rp, col in cases:
        comp = G.components(rp, col)
        for s in graphgen.sources(rp, 4, 77):
            d = oracle.bfs(rp, col, int(s), lib)
            try:
                G.check_bfs_invariants(rp, col, int(s), d, comp)
            except AssertionError as e:
                return False, str(e)
    return True, None


PINS = [pin_bruteforce_exhaustive, pin_bruteforce_atlas, pin_bruteforce_random, pin_closed_forms, pin_invariants]


# ---- the oracle itself ----

@pytest.mark.parametrize("pin", PINS, ids=lambda p: p.__name__)
def test_oracle_pin(pin):
    ok, info = pin(oracle._load())
    assert ok, info


def test_union_find_matches_scipy():
    rp, col = graphgen.erdos_renyi(2000, 1.5, 9)
    a = G.union_find(rp, col)
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    n = len(rp) - 1
    lab = connected_components(sp.csr_matrix((np.ones(len(col)), col, rp), shape=(n, n)), directed=False)[1]
    # same partition: map each union-find root to the scipy label
    m = {}
    for x, y in zip(a.tolist(), lab.tolist()):
        assert m.setdefault(x, y) == y
    assert len(set(m.values())) == len(m)


def test_oracle_rejects_bad_input():
    rp, col = G.path_graph(3)
    with pytest.raises(ValueError):
        oracle.bfs(rp, col, 3)
    with pytest.raises(ValueError):
        oracle.bfs(rp, col, -1)
    bad = col.copy()
    bad[0] = 7
    with pytest.raises(ValueError):
        oracle.bfs(rp, bad, 0)


def test_oracle_many_matches_single():
    rp, col = graphgen.rmat(9, seed=4)
    srcs = graphgen.sources(rp, 6, 5)
    many = oracle.bfs_many(rp, col, srcs)
    for i, s in enumerate(srcs):
        assert np.array_equal(many[i], oracle.bfs(rp, col, int(s)))


def test_uint8_encoding():
    d = np.array([0, 1, -1, 254], dtype=np.int32)
    assert oracle.to_uint8(d).tolist() == [0, 1, 255, 254]
    with pytest.raises(OverflowError):
        oracle.to_uint8(np.array([255], dtype=np.int32))


# ---- planted mistakes: each must trip at least one pin ----

MUTANTS = {
    "dropped +1": ("dist[v] = dist[u] + 1;", "dist[v] = dist[u];"),
    "source level 1": ("dist[src] = 0;", "dist[src] = 1;"),
    "skip last neighbour": ("j < row_ptr[u + 1]; ++j", "j < row_ptr[u + 1] - 1; ++j"),
    "skip first neighbour": ("int64_t j = row_ptr[u];", "int64_t j = row_ptr[u] + 1;"),
    "row index for column": ("int64_t v = col[j];", "int64_t v = col[u];"),
    "LIFO instead of FIFO": ("int64_t u = queue[head++];", "int64_t u = queue[--tail];"),
    "no visited test": ("if (dist[v] == -1) {", "if (dist[v] == -1 || dist[v] > dist[u]) {"),
    "next row pointer": ("row_ptr[u + 1]; ++j", "row_ptr[u + 2 > n ? n : u + 2]; ++j"),
}


def _run_pins_on(lib_path: str) -> list[str]:
    """Names of the pins that fail for the oracle library at ``lib_path``."""
    lib = oracle.load_library(lib_path)
    caught = []
    for pin in PINS:
        try:
            ok, _ = pin(lib)
        except (ValueError, IndexError, AssertionError):
            ok = False
        if not ok:
            caught.append(pin.__name__)
    return caught


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    """Each mutant runs in a child process: a mutant that corrupts memory and
    aborts is also a detected failure, and cannot take the test run down."""
    old, new = MUTANTS[name]
    src = open(oracle._SRC).read()
    assert old in src, f"mutation anchor missing: {old}"
    mutated = src.replace(old, new)
    if name == "LIFO instead of FIFO":
        mutated = mutated.replace("while (head < tail)", "while (tail > 0)")
    path = tmp_path / "mutant.c"
    path.write_text(mutated)
    so = oracle.build(force=True, src=str(path), out=str(tmp_path / "libmutant.so"))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r); from tests.test_oracle_pins import _run_pins_on; "
            "print('CAUGHT', ','.join(_run_pins_on(%r)))" % (root, so))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return  # the mutant crashed the process: caught
    line = [x for x in r.stdout.splitlines() if x.startswith("CAUGHT")][-1]
    assert line.strip() != "CAUGHT", f"mutant '{name}' passed every pin"


def test_golden_oracle_distances():
    """Oracle output hashes stored by tests/golden/make_golden.py (cross-machine regression:
    the same seeded graphs and the same distances on x86 and Arm hosts)."""
    import hashlib
    import json
    path = os.path.join(os.path.dirname(__file__), "golden", "graphs.json")
    with open(path) as f:
        gold = json.load(f)
    for name, rec in gold["graphs"].items():
        rp, col = eval("graphgen." + rec["call"])  # noqa: S307 - fixed calls from the fixture
        for s, want in zip(rec["sources"], rec["dist"]):
            d = oracle.bfs(rp, col, s)
            assert hashlib.sha256(d.astype(np.int32).tobytes()).hexdigest() == want["sha256"], (name, s)
            assert int((d >= 0).sum()) == want["reached"] and int(d.max()) == want["eccentricity"]
