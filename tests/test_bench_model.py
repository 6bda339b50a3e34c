"""The benchmark's measurement arithmetic on hand-worked cases (CPU).

harmonic_gteps is the harmonic mean of per-BFS rates; algorithmic_bytes is the
compulsory-byte model of the method behind roofline.achieved (init 4n + n/8;
top-down 4|F| + 2*RP*|F| + 4*E_td + 4|F'| + 4|F'|; bottom-up 3n/8 + RP*U +
4*E_bu + 4|F'|; conversion n/8 + 4|F|); layout_bytes is the library-layout
model reported beside it.  The expected values below are worked out term by
term from each model's definition (query overhead, then each level's
top-down / bottom-up / conversion terms)."""
from __future__ import annotations

import pytest

import bench


def test_harmonic_gteps():
    # Rates 2 and 4 GTEPS: harmonic mean 2 / (1/2 + 1/4) = 8/3.
    assert bench.harmonic_gteps([2e9, 4e9], [1.0, 1.0]) == pytest.approx(8 / 3)
    # One BFS: its own rate.
    assert bench.harmonic_gteps([5e8], [0.25]) == pytest.approx(2.0)


LEVELS = [
    # top-down from the source: 1 frontier vertex, 2 entries, 2 found
    dict(direction=0, converted=0, frontier=1, edges=2, unvisited=0, found=2),
    # converted to bottom-up: 2 frontier vertices, 5 unvisited scanned, 10 entries, 3 found
    dict(direction=1, converted=1, frontier=2, edges=10, unvisited=5, found=3),
    # converted back to top-down: 3 frontier vertices, 6 entries, none found
    dict(direction=0, converted=1, frontier=3, edges=6, unvisited=0, found=0),
]


def test_algorithmic_bytes_compulsory_model():
    n = 64
    init = 4 * n + n / 8                                     # dist, visited
    l0 = 4 * 1 + 2 * 8 * 1 + 4 * 2 + 4 * 2 + 4 * 2          # queue, row ptrs, ids, dist, append
    l1 = (n / 8 + 4 * 2) + (3 * n / 8 + 8 * 5 + 4 * 10 + 4 * 3)
    l2 = (n / 8 + 4 * 3) + (4 * 3 + 2 * 8 * 3 + 4 * 6 + 0)
    assert bench.algorithmic_bytes(n, 8, LEVELS) == pytest.approx(init + l0 + l1 + l2)
    assert init + l0 + l1 + l2 == 544                       # 264 + 44 + 132 + 104
    assert bench.algorithmic_bytes(n, 4, LEVELS) == pytest.approx(492)  # 264 + 36 + 112 + 80


def test_algorithmic_bytes_counts_probes_when_bitmap_exceeds_half_l2():
    # n/8 = 8 bytes against half of an 8-byte "L2": each of the 2 + 10 + 6 probes costs 4 bytes.
    assert bench.algorithmic_bytes(64, 8, LEVELS, l2_bytes=8) == pytest.approx(544 + 4 * 18)


def test_algorithmic_bytes_path_closed_form():
    """Top-down BFS along a path of 10 vertices from one end: every level has
    one frontier vertex and finds one (the last finds none); degrees 1, 2 x 8, 1."""
    import oracle
    from tests import graphs as G
    from tests.replay import replay
    rp, col = G.path_graph(10)
    _, lv = replay(rp, col, 0, oracle.bfs(rp, col, 0), policy=3)
    want = (4 * 10 + 10 / 8) + 10 * (4 + 2 * 8) + 4 * 18 + 8 * 9
    assert bench.algorithmic_bytes(10, 8, lv) == pytest.approx(want)
    assert want == 385.25


def test_layout_bytes_head_table():
    n = 64
    query = n + n / 4 + 5 * n                                # level bytes, visited init, expansion
    l0 = 8 * 1 + 4 * 2 + (16 + 1 + 8 + 4) * 2                # items, ids, per found: head, byte, item, queue
    l1 = (n / 8 + 4 * 2) + (3 * n / 8 + 16 * 5 + 4 * max(0, 10 - 2 * 5) + 3)
    l2 = (n / 8 + (16 + 8) * 3) + (8 * 3 + 4 * 6 + 0)
    assert bench.layout_bytes(n, 8, LEVELS) == pytest.approx(query + l0 + l1 + l2)
    assert query + l0 + l1 + l2 == 725


def test_layout_bytes_row_pointers_no_queue():
    n, rp = 64, 4
    query = n + n / 4 + 5 * n
    l0 = 8 * 1 + 4 * 2 + (2 * rp + 1 + 8) * 2
    l1 = (n / 8 + 4 * 2) + (3 * n / 8 + rp * 5 + 4 * 10 + 3)
    l2 = (n / 8 + (2 * rp + 8) * 3) + (8 * 3 + 4 * 6)
    got = bench.layout_bytes(n, rp, LEVELS, head=False, queue=False)
    assert got == pytest.approx(query + l0 + l1 + l2)
    assert got == 657  # 400 + 50 + 103 + 104


def test_msbfs_bytes_hand_worked():
    """256 sources (W = 4 words, 32-byte masks), 8-byte row pointers, n = 100 vertices of which 80
    have edges; one push level (2 frontier vertices, 10 pushed entries) and two pull levels
    (50 + 20 vertices missing a lane, 300 + 40 entries examined); 60 vertices gained a lane in all;
    uint8 output."""
    st = dict(pull_levels=2, push_levels=1, pull_active=70, pulled_edges=340, push_frontier=2, pushed_edges=10,
              found=60)
    pull = 2 * (2 * 32 * 80) + 8 * 70 + (4 + 32) * 340        # masks of scanned vertices, row ptrs, gathers
    push = (32 + 2 * 8) * 2 + (4 + 32) * 10                   # frontier masks + row ptrs, pushed entries
    found = 2 * 32 * 60
    out = 256 * 100 * 1
    assert bench.msbfs_bytes(100, 80, 256, 8, st, 1) == pull + push + found + out
    assert pull + push + found + out == 10240 + 560 + 12240 + 96 + 360 + 3840 + 25600
    # 64 sources: one word (8-byte masks), int32 output
    st1 = dict(st)
    assert bench.msbfs_bytes(100, 80, 64, 4, st1, 4) == (2 * (2 * 8 * 80) + 4 * 70 + 12 * 340 + (8 + 8) * 2
                                                         + 12 * 10 + 16 * 60 + 64 * 100 * 4)


def test_graphset_bytes():
    # 3 graphs, 10 vertices, 40 entries: 8 * (10 + 3) row pointers + 4 * 40 list + 4 * 10 distances
    assert bench.graphset_bytes(10, 40, 3) == 104 + 160 + 40


def test_launches_per_query_counts_the_reset_and_the_levels():
    """gpu_launches claims two launches per query (control-block reset + one persistent, graph or
    local kernel); with one launch per level: reset, init, every level, two per direction change
    (the worst case: zeroing + scatter), final expansion."""
    from types import SimpleNamespace
    per_src = [{"stats": {"levels": 7, "conversions": 2}}, {"stats": {"levels": 9, "conversions": 0}}]
    for launch in (0, 2):
        assert bench.launches_per_query(SimpleNamespace(launch=launch), per_src) == 4
    assert bench.launches_per_query(SimpleNamespace(launch=1), per_src) == (3 + 7 + 4) + (3 + 9)
