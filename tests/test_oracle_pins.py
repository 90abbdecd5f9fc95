"""Pins for the CPU oracle: each ties it to the mathematics, not to itself.

* BFS: exhaustive brute force over every digraph on 3 and 4 vertices, random
  graphs up to 64 vertices, a hand-worked fixture, and the directed-BFS
  characterisation on the full-size power-law graphs.
* SSSP: (n-1)-round Bellman-Ford on random graphs up to 64 vertices, the
  hand-worked fixture, unit weights reducing to BFS, and the
  triangle-inequality-plus-tightness characterisation at full size.
* Tessellation: hand-derived point counts (tests/golden/bezier_counts.txt),
  exact endpoints, the straight-line closed form, an independent Horner form,
  and the offsets-as-exclusive-scan identity.
* Planted mistakes: plausible errors, made on the CPU in copies of the
  oracle's output or of its formula, must fail these checks.
* Library routines: BFS levels and SSSP distances equal scipy.sparse.csgraph's
  unweighted shortest paths and Dijkstra on R-MAT digraphs.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from conftest import read_golden
from invariants import (bellman_ford, brute_force_hops, check_bfs_levels, check_sssp_dist,
                        csr_from_edges)
from paper_2201_02789_gb300 import gen


# ------------------------------------------------------------------------ BFS

@pytest.mark.parametrize("n", [3, 4])
def test_bfs_exhaustive_tiny_digraphs(n):
    pairs = [(u, v) for u in range(n) for v in range(n) if u != v]
    for mask in range(1 << len(pairs)):
        edges = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        row_ptr, col = csr_from_edges(n, edges) if edges else (np.zeros(n + 1, np.int32), np.zeros(0, np.int32))
        for src in range(n):
            got = oracle.bfs(row_ptr, col, src)
            assert list(got) == brute_force_hops(n, edges, src), (edges, src)


def _random_graph(rng, n, m, wmax=255, self_loops=True):
    us = rng.integers(0, n, m)
    vs = rng.integers(0, n, m)
    edges = [(int(u), int(v)) for u, v in zip(us, vs) if self_loops or u != v]
    ws = [int(x) for x in rng.integers(1, wmax + 1, len(edges))]
    return edges, ws


def test_bfs_random_vs_bruteforce():
    rng = np.random.default_rng(11)
    for _ in range(300):
        n = int(rng.integers(1, 65))
        m = int(rng.integers(0, 4 * n + 1))
        edges, _ = _random_graph(rng, n, m)
        if not edges:
            row_ptr, col = np.zeros(n + 1, np.int32), np.zeros(0, np.int32)
        else:
            row_ptr, col = csr_from_edges(n, edges)
        src = int(rng.integers(0, n))
        assert list(oracle.bfs(row_ptr, col, src)) == brute_force_hops(n, edges, src)


def test_bfs_hand_worked(tiny_graph):
    row_ptr, col, _, level, _ = tiny_graph
    np.testing.assert_array_equal(oracle.bfs(row_ptr, col, 0), level)


@pytest.mark.parametrize("which", ["bfs4k", "rmat14"])
def test_bfs_characterisation_full_size(which):
    g = gen.bfs4k() if which == "bfs4k" else gen.rmat(14, 16, seed=7)
    for src in [0, 1, g.n // 2]:
        lv = oracle.bfs(g.row_ptr, g.col, src)
        assert check_bfs_levels(g.row_ptr, g.col, src, lv) == []


def test_bfs_expand_matches_definition():
    g = gen.zipf_digraph(512, 2.1, 1, 128, seed=5)
    level = np.full(g.n, -1, np.int32)
    level[3] = 0
    frontier = np.array([3], np.int32)
    L = 0
    ref = brute_force_hops(g.n, list(zip(np.repeat(np.arange(g.n), np.diff(g.row_ptr)), g.col)), 3)
    while frontier.size:
        nxt = oracle.bfs_expand(g.row_ptr, g.col, frontier, L, level)
        assert len(set(nxt.tolist())) == nxt.size
        assert np.all(level[nxt] == L + 1)
        frontier, L = nxt, L + 1
    assert list(level) == ref


# ----------------------------------------------------------------------- SSSP

def test_sssp_random_vs_bellman_ford():
    rng = np.random.default_rng(12)
    for trial in range(300):
        n = int(rng.integers(1, 65))
        m = int(rng.integers(0, 5 * n + 1))
        wmax = 255 if trial % 3 else 2 ** 24
        edges, ws = _random_graph(rng, n, m, wmax=wmax)
        if not edges:
            row_ptr, col, w = np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint32)
        else:
            row_ptr, col, w = csr_from_edges(n, edges, ws)
        src = int(rng.integers(0, n))
        got = oracle.sssp(row_ptr, col, w, src)
        ref = bellman_ford(n, [(u, v, ww) for (u, v), ww in zip(edges, ws)], src)
        ref = [0xFFFFFFFF if d is None else d for d in ref]
        assert list(got) == ref


def test_sssp_hand_worked(tiny_graph):
    row_ptr, col, w, _, dist = tiny_graph
    np.testing.assert_array_equal(oracle.sssp(row_ptr, col, w, 0), dist)


def test_sssp_unit_weights_is_bfs():
    g = gen.rmat(12, 8, seed=9)
    ones = np.ones(g.m, np.uint32)
    lv = oracle.bfs(g.row_ptr, g.col, 0)
    d = oracle.sssp(g.row_ptr, g.col, ones, 0)
    expect = np.where(lv < 0, np.int64(0xFFFFFFFF), lv.astype(np.int64)).astype(np.uint32)
    np.testing.assert_array_equal(d, expect)


@pytest.mark.parametrize("which", ["bfs4k", "rmat14"])
def test_sssp_characterisation_full_size(which):
    g = gen.bfs4k() if which == "bfs4k" else gen.rmat(14, 16, seed=7)
    for src in [0, 5]:
        d = oracle.sssp(g.row_ptr, g.col, g.w, src)
        lv = oracle.bfs(g.row_ptr, g.col, src)
        assert check_sssp_dist(g.row_ptr, g.col, g.w, src, d, lv) == []


def test_sssp_relax_pass_definition():
    rng = np.random.default_rng(3)
    edges, ws = _random_graph(rng, 40, 160)
    row_ptr, col, w = csr_from_edges(40, edges, ws)
    din = np.full(40, 0xFFFFFFFF, np.uint32)
    din[[1, 2, 7]] = [0, 10, 3]
    fr = np.array([1, 2, 7, 9], np.int32)
    out = oracle.sssp_relax_pass(row_ptr, col, w, fr, din)
    ref = din.astype(np.int64).copy()
    for (u, v), ww in zip(edges, ws):
        if u in (1, 2, 7, 9) and din[u] != 0xFFFFFFFF:
            ref[v] = min(ref[v], int(din[u]) + ww)
    np.testing.assert_array_equal(out, ref.astype(np.uint32))


# --------------------------------------------------------------- tessellation

def test_bezier_counts_hand_derived():
    rows = read_golden("bezier_counts.txt")["rows"]
    assert len(rows) >= 12
    for r in rows:
        p = np.array([float(x) for x in r[:6]], np.float32)
        assert oracle.bezier_count(p) == int(r[6]), r


def test_bezier_endpoints_exact():
    ctrl = gen.bezier_curves(2000, seed=21)
    for c in range(0, 2000, 7):
        p = ctrl[c].reshape(6)
        N = oracle.bezier_count(p)
        assert 4 <= N <= 4096
        np.testing.assert_array_equal(oracle.bezier_point(p, N, 0), p[0:2].astype(np.float64))
        np.testing.assert_array_equal(oracle.bezier_point(p, N, N - 1), p[4:6].astype(np.float64))


def test_bezier_straight_line_closed_form():
    rng = np.random.default_rng(5)
    for _ in range(200):
        p0 = rng.integers(0, 1 << 23, 2) * 2.0 ** -24
        p2 = rng.integers(0, 1 << 23, 2) * 2.0 ** -24
        p1 = (p0 + p2) / 2                   # exact: multiples of 2^-25 fit float32
        p = np.array([p0[0], p0[1], p1[0], p1[1], p2[0], p2[1]], np.float32)
        N = oracle.bezier_count(p)
        assert N == 4                        # zero second difference
        for j in range(N):
            t = j / (N - 1)
            ref = p0 + t * (p2 - p0)
            np.testing.assert_allclose(oracle.bezier_point(p, N, j), ref, rtol=0, atol=4e-16)


def test_bezier_horner_form_agrees():
    ctrl = gen.bezier_curves(300, seed=22)
    worst = 0.0
    for c in range(300):
        p = ctrl[c].reshape(6).astype(np.float64)
        P0, P1, P2 = p[0:2], p[2:4], p[4:6]
        N = oracle.bezier_count(ctrl[c])
        for j in range(0, N, max(1, N // 17)):
            t = j / (N - 1)
            horner = P0 + t * (2.0 * (P1 - P0) + t * (P0 - 2.0 * P1 + P2))
            worst = max(worst, float(np.abs(horner - oracle.bezier_point(ctrl[c], N, j)).max()))
    assert worst <= 1e-14


def test_bezier_offsets_are_scan_of_counts():
    ctrl = gen.bezier_curves(5000, seed=23)
    off = oracle.bezier_offsets(ctrl)
    counts = np.array([oracle.bezier_count(ctrl[c]) for c in range(5000)])
    assert off[0] == 0
    np.testing.assert_array_equal(np.diff(off), counts)
    offs2, pts = oracle.bezier(ctrl[:50])
    assert pts.shape == (offs2[-1], 2)


def test_bezier_count_distribution_workload():
    """The 64K-curve workload: counts stay within [4, 4096] and are irregular."""
    off = oracle.bezier_offsets(gen.bt64k())
    counts = np.diff(off)
    assert counts.min() >= 4 and counts.max() <= 4096
    assert 3_000_000 < off[-1] < 12_000_000
    assert counts.max() > 10 * np.median(counts)


# ------------------------------------------------------------ planted mistakes

def test_planted_bfs_mistakes_are_caught():
    g = gen.bfs4k()
    lv = oracle.bfs(g.row_ptr, g.col, 0)
    reached = np.nonzero(lv > 1)[0]
    bad = lv.copy(); bad[reached[0]] += 1          # one level too deep
    assert check_bfs_levels(g.row_ptr, g.col, 0, bad)
    bad = lv.copy(); bad[reached[1]] -= 1          # one level too shallow
    assert check_bfs_levels(g.row_ptr, g.col, 0, bad)
    bad = lv.copy(); bad[reached[2]] = -1          # dropped vertex
    assert check_bfs_levels(g.row_ptr, g.col, 0, bad)
    assert check_bfs_levels(g.row_ptr, g.col, 1, lv)  # wrong source


def test_planted_sssp_mistakes_are_caught():
    g = gen.bfs4k()
    d = oracle.sssp(g.row_ptr, g.col, g.w, 0)
    lv = oracle.bfs(g.row_ptr, g.col, 0)
    r = np.nonzero((d > 0) & (d != 0xFFFFFFFF))[0]
    for delta in (+1, -1):
        bad = d.copy(); bad[r[3]] = np.uint32(int(bad[r[3]]) + delta)
        assert check_sssp_dist(g.row_ptr, g.col, g.w, 0, bad, lv)
    # a relaxation that drops the weight (d[u] instead of d[u]+w) is caught
    hop_only = np.where(lv < 0, np.int64(0xFFFFFFFF), lv.astype(np.int64)).astype(np.uint32)
    assert check_sssp_dist(g.row_ptr, g.col, g.w, 0, hop_only, lv)


def test_planted_count_mistakes_are_caught():
    """Floor instead of ceil, a dropped factor 2 in the second difference, or a
    transposed control point each change a hand-derived count."""
    rows = read_golden("bezier_counts.txt")["rows"]

    def count(p, mistake):
        x0, y0, x1, y1, x2, y2 = [float(v) for v in p]
        k = 1.0 if mistake == "drop2" else 2.0
        if mistake == "swap":
            x1, y1, x2, y2 = x2, y2, x1, y1
        sx, sy = (x0 - k * x1) + x2, (y0 - k * y1) + y2
        cx, cy = x2 - x0, y2 - y0
        s2, c2 = sx * sx + sy * sy, cx * cx + cy * cy
        if c2 == 0:
            return 4096 if s2 > 0 else 4
        v = math.sqrt(math.sqrt(s2) / math.sqrt(c2)) * 64
        t = math.floor(v) if mistake == "floor" else math.ceil(v)
        return int(min(max(t, 4), 4096))

    for mistake in ("floor", "drop2", "swap"):
        caught = sum(count(r[:6], mistake) != int(r[6]) for r in rows)
        assert caught >= 1, mistake
    assert all(count(r[:6], None) == int(r[6]) for r in rows)


# ------------------------------------------------------ library shortest paths

def _scipy_csr(g, weights):
    """The graph as a scipy CSR matrix with one entry per (u, v): parallel edges keep their
    least weight (scipy's graph routines do not take duplicate entries)."""
    sp = pytest.importorskip("scipy.sparse")
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr.astype(np.int64)))
    key = src.astype(np.int64) * g.n + g.col
    order = np.lexsort((weights, key))
    key, w = key[order], weights[order]
    first = np.ones(len(key), bool)
    first[1:] = key[1:] != key[:-1]
    key, w = key[first], w[first]
    return sp.csr_matrix((w.astype(np.float64), (key // g.n, key % g.n)), shape=(g.n, g.n))


@pytest.mark.parametrize("seed", [41, 42, 43])
def test_bfs_and_sssp_match_scipy_csgraph(seed):
    """BFS levels are unweighted shortest-path lengths and SSSP distances Dijkstra's, as
    scipy.sparse.csgraph computes them, on R-MAT digraphs with parallel edges and hubs."""
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    g = gen.rmat(11, 12, seed=seed)
    a = _scipy_csr(g, g.w)
    for src in (0, 17, g.n - 1):
        hops = csgraph.shortest_path(a, directed=True, unweighted=True, indices=src)
        want = np.where(np.isinf(hops), -1, hops).astype(np.int64)
        np.testing.assert_array_equal(oracle.bfs(g.row_ptr, g.col, src).astype(np.int64), want)
        dist = csgraph.dijkstra(a, directed=True, indices=src)
        want = np.where(np.isinf(dist), 0xFFFFFFFF, dist).astype(np.int64)
        np.testing.assert_array_equal(oracle.sssp(g.row_ptr, g.col, g.w, src).astype(np.int64), want)
