"""Independent checks that pin BFS/SSSP/tessellation results to the mathematics.

None of these reuse the oracle: they are textbook brute force (tiny inputs) or
characterisations that hold at any size and determine the answer uniquely.

BFS on a digraph (the "|level(u) - level(v)| <= 1 on every edge" test holds only
for undirected graphs, so the directed form is used): with level(src) = 0,
  (a) every edge u->v with u reached has v reached and level(v) <= level(u) + 1;
  (b) every reached v != src has an in-edge u->v with level(u) = level(v) - 1.
(a) implies level(v) <= hop(v) by induction along a shortest path, and (b)
implies level(v) >= hop(v) by induction on level; together level == hop.

SSSP: with dist(src) = 0,
  (a) every edge u->v with u reached has dist(v) <= dist(u) + w (in uint64);
  (b) every reached v != src has an in-edge with dist(v) = dist(u) + w;
  (c) reached exactly when BFS-reachable.
(a) gives dist <= true distance along any path, (b) gives a path achieving
dist(v) (weights >= 1 make the tight in-edges acyclic), so dist == distance.
"""
from __future__ import annotations

import numpy as np

UNREACHED_DIST = np.uint32(0xFFFFFFFF)


def edge_sources(row_ptr: np.ndarray) -> np.ndarray:
    n = row_ptr.shape[0] - 1
    return np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr.astype(np.int64)))


def check_bfs_levels(row_ptr, col, src: int, level) -> list[str]:
    """Return a list of violated properties (empty = level is the exact hop distance)."""
    row_ptr = np.asarray(row_ptr, np.int64)
    col = np.asarray(col, np.int64)
    level = np.asarray(level, np.int64)
    n = row_ptr.shape[0] - 1
    errs = []
    if level.shape != (n,):
        return [f"shape {level.shape} != ({n},)"]
    if level[src] != 0:
        errs.append(f"level[src]={level[src]}")
    if np.any(level < -1):
        errs.append("level below -1")
    u = edge_sources(row_ptr)
    lu, lv = level[u], level[col]
    reached_u = lu >= 0
    bad_a = reached_u & ((lv < 0) | (lv > lu + 1))
    if bad_a.any():
        k = int(np.nonzero(bad_a)[0][0])
        errs.append(f"edge {u[k]}->{col[k]}: level {lu[k]} -> {lv[k]}")
    tight = reached_u & (lv == lu + 1)
    has_parent = np.zeros(n, bool)
    has_parent[col[tight]] = True
    need = (level > 0)
    missing = need & ~has_parent
    if missing.any():
        errs.append(f"vertex {int(np.nonzero(missing)[0][0])} has no parent one level up")
    others_zero = (level == 0)
    others_zero[src] = False
    if others_zero.any():
        errs.append("a vertex other than src has level 0")
    return errs


def check_sssp_dist(row_ptr, col, w, src: int, dist, reach_level=None) -> list[str]:
    """Return violated properties (empty = dist is exactly the shortest-path distance)."""
    row_ptr = np.asarray(row_ptr, np.int64)
    col = np.asarray(col, np.int64)
    w = np.asarray(w, np.uint64)
    dist = np.asarray(dist, np.uint32)
    n = row_ptr.shape[0] - 1
    errs = []
    if dist.shape != (n,):
        return [f"shape {dist.shape} != ({n},)"]
    if dist[src] != 0:
        errs.append(f"dist[src]={dist[src]}")
    d = dist.astype(np.uint64)
    reached = dist != UNREACHED_DIST
    u = edge_sources(row_ptr)
    ru = reached[u]
    du = d[u]
    dv = d[col]
    rv = reached[col]
    cand = du + w
    bad_a = ru & (~rv | (dv > cand))
    if bad_a.any():
        k = int(np.nonzero(bad_a)[0][0])
        errs.append(f"edge {u[k]}->{col[k]} w={w[k]}: {du[k]} + w < {dv[k]} or target unreached")
    tight = ru & rv & (dv == cand)
    has_parent = np.zeros(n, bool)
    has_parent[col[tight]] = True
    need = reached.copy()
    need[src] = False
    missing = need & ~has_parent
    if missing.any():
        errs.append(f"vertex {int(np.nonzero(missing)[0][0])} has no tight in-edge")
    if reach_level is not None:
        rl = np.asarray(reach_level) >= 0
        if not np.array_equal(rl, reached):
            errs.append("reached set differs from BFS reachability")
    return errs


def brute_force_hops(n: int, edges: list[tuple[int, int]], src: int) -> list[int]:
    """Hop distances by relaxation to a fixed point (at most n rounds)."""
    level = [-1] * n
    level[src] = 0
    for _ in range(n):
        changed = False
        for u, v in edges:
            if level[u] >= 0 and (level[v] < 0 or level[v] > level[u] + 1):
                level[v] = level[u] + 1
                changed = True
        if not changed:
            break
    return level


def bellman_ford(n: int, edges: list[tuple[int, int, int]], src: int) -> list[int]:
    """Shortest distances by n-1 rounds of relaxing every edge (None = unreachable)."""
    INF = None
    d = [INF] * n
    d[src] = 0
    for _ in range(max(n - 1, 1)):
        for u, v, w in edges:
            if d[u] is not None and (d[v] is None or d[u] + w < d[v]):
                d[v] = d[u] + w
    return d


def csr_from_edges(n: int, edges, weights=None):
    """CSR arrays (row_ptr, col[, w]) from an edge list, sorted stably by source."""
    order = sorted(range(len(edges)), key=lambda i: edges[i][0])
    row_ptr = np.zeros(n + 1, np.int32)
    for u, _ in (e[:2] for e in edges):
        row_ptr[u + 1] += 1
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    col = np.array([edges[i][1] for i in order], np.int32).reshape(-1)
    if weights is None:
        return row_ptr, col
    w = np.array([weights[i] for i in order], np.uint32).reshape(-1)
    return row_ptr, col, w


def bezier_tolerance_ok(got, ref, rel: float = 1e-5) -> tuple[bool, float]:
    """|g - r| <= rel * max(|r|, 1) element-wise; returns (ok, worst ratio)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.maximum(np.abs(ref), 1.0)
    ratio = np.abs(got - ref) / (rel * scale)
    worst = float(ratio.max()) if ratio.size else 0.0
    return worst <= 1.0, worst


def bezier_relative_error(got, ref, floor: float = 1e-3) -> float:
    """The largest strict relative error |g - r| / |r| over coordinates with |r| >= floor."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    big = np.abs(ref) >= floor
    return float((np.abs(got - ref)[big] / np.abs(ref[big])).max()) if big.any() else 0.0
