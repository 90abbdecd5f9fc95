"""Triangle counting, the second CSR workload: oracle pins (CPU) and GPU parity.

Pins tie the oracle to mathematics, not to itself: closed forms (complete
graphs K_n have C(n,3) triangles, cycles C_n with n > 3 none, the wheel with a
k-cycle rim k), an independent brute force over all vertex triples and the
trace(A^3)/6 identity on random small graphs, and planted mistakes (counting
ordered instead of increasing triples, or dropping the closing-edge test) that
the closed forms catch. The GPU path gets the degree orientation of each
graph, the oracle the symmetric graph itself, so the two also differ in input.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from invariants import csr_from_edges
from paper_2201_02789_gb300 import gen


def undirected(n, edges):
    """Symmetric sorted CSR of a simple undirected graph from an edge list."""
    es = sorted({(a, b) for u, v in edges if u != v for a, b in ((u, v), (v, u))})
    if not es:
        return gen.Csr(n, np.zeros(n + 1, np.int32), np.zeros(0, np.int32))
    rp, col, _ = csr_from_edges(n, es, [1] * len(es))
    return gen.Csr(n, rp, col)


def complete(n):
    return undirected(n, list(itertools.combinations(range(n), 2)))


def cycle(n):
    return undirected(n, [(i, (i + 1) % n) for i in range(n)])


def wheel(k):
    return undirected(k + 1, [(i, (i + 1) % k) for i in range(k)] + [(k, i) for i in range(k)])


def clique_with_pendants(k, npend, seed):
    """K_k plus npend vertices of degree 2, each joined to an adjacent pair of clique
    vertices (one triangle each): oriented edges between clique vertices join lists of
    similar length, a pendant's 2-entry list meets a clique vertex's long one."""
    r = gen.uniform_f64(seed, 901, 0, 2 * npend)
    edges = list(itertools.combinations(range(k), 2))
    for i in range(npend):
        a = int(r[2 * i] * k)
        b = (a + 1 + int(r[2 * i + 1] * (k - 1))) % k
        edges += [(k + i, a), (k + i, b)]
    return undirected(k + npend, edges)


def random_graph(n, p, seed):
    u = gen.uniform_f64(seed, 900, 0, n * n).reshape(n, n)
    return undirected(n, [(a, b) for a in range(n) for b in range(a + 1, n) if u[a, b] < p])


def brute(g):
    adj = np.zeros((g.n, g.n), bool)
    for u in range(g.n):
        adj[u, g.col[g.row_ptr[u]:g.row_ptr[u + 1]]] = True
    return sum(1 for a, b, c in itertools.combinations(range(g.n), 3) if adj[a, b] and adj[a, c] and adj[b, c])


def trace_a3(g):
    a = np.zeros((g.n, g.n), np.int64)
    for u in range(g.n):
        a[u, g.col[g.row_ptr[u]:g.row_ptr[u + 1]]] = 1
    return int(np.trace(a @ a @ a)) // 6


@pytest.mark.parametrize("n", range(1, 9))
def test_complete_graph_closed_form(n):
    assert oracle.triangles(complete(n).row_ptr, complete(n).col) == math.comb(n, 3)


@pytest.mark.parametrize("n", range(3, 10))
def test_cycles_and_wheels(n):
    c = cycle(n)
    assert oracle.triangles(c.row_ptr, c.col) == (1 if n == 3 else 0)
    w = wheel(n + 1)
    assert oracle.triangles(w.row_ptr, w.col) == n + 1


@pytest.mark.parametrize("seed", range(6))
def test_random_vs_brute_force_and_trace(seed):
    g = random_graph(14 + seed, 0.2 + 0.1 * seed, seed)
    t = oracle.triangles(g.row_ptr, g.col)
    assert t == brute(g) == trace_a3(g)


def test_lopsided_graph_takes_both_intersection_paths():
    """The oracle's count on the clique-with-pendants graph is its closed form, and its
    orientation has edges whose lists differ in length by more than 16x (the binary-search
    path) as well as edges with lists of similar length (the merge path)."""
    k, npend = 48, 400
    u = clique_with_pendants(k, npend, seed=35)
    assert oracle.triangles(u.row_ptr, u.col) == k * (k - 1) * (k - 2) // 6 + npend
    dag = gen.oriented_by_degree(u)
    deg = np.diff(dag.row_ptr.astype(np.int64))
    src = np.repeat(np.arange(dag.n), deg)
    lo, hi = np.minimum(deg[src], deg[dag.col]), np.maximum(deg[src], deg[dag.col])
    assert (hi > 16 * np.maximum(lo, 1)).any() and ((hi <= 16 * lo) & (lo >= 8)).any()


def test_orientation_keeps_every_edge_once():
    u = gen.undirected_simple(gen.rmat(10, 8, seed=31, weights=None))
    d = gen.oriented_by_degree(u)
    assert d.m * 2 == u.m
    src = np.repeat(np.arange(d.n), np.diff(d.row_ptr))
    pairs = {(min(a, b), max(a, b)) for a, b in zip(src, d.col)}
    assert len(pairs) == d.m and all(a != b for a, b in pairs)
    assert all(np.all(np.diff(d.col[d.row_ptr[v]:d.row_ptr[v + 1]]) > 0) for v in range(d.n))


def test_planted_mistakes_are_caught():
    """Counting every ordered triple (u, v, w) with the three edges present, or
    counting paths u - v - w without the closing edge, breaks the closed forms."""
    def ordered(g):
        adj = [set(g.col[g.row_ptr[u]:g.row_ptr[u + 1]]) for u in range(g.n)]
        return sum(1 for u in range(g.n) for v in adj[u] for w in adj[v] if w in adj[u])

    def open_paths(g):
        adj = [set(g.col[g.row_ptr[u]:g.row_ptr[u + 1]]) for u in range(g.n)]
        return sum(1 for u in range(g.n) for v in adj[u] if v > u for w in adj[v] if w > v)

    k5, c6 = complete(5), cycle(6)
    assert ordered(k5) != math.comb(5, 3)
    assert open_paths(c6) != 0
    assert oracle.triangles(k5.row_ptr, k5.col) == math.comb(5, 3)
    assert oracle.triangles(c6.row_ptr, c6.col) == 0


def test_oracle_rejects_unsorted_lists():
    g = complete(4)
    col = g.col.copy()
    col[0], col[1] = col[1], col[0]
    with pytest.raises(ValueError):
        oracle.triangles(g.row_ptr, col)


# --------------------------------------------------------------------- GPU parity

def _gpu_count(ctx, dag, cfg):
    import torch
    from gpu_util import DevGraph
    from paper_2201_02789_gb300 import nestpar as npb
    dg = DevGraph(dag)
    out = torch.full((1,), -1, dtype=torch.int64, device="cuda:0")
    _, st = npb.np_triangles(ctx.handle, dg.csr, out, cfg, stats=True)
    return int(out.item()), st


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2201_02789_gb300 import build as nbuild
    from paper_2201_02789_gb300 import nestpar as npb
    nbuild.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = npb.Context(0)
    yield c
    c.close()


def _tc_forms():
    from paper_2201_02789_gb300 import nestpar as npb
    out = [("nodp", npb.config("nodp")), ("cdp", npb.config("cdp")), ("tc", npb.config("tc"))]
    for gran in ("warp", "block", "multiblock", "grid_device", "grid_host"):
        for T, cf in ((1, 1), (8, 4), (64, 16)):
            out.append((f"{gran}-T{T}-C{cf}", npb.config("tca", granularity=gran, threshold=T, cfactor=cf,
                                                          group_blocks=3)))
    return out


TC_GRAPHS = {
    "k9": lambda: complete(9),
    "wheel40": lambda: wheel(40),
    "rmat12": lambda: gen.undirected_simple(gen.rmat(12, 16, seed=33, weights=None)),
    "road": lambda: gen.undirected_simple(gen.road_grid(40, 50, seed=6, weights=None)),
    "empty": lambda: undirected(5, []),
    # both intersection paths: merges between clique lists, binary searches from 2-entry lists
    "lopsided": lambda: clique_with_pendants(48, 400, seed=35),
}


@pytest.mark.gpu
@pytest.mark.parametrize("gname", list(TC_GRAPHS))
def test_gpu_triangles_all_forms(ctx, gname):
    u = TC_GRAPHS[gname]()
    ref = oracle.triangles(u.row_ptr, u.col)
    dag = gen.oriented_by_degree(u)
    for name, cfg in _tc_forms():
        got, st = _gpu_count(ctx, dag, cfg)
        assert got == ref, (gname, name)
        assert st["error"] == 0 and st["parents"] == dag.n and st["items"] == dag.m


@pytest.mark.gpu
def test_gpu_triangles_run_nested_subset(ctx):
    """np_run_nested over a parent subset adds that subset's triangles (at their
    lowest vertex in the orientation) into the caller's partial counts."""
    import torch
    from gpu_util import DevGraph
    from paper_2201_02789_gb300 import nestpar as npb
    u = gen.undirected_simple(gen.rmat(11, 12, seed=34, weights=None))
    dag = gen.oriented_by_degree(u)
    dg = DevGraph(dag)
    ids = np.arange(0, dag.n, 3, dtype=np.int32)
    # expected: triangles whose first (lowest-rank) vertex is in ids, counted on the CPU
    outs = [set(dag.col[dag.row_ptr[v]:dag.row_ptr[v + 1]]) for v in range(dag.n)]
    exp = sum(len(outs[p] & outs[v]) for p in ids for v in outs[p])
    parts = torch.zeros(npb.NP_TRI_SLOTS, dtype=torch.int64, device="cuda:0")
    ids_d = torch.from_numpy(ids).cuda()
    body = npb.np_body(kind=npb.NP_BODY_TRIANGLES, tri_counts=parts.data_ptr())
    npb.np_run_nested(ctx.handle, npb.np_parents(ids_d.data_ptr(), len(ids)), npb.NP_COUNT_CSR_DEGREE, dg.csr,
                      body, npb.config("tca", threshold=4))
    assert int(parts.sum().item()) == exp


@pytest.mark.gpu
@pytest.mark.slow
def test_gpu_triangles_full_size(ctx):
    """The benchmark's workload: R-MAT scale 17 made simple and undirected (3.7e6 edges,
    36,004,405 triangles)."""
    from paper_2201_02789_gb300 import nestpar as npb
    import bench
    u, dag = gen.tc_rmat17()
    ref = oracle.triangles(u.row_ptr, u.col)
    # the library default, the configuration bench.py times, and the No-CDP form
    for cfg in (npb.config("tca"), npb.config("tca", **bench.TUNED["tc-rmat17"]), npb.config("nodp")):
        got, st = _gpu_count(ctx, dag, cfg)
        assert got == ref and st["error"] == 0


def test_oracle_matches_networkx_triangles():
    """The triangle oracle against networkx's count (per-vertex triangles / 3) on simple
    undirected R-MAT graphs with hubs."""
    nx = pytest.importorskip("networkx")
    for seed in (36, 37):
        u = gen.undirected_simple(gen.rmat(10, 16, seed=seed, weights=None))
        G = nx.Graph()
        G.add_nodes_from(range(u.n))
        src = np.repeat(np.arange(u.n), np.diff(u.row_ptr))
        G.add_edges_from(zip(src.tolist(), u.col.tolist()))
        assert oracle.triangles(u.row_ptr, u.col) == sum(nx.triangles(G).values()) // 3
