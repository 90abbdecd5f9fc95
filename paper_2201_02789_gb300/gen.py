"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random inputs; it contains none of the method's
arithmetic (no traversal, no child counts, no tessellation). It is shared by
the CUDA path's tests/bench and by the CPU oracle's tests: the two sides
share nothing else.

Generator: splitmix64 used as a counter-based generator. Output ``i`` of
stream ``s`` under seed ``seed`` is ``mix(key(seed, s) + (i + 1) * GAMMA)``
where ``mix`` is the splitmix64 finaliser (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014). Everything is
vectorised in numpy uint64 arithmetic, so the same seed gives the same bytes
on x86-64 and aarch64.

Workload recipes (the paper's datasets are not available; these stand in):

* ``zipf_digraph``: out-degree k ~ P(k) proportional to k^-alpha on
  [kmin, kmax] by inverse CDF; neighbours uniform without replacement,
  excluding the vertex itself; adjacency sorted ascending (stands in for the
  CNR-style skewed web graph of the paper's Table "Benchmarks and Datasets").
* ``rmat``: R-MAT (Chakrabarti et al., SDM 2004) with the Graph500
  probabilities a,b,c,d; per level the destination bit is set in quadrants b
  and d, the source bit in c and d; self-loops are redrawn, duplicates kept,
  no vertex permutation (vertex 0 is the top hub); CSR sorted by (src, dst).
  Stands in for KRON (kron_g500-simple-logn16).
* ``bezier_curves``: quadratic Bezier control points uniform in [0,1]^2 as
  float32 multiples of 2^-24 (stands in for the T*-C* line sets).
* ``road_grid``: a 2-D grid digraph with degree <= 8, standing in for the
  low-nested-parallelism road graph (USA-road-d.NY) of the evaluation.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1

# named streams (documented constants; any fixed distinct values would do)
S_DEGREE, S_NEIGH, S_RMAT, S_WEIGHT, S_BEZIER, S_BATCH, S_SOURCE, S_ROAD = range(1, 9)


def _mix(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser on a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _mix_int(z: int) -> int:
    z &= _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    """Key of stream ``stream`` under ``seed``."""
    return _mix_int(((seed & 0xFFFFFFFF) << 32) ^ (stream & 0xFFFFFFFF) ^ 0xD1B54A32D192ED03)


def u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of a stream, as uint64."""
    key = np.uint64(stream_key(seed, stream))
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + idx * GAMMA)


def uniform_f64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (u64(seed, stream, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_f32(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Uniform float32 in [0, 1): multiples of 2^-24 (exact in float32)."""
    v = (u64(seed, stream, start, count) >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)
    return v.astype(np.float32)


def uniform_int(seed: int, stream: int, start: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi] by multiply-shift of the top 32 bits."""
    span = np.uint64(hi - lo + 1)
    top = u64(seed, stream, start, count) >> np.uint64(32)
    with np.errstate(over="ignore"):
        return ((top * span) >> np.uint64(32)).astype(np.int64) + lo


@dataclass
class Csr:
    """CSR digraph: row_ptr int32[n+1], col int32[m], optional weights uint32[m]."""
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray | None = None

    @property
    def m(self) -> int:
        return int(self.col.shape[0])


def _csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    key = src.astype(np.int64) * np.int64(n) + dst.astype(np.int64)
    key.sort(kind="stable")
    s = (key // n).astype(np.int64)
    d = (key % n).astype(np.int32)
    counts = np.bincount(s, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2 ** 31:
        raise ValueError("edge count exceeds int32 CSR")
    return row_ptr.astype(np.int32), d


def zipf_degrees(n: int, alpha: float, kmin: int, kmax: int, seed: int) -> np.ndarray:
    """Out-degrees with P(k) proportional to k^-alpha on [kmin, kmax] (inverse CDF)."""
    ks = np.arange(kmin, kmax + 1, dtype=np.float64)
    p = ks ** (-alpha)
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    u = uniform_f64(seed, S_DEGREE, 0, n)
    idx = np.searchsorted(cdf, u, side="right")
    idx = np.minimum(idx, len(ks) - 1)
    return (kmin + idx).astype(np.int64)


def zipf_digraph(n: int = 4096, alpha: float = 2.1, kmin: int = 1, kmax: int = 1024,
                 seed: int = 1, weights: tuple[int, int] | None = (1, 255)) -> Csr:
    """Power-law digraph: Zipf out-degrees, neighbours uniform without replacement, no self-loops."""
    kmax = min(kmax, n - 1)
    deg = zipf_degrees(n, alpha, kmin, kmax, seed)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    col = np.empty(int(row_ptr[-1]), dtype=np.int32)
    for u in range(n):
        k = int(deg[u])
        # random keys over the n-1 candidates (all vertices except u); the k smallest keys win
        keys = u64(seed, S_NEIGH, u * n, n - 1)
        pick = np.argpartition(keys, k - 1)[:k] if k < n - 1 else np.arange(n - 1)
        cand = pick.astype(np.int64)
        cand = cand + (cand >= u)          # skip u itself
        col[row_ptr[u]:row_ptr[u + 1]] = np.sort(cand).astype(np.int32)
    g = Csr(n, row_ptr.astype(np.int32), col)
    if weights is not None:
        g.w = uniform_int(seed, S_WEIGHT, 0, g.m, weights[0], weights[1]).astype(np.uint32)
    return g


_RMAT_Q = 16  # bits of resolution per quadrant draw


def _rmat_edges(scale: int, count: int, first: int, seed: int, stream: int,
                a: float, b: float, c: float) -> tuple[np.ndarray, np.ndarray]:
    """Draw edges ``first .. first+count-1`` of an R-MAT stream (scale levels each).

    Level ``l`` of edge ``e`` uses 16-bit field ``l % 4`` (least significant first) of
    output ``e * ceil(scale/4) + l // 4`` of the stream.
    """
    ta, tb, tc = _rmat_thresholds(a, b, c)
    words = (scale + 3) // 4                       # four 16-bit draws per 64-bit output
    raw = u64(seed, stream, first * words, count * words)
    # 16-bit fields in significance order, independent of host byte order
    raw = np.ascontiguousarray(raw.reshape(count, words).T)      # [words, count]
    src = np.zeros(count, dtype=np.uint32)
    dst = np.zeros(count, dtype=np.uint32)
    for lvl in range(scale):
        r = ((raw[lvl // 4] >> np.uint64(16 * (lvl % 4))) & np.uint64(0xFFFF)).astype(np.uint16)
        shift = np.uint32(scale - 1 - lvl)
        src |= (r >= tb).astype(np.uint32) << shift                       # quadrants c, d
        dst |= (((r >= ta) & (r < tb)) | (r >= tc)).astype(np.uint32) << shift  # quadrants b, d
    return src.astype(np.int64), dst.astype(np.int64)


_NATIVE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libnpgen.so")
_native_lib = None


def native_available() -> bool:
    """True when the C twin of the R-MAT recipe (gen_native.c) has been built."""
    global _native_lib
    if _native_lib is None and os.path.exists(_NATIVE_PATH):
        L = ctypes.CDLL(_NATIVE_PATH)
        L.npgen_rmat.argtypes = [ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                 ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                 ctypes.c_uint32]
        L.npgen_rmat.restype = ctypes.c_int
        _native_lib = L
    return _native_lib is not None


def _rmat_thresholds(a: float, b: float, c: float) -> tuple[int, int, int]:
    ta = round(a * (1 << _RMAT_Q))
    tb = ta + round(b * (1 << _RMAT_Q))
    tc = tb + round(c * (1 << _RMAT_Q))
    return ta, tb, tc


def rmat_native(scale: int, nv: int, me: int, a: float, b: float, c: float, seed: int,
                weights: tuple[int, int] | None) -> Csr:
    """gen.rmat through the C twin (same bytes; releases the GIL, so instances can be drawn in threads)."""
    if not native_available():
        raise RuntimeError("libnpgen.so is not built (paper_2201_02789_gb300.build.build_gen())")
    ta, tb, tc = _rmat_thresholds(a, b, c)
    row_ptr = np.empty(nv + 1, dtype=np.int32)
    col = np.empty(max(me, 1), dtype=np.int32)
    w = np.empty(max(me, 1), dtype=np.uint32) if weights is not None else None
    rc = _native_lib.npgen_rmat(scale, nv, me, seed & ((1 << 64) - 1), S_RMAT, S_WEIGHT, ta, tb, tc,
                                row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data if w is not None else None,
                                weights[0] if weights else 0, weights[1] if weights else 0)
    if rc != 0:
        raise RuntimeError("native R-MAT generation failed")
    g = Csr(nv, row_ptr, col[:me])
    if w is not None:
        g.w = w[:me]
    return g


def rmat(scale: int = 20, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 2, n: int | None = None, m: int | None = None,
         weights: tuple[int, int] | None = (1, 255), chunk: int = 1 << 21, native: bool | None = None) -> Csr:
    """R-MAT digraph. Self-loops (and endpoints >= n when n < 2^scale) are redrawn.

    ``native`` None uses the C twin when it is built (identical output), True requires it, False forbids it."""
    nv = (1 << scale) if n is None else n
    if nv > (1 << scale):
        raise ValueError("n exceeds 2^scale")
    me = edge_factor * nv if m is None else m
    if native or (native is None and native_available()):
        return rmat_native(scale, nv, me, a, b, c, seed, weights)
    src = np.empty(me, dtype=np.int64)
    dst = np.empty(me, dtype=np.int64)
    for lo in range(0, me, chunk):
        cnt = min(chunk, me - lo)
        s, d = _rmat_edges(scale, cnt, lo, seed, S_RMAT, a, b, c)
        src[lo:lo + cnt] = s
        dst[lo:lo + cnt] = d
    attempt = 0
    while True:
        bad = np.nonzero((src == dst) | (src >= nv) | (dst >= nv))[0]
        if bad.size == 0:
            break
        attempt += 1
        if attempt > 10000:
            raise RuntimeError("R-MAT redraw did not converge")
        # redraws come from stream S_RMAT + 1000*attempt, indexed by edge id
        s, d = _rmat_edges(scale, bad.size, 0, seed ^ (attempt * 0x51ED27), S_RMAT + 1000 * attempt, a, b, c)
        src[bad] = s
        dst[bad] = d
    row_ptr, col = _csr_from_edges(nv, src, dst)
    g = Csr(nv, row_ptr, col)
    if weights is not None:
        g.w = uniform_int(seed, S_WEIGHT, 0, g.m, weights[0], weights[1]).astype(np.uint32)
    return g


def road_grid(rows: int, cols: int, seed: int = 6, weights: tuple[int, int] | None = (1, 255)) -> Csr:
    """Grid digraph: each cell links to its 4 axis neighbours and, with probability 1/2 each,
    to its 4 diagonal neighbours (out-degree 2..8, mean about 5.6)."""
    n = rows * cols
    r = np.arange(n, dtype=np.int64) // cols
    cc = np.arange(n, dtype=np.int64) % cols
    srcs, dsts = [], []
    offs = [(-1, 0), (1, 0), (0, -1), (0, 1), (-1, -1), (-1, 1), (1, -1), (1, 1)]
    coin = u64(seed, S_ROAD, 0, n) if n else np.zeros(0, np.uint64)
    for k, (dr, dc) in enumerate(offs):
        rr, c2 = r + dr, cc + dc
        ok = (rr >= 0) & (rr < rows) & (c2 >= 0) & (c2 < cols)
        if k >= 4:
            ok &= ((coin >> np.uint64(k)) & np.uint64(1)).astype(bool)
        srcs.append(np.nonzero(ok)[0])
        dsts.append((rr * cols + c2)[ok])
    src = np.concatenate(srcs)
    dst = np.concatenate(dsts)
    row_ptr, col = _csr_from_edges(n, src, dst)
    g = Csr(n, row_ptr, col)
    if weights is not None:
        g.w = uniform_int(seed, S_WEIGHT, 0, g.m, weights[0], weights[1]).astype(np.uint32)
    return g


def bezier_curves(ncurves: int = 65536, seed: int = 3) -> np.ndarray:
    """Quadratic Bezier control points, float32 [ncurves, 3, 2], uniform in [0,1)^2."""
    return uniform_f32(seed, S_BEZIER, 0, ncurves * 6).reshape(ncurves, 3, 2)


@dataclass
class BatchInstance:
    scale: int
    n: int
    edge_factor: int
    seed: int


def batch_specs(count: int = 512, seed: int = 4, log2_lo: float = 10.0, log2_hi: float = 20.0,
                ef_lo: int = 8, ef_hi: int = 32) -> list[BatchInstance]:
    """Instance sizes for the batched workload: n log-uniform in [2^lo, 2^hi], edge factor uniform."""
    u = uniform_f64(seed, S_BATCH, 0, count)
    efs = uniform_int(seed, S_BATCH + 100, 0, count, ef_lo, ef_hi)
    out = []
    for i in range(count):
        n = int(math.floor(2.0 ** (log2_lo + (log2_hi - log2_lo) * float(u[i]))))
        n = max(n, 2)
        scale = max(1, math.ceil(math.log2(n)))
        out.append(BatchInstance(scale, n, int(efs[i]), seed * 1000003 + i))
    return out


def batch_instance(spec: BatchInstance, weights: tuple[int, int] | None = (1, 255),
                   native: bool | None = None) -> Csr:
    """One batched-workload graph: R-MAT at scale ceil(log2 n) on n vertices, m = edge_factor * n."""
    return rmat(spec.scale, spec.edge_factor, seed=spec.seed, n=spec.n, weights=weights, native=native)


def batch_graphs(specs: list[BatchInstance], weights: tuple[int, int] | None = (1, 255),
                 threads: int | None = None) -> list[Csr]:
    """All instances of a batch, drawn in parallel threads by the C twin when it is built."""
    if not native_available():
        return [batch_instance(s, weights, native=False) for s in specs]
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 4) as ex:
        return list(ex.map(lambda s: batch_instance(s, weights, native=True), specs))


def random_sources(g: Csr, count: int, seed: int) -> np.ndarray:
    """Sources uniform over the vertices with out-degree > 0."""
    deg = np.diff(g.row_ptr.astype(np.int64))
    cand = np.nonzero(deg > 0)[0]
    idx = uniform_int(seed, S_SOURCE, 0, count, 0, len(cand) - 1)
    return cand[idx].astype(np.int32)


def undirected_simple(g: Csr) -> Csr:
    """The simple undirected graph under a digraph: both directions of every
    edge, self-loops and duplicates dropped, adjacency lists sorted (no weights)."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr.astype(np.int64)))
    dst = g.col.astype(np.int64)
    keep = src != dst
    a = np.concatenate([src[keep], dst[keep]])
    b = np.concatenate([dst[keep], src[keep]])
    key = np.unique(a * g.n + b)
    row_ptr, col = _csr_from_edges(g.n, key // g.n, key % g.n)
    return Csr(g.n, row_ptr, col)


def oriented_by_degree(u: Csr) -> Csr:
    """An acyclic orientation of a simple undirected graph: each edge points from
    the endpoint of lower (degree, id) to the other; out-lists sorted by id. Input
    preparation for triangle counting (keeps high-degree vertices' out-lists short)."""
    deg = np.diff(u.row_ptr.astype(np.int64))
    src = np.repeat(np.arange(u.n, dtype=np.int64), deg)
    dst = u.col.astype(np.int64)
    rank = np.empty(u.n, dtype=np.int64)
    rank[np.lexsort((np.arange(u.n), deg))] = np.arange(u.n)
    fwd = rank[src] < rank[dst]
    row_ptr, col = _csr_from_edges(u.n, src[fwd], dst[fwd])
    return Csr(u.n, row_ptr, col)


# ---- named workloads ------------------------------------------------------------------

def bfs4k() -> Csr:
    """BFS workload: 4096 vertices, Zipf(2.1) out-degrees on [1, 1024], seed 1."""
    return zipf_digraph(4096, 2.1, 1, 1024, seed=1)


def rmat20() -> Csr:
    """SSSP/BFS workload: R-MAT scale 20, edge factor 16, (.57,.19,.19,.05), weights 1..255, seed 2."""
    return rmat(20, 16, 0.57, 0.19, 0.19, seed=2)


def tc_rmat17() -> tuple[Csr, Csr]:
    """Triangle-counting workload: the simple undirected graph under R-MAT scale 17, edge
    factor 16 (Graph500 probabilities, seed 7), and its degree orientation."""
    u = undirected_simple(rmat(17, 16, seed=7, weights=None))
    return u, oriented_by_degree(u)


def bt64k() -> np.ndarray:
    """Tessellation workload: 65536 quadratic curves in [0,1)^2, seed 3."""
    return bezier_curves(65536, seed=3)
