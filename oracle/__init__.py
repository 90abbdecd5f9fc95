"""CPU oracle (TEST INFRASTRUCTURE ONLY).

Plain, slow, serial reference results for the nested-parallel workloads:
FIFO-queue BFS, binary-heap Dijkstra, FP64 quadratic Bezier tessellation and
triangle counting by its definition (every u < v < w pairwise adjacent),
in ``oracle.c`` (compiled with gcc, ``-O2 -ffp-contract=off``) behind ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package. It shares no code with the CUDA library and
never calls it; the seeded input generators (``paper_2201_02789_gb300.gen``)
are the only thing both sides use, and those hold none of the method.

Every function cites the definition it follows (see ``oracle.c``). Pins that
tie it to the mathematics rather than to itself live in
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` (gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_bfs.restype = ctypes.c_int64
            lib.oracle_bfs.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32, _i32p]
            lib.oracle_bfs_expand.restype = ctypes.c_int64
            lib.oracle_bfs_expand.argtypes = [_i32p, _i32p, _i32p, ctypes.c_int32, ctypes.c_int32,
                                              _i32p, _i32p]
            lib.oracle_sssp.restype = ctypes.c_int64
            lib.oracle_sssp.argtypes = [ctypes.c_int32, _i32p, _i32p, _u32p, ctypes.c_int32, _u32p]
            lib.oracle_sssp_relax_pass.restype = None
            lib.oracle_sssp_relax_pass.argtypes = [ctypes.c_int32, _i32p, _i32p, _u32p, _i32p,
                                                   ctypes.c_int32, _u32p, _u32p]
            lib.oracle_bezier_count.restype = ctypes.c_int32
            lib.oracle_bezier_count.argtypes = [_f32p]
            lib.oracle_bezier_point.restype = None
            lib.oracle_bezier_point.argtypes = [_f32p, ctypes.c_int32, ctypes.c_int32, _f64p]
            lib.oracle_bezier.restype = ctypes.c_int64
            lib.oracle_bezier.argtypes = [ctypes.c_int32, _f32p, _i32p, ctypes.c_void_p,
                                          ctypes.c_int64]
            lib.oracle_triangles.restype = ctypes.c_int64
            lib.oracle_triangles.argtypes = [ctypes.c_int32, _i32p, _i32p]
            _lib = lib
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def bfs(row_ptr, col, src: int) -> np.ndarray:
    """Hop levels from ``src`` (-1 = unreachable): FIFO-queue BFS."""
    row_ptr, col = _c(row_ptr, np.int32), _c(col, np.int32)
    n = row_ptr.shape[0] - 1
    level = np.empty(n, np.int32)
    rc = _load().oracle_bfs(n, row_ptr, col, int(src), level)
    if rc < 0:
        raise ValueError(f"oracle_bfs failed ({rc})")
    return level


def bfs_expand(row_ptr, col, frontier, level_L: int, level: np.ndarray):
    """One BFS expansion of ``frontier`` at level ``level_L``; updates ``level`` in place.
    Returns the newly reached vertices in order of first discovery."""
    row_ptr, col, frontier = _c(row_ptr, np.int32), _c(col, np.int32), _c(frontier, np.int32)
    assert level.dtype == np.int32 and level.flags.c_contiguous
    nxt = np.empty(level.shape[0], np.int32)
    k = _load().oracle_bfs_expand(row_ptr, col, frontier, frontier.shape[0], int(level_L), level, nxt)
    return nxt[:k].copy()


def sssp(row_ptr, col, w, src: int) -> np.ndarray:
    """Shortest-path distances (uint32, UINT32_MAX = unreachable): Dijkstra, binary heap."""
    row_ptr, col, w = _c(row_ptr, np.int32), _c(col, np.int32), _c(w, np.uint32)
    n = row_ptr.shape[0] - 1
    dist = np.empty(n, np.uint32)
    rc = _load().oracle_sssp(n, row_ptr, col, w, int(src), dist)
    if rc < 0:
        raise ValueError(f"oracle_sssp failed ({rc})")
    return dist


def sssp_relax_pass(row_ptr, col, w, frontier, dist_in) -> np.ndarray:
    """One synchronous relaxation of every out-edge of ``frontier`` (reads ``dist_in`` only)."""
    row_ptr, col, w = _c(row_ptr, np.int32), _c(col, np.int32), _c(w, np.uint32)
    frontier, dist_in = _c(frontier, np.int32), _c(dist_in, np.uint32)
    n = row_ptr.shape[0] - 1
    out = np.empty(n, np.uint32)
    _load().oracle_sssp_relax_pass(n, row_ptr, col, w, frontier, frontier.shape[0], dist_in, out)
    return out


def bezier_count(p) -> int:
    """Point count of one curve given as 6 floats (x0, y0, x1, y1, x2, y2)."""
    return int(_load().oracle_bezier_count(_c(np.asarray(p).reshape(6), np.float32)))


def bezier_point(p, N: int, j: int) -> np.ndarray:
    """Point ``j`` of ``N`` of one curve, FP64."""
    xy = np.empty(2, np.float64)
    _load().oracle_bezier_point(_c(np.asarray(p).reshape(6), np.float32), int(N), int(j), xy)
    return xy


def bezier_offsets(ctrl) -> np.ndarray:
    """Curve-order exclusive scan of the point counts, int32[ncurves + 1]."""
    ctrl = _c(ctrl, np.float32)
    nc = ctrl.shape[0]
    offsets = np.empty(nc + 1, np.int32)
    rc = _load().oracle_bezier(nc, ctrl.reshape(-1), offsets, None, 0)
    if rc < 0:
        raise ValueError(f"oracle_bezier failed ({rc})")
    return offsets


def bezier(ctrl) -> tuple[np.ndarray, np.ndarray]:
    """Offsets int32[ncurves + 1] and FP64 points [total, 2] of a tessellation."""
    ctrl = _c(ctrl, np.float32)
    nc = ctrl.shape[0]
    offsets = bezier_offsets(ctrl)
    total = int(offsets[-1])
    pts = np.empty((max(total, 1), 2), np.float64)
    rc = _load().oracle_bezier(nc, ctrl.reshape(-1), offsets, pts.ctypes.data_as(ctypes.c_void_p), total)
    if rc < 0:
        raise ValueError(f"oracle_bezier failed ({rc})")
    return offsets, pts[:total]


def triangles(row_ptr, col) -> int:
    """Triangles of a simple undirected graph (symmetric CSR, sorted adjacency lists)."""
    rp = _c(row_ptr, np.int32)
    c = _c(col, np.int32) if len(col) else np.zeros(1, np.int32)
    r = _load().oracle_triangles(int(rp.shape[0] - 1), rp, c)
    if r < 0:
        raise ValueError("adjacency lists must be strictly increasing")
    return int(r)
