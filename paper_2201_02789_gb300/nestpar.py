"""Python binding of the C ABI in ``include/nestpar.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls; all work runs
in the CUDA library ``_build/libnestpar.so``. There is no fallback: if the
library is not built, or a call fails, an exception says so. PyTorch tensors
are accepted for device (or host) buffers and only their pointers are passed;
streams are ``torch.cuda.Stream`` objects or raw ``cudaStream_t`` integers.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# NESTPAR_LIB selects another build of the same library (tuning variants)
LIB_PATH = os.environ.get("NESTPAR_LIB") or os.path.join(_PKG, "_build", "libnestpar.so")

NP_OK, NP_ERR_INVALID, NP_ERR_CUDA, NP_ERR_NOMEM, NP_ERR_CAPACITY, NP_ERR_LAUNCH, NP_ERR_TIMEOUT, \
    NP_ERR_UNSUPPORTED = range(8)
NP_VARIANT_NODP, NP_VARIANT_CDP = 0, 1
NP_GRAN_NONE, NP_GRAN_WARP, NP_GRAN_BLOCK, NP_GRAN_MULTIBLOCK, NP_GRAN_GRID_DEVICE, NP_GRAN_GRID_HOST = range(6)
NP_SCAN_LOOKBACK, NP_SCAN_ATOMIC = 0, 1
NP_DRIVER_AUTO, NP_DRIVER_HOST, NP_DRIVER_CHUNK, NP_DRIVER_WHILE, NP_DRIVER_PERSISTENT = range(5)
NP_SERIAL_SPREAD, NP_SERIAL_PACKED, NP_SERIAL_BLOCK = 0, 1, 2
NP_SMALL_PARENTS_MAX = 2048
NP_COUNT_CSR_DEGREE, NP_COUNT_BEZIER = 0, 1
NP_BODY_BFS_VISIT, NP_BODY_SSSP_RELAX, NP_BODY_BEZIER_EVAL, NP_BODY_TRIANGLES = 0, 1, 2, 3
NP_TRI_SLOTS = 256
NP_BATCH_BFS, NP_BATCH_SSSP = 0, 1
INT32_MAX = 2 ** 31 - 1

GRAN_NAMES = {"none": NP_GRAN_NONE, "warp": NP_GRAN_WARP, "block": NP_GRAN_BLOCK,
              "multiblock": NP_GRAN_MULTIBLOCK, "grid_device": NP_GRAN_GRID_DEVICE,
              "grid_host": NP_GRAN_GRID_HOST}


class NestparError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {np_status_string(status)} (status {status})")


class np_config(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("threshold", ctypes.c_int32), ("cfactor", ctypes.c_int32),
                ("granularity", ctypes.c_int32), ("group_blocks", ctypes.c_int32),
                ("agg_threshold", ctypes.c_int32), ("child_block", ctypes.c_int32),
                ("parent_block", ctypes.c_int32), ("scan", ctypes.c_int32), ("driver", ctypes.c_int32),
                ("unroll", ctypes.c_int32), ("parent_grid", ctypes.c_int32),
                ("serial", ctypes.c_int32), ("small_parents", ctypes.c_int32),
                ("sweep_parents", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]

    def replace(self, **kw) -> "np_config":
        c = np_config()
        ctypes.pointer(c)[0] = self
        for k, v in kw.items():
            if k == "granularity" and isinstance(v, str):
                v = GRAN_NAMES[v]
            setattr(c, k, v)
        return c

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class np_csr(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("weights", ctypes.c_void_p),
                ("n", ctypes.c_int32), ("m", ctypes.c_int64)]


class np_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in
                ("levels", "parents", "serial_parents", "launch_parents", "device_launches",
                 "aggregated_grids", "child_blocks", "items", "pushes", "launch_failures", "timeouts",
                 "child_items", "graph_iterations")] + \
               [("error", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_ if f != "reserved"}


NP_PROFILE_LEVELS = 64


class np_profile(ctypes.Structure):
    _fields_ = [("parent_ms", ctypes.c_double), ("child_ms", ctypes.c_double), ("other_ms", ctypes.c_double),
                ("parent_launches", ctypes.c_int64), ("child_launches", ctypes.c_int64),
                ("other_launches", ctypes.c_int64), ("longest_level_ms", ctypes.c_double),
                ("levels", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("level_parents", ctypes.c_int32 * NP_PROFILE_LEVELS),
                ("level_parent_ms", ctypes.c_double * NP_PROFILE_LEVELS),
                ("level_child_ms", ctypes.c_double * NP_PROFILE_LEVELS)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_[:8]}
        n = min(self.levels, NP_PROFILE_LEVELS)
        d["level_parents"] = list(self.level_parents[:n])
        d["level_parent_ms"] = list(self.level_parent_ms[:n])
        d["level_child_ms"] = list(self.level_child_ms[:n])
        return d


class np_parents(ctypes.Structure):
    _fields_ = [("ids", ctypes.c_void_p), ("count", ctypes.c_int32)]


class np_body(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("next_level", ctypes.c_int32), ("iteration", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("level", ctypes.c_void_p), ("dist", ctypes.c_void_p),
                ("stamp", ctypes.c_void_p), ("next", ctypes.c_void_p), ("next_count", ctypes.c_void_p),
                ("ctrl", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("points", ctypes.c_void_p),
                ("cap", ctypes.c_int64), ("tri_counts", ctypes.c_void_p)]


class np_batch_options(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("class_log2_width", ctypes.c_int32), ("max_group_edges", ctypes.c_int64),
                ("config", np_config)]


class np_batch_class(ctypes.Structure):
    _fields_ = [("log2_lo", ctypes.c_int32), ("instances", ctypes.c_int32), ("groups", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("vertices", ctypes.c_int64), ("edges", ctypes.c_int64),
                ("config", np_config), ("tuned_ms", ctypes.c_double), ("candidates", ctypes.c_int32),
                ("reserved2", ctypes.c_int32), ("device_launch_ms", ctypes.c_double),
                ("device_launch_granularity", ctypes.c_int32), ("device_launch_threshold", ctypes.c_int32)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved") and k != "config"}
        d["config"] = self.config.as_dict()
        return d


class np_server_options(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_uint64), ("max_slots", ctypes.c_int32),
                ("levels_per_step", ctypes.c_int32), ("bfs_config", np_config), ("sssp_config", np_config)]


class np_query_info(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("graph", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("slot", ctypes.c_int32), ("submit_step", ctypes.c_int64), ("admit_step", ctypes.c_int64),
                ("finish_step", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None
_VP, _I32, _I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
_SIGS = {
    "np_config_default": [ctypes.POINTER(np_config)],
    "np_create": [ctypes.POINTER(ctypes.c_void_p), _I32],
    "np_destroy": [_VP],
    "np_workspace_size": [_I64, ctypes.POINTER(np_config), ctypes.POINTER(ctypes.c_size_t)],
    "np_sync": [_VP, _VP, ctypes.POINTER(np_stats)],
    "np_bfs": [_VP, ctypes.POINTER(np_csr), _I32, _VP, ctypes.POINTER(np_config), _VP, ctypes.POINTER(np_stats)],
    "np_sssp": [_VP, ctypes.POINTER(np_csr), _I32, _VP, ctypes.POINTER(np_config), _VP, ctypes.POINTER(np_stats)],
    "np_bezier": [_VP, _VP, _I32, _VP, _VP, _I64, ctypes.POINTER(np_config), _VP, ctypes.POINTER(np_stats)],
    "np_run_nested": [_VP, ctypes.POINTER(np_parents), _I32, ctypes.POINTER(np_csr), ctypes.POINTER(np_body),
                      ctypes.POINTER(np_config), _VP, ctypes.POINTER(np_stats)],
    "np_bfs_host": [_VP, _I32, _I64, _VP, _VP, _I32, _VP, ctypes.POINTER(np_config), _VP,
                    ctypes.POINTER(np_stats)],
    "np_sssp_host": [_VP, _I32, _I64, _VP, _VP, _VP, _I32, _VP, ctypes.POINTER(np_config), _VP,
                     ctypes.POINTER(np_stats)],
    "np_bfs_host_async": [_VP, _I32, _I64, _VP, _VP, _I32, _VP, ctypes.POINTER(np_config), _VP],
    "np_sssp_host_async": [_VP, _I32, _I64, _VP, _VP, _VP, _I32, _VP, ctypes.POINTER(np_config), _VP],
    "np_bezier_noalloc": [_VP, _I32, _VP, _VP, _I64, ctypes.POINTER(np_config), _VP],
    "np_bezier_host": [_VP, _VP, _I32, _VP, _VP, _I64, ctypes.POINTER(np_config), _VP, ctypes.POINTER(np_stats)],
    "np_profile_enable": [_VP, _I32],
    "np_profile_read": [_VP, ctypes.POINTER(np_profile), _I32],
    "np_bfs_multi": [_VP, ctypes.POINTER(np_csr), _I32, _VP, _VP, _I64, ctypes.POINTER(np_config), _VP,
                     ctypes.POINTER(np_stats)],
    "np_sssp_multi": [_VP, ctypes.POINTER(np_csr), _I32, _VP, _VP, _I64, ctypes.POINTER(np_config), _VP,
                      ctypes.POINTER(np_stats)],
    "np_batch_create": [_VP, _I32, _VP, _VP, ctypes.POINTER(np_batch_options), ctypes.POINTER(ctypes.c_void_p)],
    "np_batch_destroy": [_VP],
    "np_batch_layout": [_VP, _VP, ctypes.POINTER(ctypes.c_int64)],
    "np_batch_classes": [_VP, _VP, _I32, ctypes.POINTER(ctypes.c_int32)],
    "np_batch_set_config": [_VP, _I32, ctypes.POINTER(np_config)],
    "np_batch_tune": [_VP, _VP, _I32, _VP],
    "np_batch_run": [_VP, _VP, _VP, ctypes.POINTER(np_stats)],
    "np_server_create": [_VP, _VP, _I32, ctypes.POINTER(np_server_options), ctypes.POINTER(ctypes.c_void_p)],
    "np_server_destroy": [_VP],
    "np_server_pool_info": [_VP, _I32, _I32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint64)],
    "np_server_submit": [_VP, _I32, _I32, _I32, _VP, ctypes.POINTER(ctypes.c_int64)],
    "np_server_step": [_VP, ctypes.POINTER(ctypes.c_int32)],
    "np_server_poll": [_VP, _I64, ctypes.POINTER(np_query_info)],
    "np_server_finished": [_VP, _VP, _I32, ctypes.POINTER(ctypes.c_int32)],
    "np_triangles": [_VP, ctypes.POINTER(np_csr), _VP, ctypes.POINTER(np_config), _VP, ctypes.POINTER(np_stats)],
    "np_selftest_wait": [_VP, _I32, _I64, _VP],
    "np_status_string": [_I32],
    "np_version": [],
}


def lib() -> ctypes.CDLL:
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "paper_2201_02789_gb300.build.build() (needs nvcc)")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_char_p if name == "np_status_string" else ctypes.c_int32
            _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


# ---------------------------------------------------------------- marshalling

def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s) -> int | None:
    if s is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(status: int, where: str, check: bool) -> int:
    if check and status != NP_OK:
        raise NestparError(status, where)
    return status


def _cfg(cfg) -> np_config:
    return cfg if cfg is not None else np_config_default()


def make_csr(row_ptr, col_idx, weights=None, n: int | None = None, m: int | None = None) -> np_csr:
    n = int(row_ptr.shape[0] - 1) if n is None else n
    m = int(col_idx.shape[0]) if m is None else m
    return np_csr(_ptr(row_ptr), _ptr(col_idx), _ptr(weights), n, m)


# ------------------------------------------------------------ entry points

def np_status_string(status: int) -> str:
    return lib().np_status_string(int(status)).decode()


def np_version() -> int:
    return int(lib().np_version())


def np_config_default() -> np_config:
    c = np_config()
    _check(lib().np_config_default(ctypes.byref(c)), "np_config_default", True)
    return c


def np_create(device: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().np_create(ctypes.byref(h), int(device)), "np_create", True)
    return h


def np_destroy(ctx) -> int:
    return _check(lib().np_destroy(ctx), "np_destroy", True)


def np_workspace_size(max_parents: int, cfg=None) -> int:
    b = ctypes.c_size_t()
    _check(lib().np_workspace_size(int(max_parents), ctypes.byref(_cfg(cfg)), ctypes.byref(b)),
           "np_workspace_size", True)
    return int(b.value)


def np_sync(ctx, stream=None, check: bool = True) -> tuple[int, dict]:
    st = np_stats()
    s = lib().np_sync(ctx, _stream(stream), ctypes.byref(st))
    return _check(s, "np_sync", check), st.as_dict()


def _stats_arg(stats: bool):
    return (np_stats(), True) if stats else (None, False)


def np_bfs(ctx, g: np_csr, src: int, level, cfg=None, stream=None, stats: bool = False, check: bool = True):
    st, want = _stats_arg(stats)
    s = lib().np_bfs(ctx, ctypes.byref(g), int(src), _ptr(level), ctypes.byref(_cfg(cfg)), _stream(stream),
                     ctypes.byref(st) if want else None)
    _check(s, "np_bfs", check)
    return (s, st.as_dict()) if want else s


def np_sssp(ctx, g: np_csr, src: int, dist, cfg=None, stream=None, stats: bool = False, check: bool = True):
    st, want = _stats_arg(stats)
    s = lib().np_sssp(ctx, ctypes.byref(g), int(src), _ptr(dist), ctypes.byref(_cfg(cfg)), _stream(stream),
                      ctypes.byref(st) if want else None)
    _check(s, "np_sssp", check)
    return (s, st.as_dict()) if want else s


def np_bezier(ctx, ctrl, ncurves: int, offsets, points, cap: int, cfg=None, stream=None, stats: bool = False,
              check: bool = True):
    st, want = _stats_arg(stats)
    s = lib().np_bezier(ctx, _ptr(ctrl), int(ncurves), _ptr(offsets), _ptr(points), int(cap),
                        ctypes.byref(_cfg(cfg)), _stream(stream), ctypes.byref(st) if want else None)
    _check(s, "np_bezier", check)
    return (s, st.as_dict()) if want else s


NP_NOALLOC_MAX_CURVES = 65536


def np_bezier_noalloc(ctrl, ncurves: int, offsets, points, cap: int, cfg=None, stream=None,
                      check: bool = True) -> int:
    """Tessellation without a context and without any allocation, for callers that
    cannot allocate device memory when they call (their memory belongs to their own
    pool or a fixed budget, or an allocation would stall a latency-critical loop).
    Scratch is a static device array sized for NP_NOALLOC_MAX_CURVES curves; calls
    that overlap on the GPU race on it. Make the first call on a device before any
    stream capture (it looks up and clears that array). offsets[ncurves] reports the
    outcome: the total, > cap on a capacity shortfall, -1 if a bounded wait gave up."""
    s = lib().np_bezier_noalloc(_ptr(ctrl), int(ncurves), _ptr(offsets), _ptr(points), int(cap),
                                ctypes.byref(_cfg(cfg)), _stream(stream))
    return _check(s, "np_bezier_noalloc", check)


def np_run_nested(ctx, parents: np_parents, count_kind: int, g: np_csr | None, body: np_body, cfg=None,
                  stream=None, stats: bool = False, check: bool = True):
    st, want = _stats_arg(stats)
    s = lib().np_run_nested(ctx, ctypes.byref(parents), int(count_kind), ctypes.byref(g) if g is not None else None,
                            ctypes.byref(body), ctypes.byref(_cfg(cfg)), _stream(stream),
                            ctypes.byref(st) if want else None)
    _check(s, "np_run_nested", check)
    return (s, st.as_dict()) if want else s


def np_bfs_host(ctx, row_ptr: np.ndarray, col_idx: np.ndarray, src: int, level_out: np.ndarray, cfg=None,
                stream=None, stats: bool = False, check: bool = True):
    st, want = _stats_arg(stats)
    s = lib().np_bfs_host(ctx, int(row_ptr.shape[0] - 1), int(col_idx.shape[0]), _ptr(row_ptr), _ptr(col_idx),
                          int(src), _ptr(level_out), ctypes.byref(_cfg(cfg)), _stream(stream),
                          ctypes.byref(st) if want else None)
    _check(s, "np_bfs_host", check)
    return (s, st.as_dict()) if want else s


def np_sssp_host(ctx, row_ptr, col_idx, weights, src: int, dist_out, cfg=None, stream=None,
                 stats: bool = False, check: bool = True):
    st, want = _stats_arg(stats)
    s = lib().np_sssp_host(ctx, int(row_ptr.shape[0] - 1), int(col_idx.shape[0]), _ptr(row_ptr), _ptr(col_idx),
                           _ptr(weights), int(src), _ptr(dist_out), ctypes.byref(_cfg(cfg)), _stream(stream),
                           ctypes.byref(st) if want else None)
    _check(s, "np_sssp_host", check)
    return (s, st.as_dict()) if want else s


def np_bfs_host_async(ctx, row_ptr, col_idx, src: int, level_out, cfg=None, stream=None, check: bool = True):
    """Stream-ordered np_bfs_host: returns once the copies, the solve and the copy out are
    enqueued on `stream`; the host arrays must stay alive until the stream passes the call."""
    s = lib().np_bfs_host_async(ctx, int(row_ptr.shape[0] - 1), int(col_idx.shape[0]), _ptr(row_ptr),
                                _ptr(col_idx), int(src), _ptr(level_out), ctypes.byref(_cfg(cfg)), _stream(stream))
    return _check(s, "np_bfs_host_async", check)


def np_sssp_host_async(ctx, row_ptr, col_idx, weights, src: int, dist_out, cfg=None, stream=None,
                       check: bool = True):
    """Stream-ordered np_sssp_host (see np_bfs_host_async)."""
    s = lib().np_sssp_host_async(ctx, int(row_ptr.shape[0] - 1), int(col_idx.shape[0]), _ptr(row_ptr),
                                 _ptr(col_idx), _ptr(weights), int(src), _ptr(dist_out), ctypes.byref(_cfg(cfg)),
                                 _stream(stream))
    return _check(s, "np_sssp_host_async", check)


def np_profile_enable(ctx, on: bool = True) -> int:
    return _check(lib().np_profile_enable(ctx, 1 if on else 0), "np_profile_enable", True)


def np_profile_read(ctx, reset: bool = False) -> dict:
    p = np_profile()
    _check(lib().np_profile_read(ctx, ctypes.byref(p), 1 if reset else 0), "np_profile_read", True)
    return p.as_dict()


def np_bezier_host(ctx, ctrl, ncurves: int, offsets_out, points_out, cap: int, cfg=None, stream=None,
                   stats: bool = False, check: bool = True):
    st, want = _stats_arg(stats)
    s = lib().np_bezier_host(ctx, _ptr(ctrl), int(ncurves), _ptr(offsets_out), _ptr(points_out), int(cap),
                             ctypes.byref(_cfg(cfg)), _stream(stream), ctypes.byref(st) if want else None)
    _check(s, "np_bezier_host", check)
    return (s, st.as_dict()) if want else s


# ------------------------------------------------------------ configurations

def np_triangles(ctx, dag: np_csr, count, cfg=None, stream=None, stats: bool = False, check: bool = True):
    st, want = _stats_arg(stats)
    s = lib().np_triangles(ctx, ctypes.byref(dag), _ptr(count), ctypes.byref(_cfg(cfg)), _stream(stream),
                           ctypes.byref(st) if want else None)
    _check(s, "np_triangles", check)
    return (s, st.as_dict()) if want else s


def np_bfs_multi(ctx, g: np_csr, sources, level, ld: int, cfg=None, stream=None, stats: bool = False,
                 check: bool = True):
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
    st, want = _stats_arg(stats)
    s = lib().np_bfs_multi(ctx, ctypes.byref(g), int(src.shape[0]), src.ctypes.data, _ptr(level), int(ld),
                           ctypes.byref(_cfg(cfg)), _stream(stream), ctypes.byref(st) if want else None)
    _check(s, "np_bfs_multi", check)
    return (s, st.as_dict()) if want else s


def np_sssp_multi(ctx, g: np_csr, sources, dist, ld: int, cfg=None, stream=None, stats: bool = False,
                  check: bool = True):
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
    st, want = _stats_arg(stats)
    s = lib().np_sssp_multi(ctx, ctypes.byref(g), int(src.shape[0]), src.ctypes.data, _ptr(dist), int(ld),
                            ctypes.byref(_cfg(cfg)), _stream(stream), ctypes.byref(st) if want else None)
    _check(s, "np_sssp_multi", check)
    return (s, st.as_dict()) if want else s


def multi_stride(n: int) -> int:
    """Row stride of np_bfs_multi / np_sssp_multi outputs: the next power of two >= n."""
    return 1 << max(0, (int(n) - 1).bit_length())


def np_batch_create(ctx, graphs: list[np_csr], sources, kind: int, cfg=None, class_log2_width: int = 0,
                    max_group_edges: int = 0) -> ctypes.c_void_p:
    arr = (np_csr * len(graphs))(*graphs)
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
    opt = np_batch_options(int(kind), int(class_log2_width), int(max_group_edges), _cfg(cfg))
    h = ctypes.c_void_p()
    _check(lib().np_batch_create(ctx, len(graphs), ctypes.cast(arr, ctypes.c_void_p), src.ctypes.data,
                                 ctypes.byref(opt), ctypes.byref(h)), "np_batch_create", True)
    return h


def np_batch_destroy(b) -> int:
    return _check(lib().np_batch_destroy(b), "np_batch_destroy", True)


def np_batch_layout(b, count: int) -> tuple[np.ndarray, int]:
    off = np.zeros(count, dtype=np.int64)
    tot = ctypes.c_int64()
    _check(lib().np_batch_layout(b, off.ctypes.data, ctypes.byref(tot)), "np_batch_layout", True)
    return off, int(tot.value)


def np_batch_classes(b) -> list[dict]:
    n = ctypes.c_int32()
    _check(lib().np_batch_classes(b, None, 0, ctypes.byref(n)), "np_batch_classes", True)
    arr = (np_batch_class * max(1, n.value))()
    _check(lib().np_batch_classes(b, ctypes.cast(arr, ctypes.c_void_p), n.value, ctypes.byref(n)),
           "np_batch_classes", True)
    return [arr[i].as_dict() for i in range(n.value)]


def np_batch_set_config(b, cls: int, cfg, check: bool = True) -> int:
    return _check(lib().np_batch_set_config(b, int(cls), ctypes.byref(cfg)), "np_batch_set_config", check)


def np_batch_tune(b, out, reps: int = 0, stream=None) -> int:
    return _check(lib().np_batch_tune(b, _ptr(out), int(reps), _stream(stream)), "np_batch_tune", True)


def np_batch_run(b, out, stream=None, stats: bool = False, check: bool = True):
    st, want = _stats_arg(stats)
    s = lib().np_batch_run(b, _ptr(out), _stream(stream), ctypes.byref(st) if want else None)
    _check(s, "np_batch_run", check)
    return (s, st.as_dict()) if want else s


def np_server_create(ctx, graphs: list[np_csr], memory_budget: int = 0, max_slots: int = 0,
                     levels_per_step: int = 0, bfs_cfg=None, sssp_cfg=None, check: bool = True):
    arr = (np_csr * len(graphs))(*graphs)
    opt = np_server_options(int(memory_budget), int(max_slots), int(levels_per_step), _cfg(bfs_cfg), _cfg(sssp_cfg))
    h = ctypes.c_void_p()
    s = lib().np_server_create(ctx, ctypes.cast(arr, ctypes.c_void_p), len(graphs), ctypes.byref(opt),
                               ctypes.byref(h))
    _check(s, "np_server_create", check)
    return h if s == NP_OK else s


def np_server_destroy(sv) -> int:
    return _check(lib().np_server_destroy(sv), "np_server_destroy", True)


def np_server_pool_info(sv, graph: int, kind: int) -> tuple[int, int]:
    slots = ctypes.c_int32()
    b = ctypes.c_uint64()
    _check(lib().np_server_pool_info(sv, int(graph), int(kind), ctypes.byref(slots), ctypes.byref(b)),
           "np_server_pool_info", True)
    return int(slots.value), int(b.value)


def np_server_submit(sv, graph: int, kind: int, src: int, out, check: bool = True) -> int:
    t = ctypes.c_int64()
    s = lib().np_server_submit(sv, int(graph), int(kind), int(src), _ptr(out), ctypes.byref(t))
    _check(s, "np_server_submit", check)
    return int(t.value) if s == NP_OK else -s


def np_server_step(sv, check: bool = True) -> int:
    k = ctypes.c_int32()
    _check(lib().np_server_step(sv, ctypes.byref(k)), "np_server_step", check)
    return int(k.value)


def np_server_poll(sv, ticket: int) -> dict:
    q = np_query_info()
    _check(lib().np_server_poll(sv, int(ticket), ctypes.byref(q)), "np_server_poll", True)
    return q.as_dict()


def np_server_finished(sv, max_count: int = 4096) -> list[int]:
    buf = np.zeros(max(1, max_count), dtype=np.int64)
    k = ctypes.c_int32()
    _check(lib().np_server_finished(sv, buf.ctypes.data, int(max_count), ctypes.byref(k)), "np_server_finished", True)
    return buf[:k.value].tolist()


def np_selftest_wait(ctx, which: int, limit_ns: int = 0, stream=None) -> int:
    """Status of one bounded wait on a flag nothing sets (expected NP_ERR_TIMEOUT)."""
    return int(lib().np_selftest_wait(ctx, int(which), int(limit_ns), _stream(stream)))


def config(form: str = "tca", **kw) -> np_config:
    """Named forms of the paper's evaluation: 'nodp', 'cdp' (plain device launch),
    't', 'c', 'tc', 'a', 'ta', 'ca', 'tca' (library default, grid-host aggregation).
    Keyword arguments override fields (granularity may be given by name)."""
    base = np_config_default()
    plain = dict(threshold=0, cfactor=1, granularity=NP_GRAN_NONE)
    forms = {
        "nodp": dict(variant=NP_VARIANT_NODP),
        "cdp": plain,
        "t": dict(plain, threshold=base.threshold),
        "c": dict(plain, cfactor=base.cfactor),
        "tc": dict(plain, threshold=base.threshold, cfactor=base.cfactor),
        "a": dict(plain, granularity=base.granularity),
        "ta": dict(plain, threshold=base.threshold, granularity=base.granularity),
        "ca": dict(plain, cfactor=base.cfactor, granularity=base.granularity),
        "tca": {},
    }
    return base.replace(**forms[form]).replace(**kw)


class Context:
    """Owns an ``np_ctx`` (workspace, graph cache) on one device."""

    def __init__(self, device: int = 0):
        self.device = device
        self.handle = np_create(device)

    def close(self):
        if self.handle:
            np_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
