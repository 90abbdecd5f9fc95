"""Helpers for the GPU tests: device copies of generated inputs and a shared context."""
from __future__ import annotations

import numpy as np
import torch

from paper_2201_02789_gb300 import nestpar as npb
from paper_2201_02789_gb300.devgraph import DevGraph  # noqa: F401  (re-exported for the tests)


def bfs(ctx, dg: DevGraph, src: int, cfg, stats=False):
    level = torch.empty(dg.n, dtype=torch.int32, device=dg.row_ptr.device)
    r = npb.np_bfs(ctx.handle, dg.csr, src, level, cfg, stats=stats)
    out = level.cpu().numpy()
    return (out, r[1]) if stats else out


def sssp(ctx, dg: DevGraph, src: int, cfg, stats=False):
    dist = torch.empty(dg.n, dtype=torch.int32, device=dg.row_ptr.device)
    r = npb.np_sssp(ctx.handle, dg.csr, src, dist, cfg, stats=stats)
    out = dist.cpu().numpy().view(np.uint32)
    return (out, r[1]) if stats else out


def bezier(ctx, ctrl: np.ndarray, cfg, cap=None, stats=False, check=True):
    dev = torch.device("cuda:0")
    nc = ctrl.shape[0]
    c_d = torch.from_numpy(np.ascontiguousarray(ctrl)).to(dev)
    off = torch.full((nc + 1,), -7, dtype=torch.int32, device=dev)
    if cap is None:
        cap = nc * 4096
    pts = torch.full((max(cap, 1), 2), float("nan"), dtype=torch.float32, device=dev)
    r = npb.np_bezier(ctx.handle, c_d, nc, off, pts, cap, cfg, stats=True, check=check)
    status, st = r
    return status, off.cpu().numpy(), pts.cpu().numpy(), st


def form_grid():
    """(name, config) pairs spanning variant x threshold x cfactor x granularity."""
    out = [("nodp", npb.config("nodp"))]
    grans = [("none", npb.NP_GRAN_NONE, {}), ("warp", npb.NP_GRAN_WARP, {}), ("block", npb.NP_GRAN_BLOCK, {}),
             ("mb1", npb.NP_GRAN_MULTIBLOCK, {"group_blocks": 1}),
             ("mb3", npb.NP_GRAN_MULTIBLOCK, {"group_blocks": 3}),
             ("mb8", npb.NP_GRAN_MULTIBLOCK, {"group_blocks": 8}),
             ("griddev", npb.NP_GRAN_GRID_DEVICE, {}),
             # (appending frontier: the library default sweeps levels of 4096 parents or more)
             ("gridhost-spread", npb.NP_GRAN_GRID_HOST, {"serial": npb.NP_SERIAL_SPREAD, "sweep_parents": 0}),
             ("gridhost-block", npb.NP_GRAN_GRID_HOST, {"serial": npb.NP_SERIAL_BLOCK}),
             ("gridhost-packed", npb.NP_GRAN_GRID_HOST, {"serial": npb.NP_SERIAL_PACKED}),
             # (the small-level loop off, so that the grids and the sweep run every level)
             ("gridhost-sweep", npb.NP_GRAN_GRID_HOST, {"sweep_parents": 1, "small_parents": 0})]
    for gname, gran, extra in grans:
        scans = ([("", npb.NP_SCAN_ATOMIC), ("-lb", npb.NP_SCAN_LOOKBACK)]
                 if gran in (npb.NP_GRAN_MULTIBLOCK, npb.NP_GRAN_GRID_DEVICE, npb.NP_GRAN_GRID_HOST) else [("", npb.NP_SCAN_ATOMIC)])
        for sname, scan in scans:
            for T in (0, 1, 32, 128, 1024, npb.INT32_MAX):
                for cf in (1, 2, 4, 8, 16):
                    out.append((f"{gname}{sname}-T{T}-C{cf}",
                                npb.config("tca", granularity=gran, threshold=T, cfactor=cf, scan=scan, **extra)))
    return out
