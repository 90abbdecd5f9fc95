"""Parity of a library variant built with a non-default build option.

Run as a script with NESTPAR_LIB naming the variant's libnestpar.so (one process
loads one copy of the library). It checks, against the oracle, BFS and SSSP on the
4096-vertex graph for a slice of the form grid that reaches every child-grid path
the options change (grid-host children of every coarsening factor and child block,
device-launched aggregated grids, the CTA-tiled and packed serial forms), then the
library default on the full R-MAT scale-20 graph. Exit status 0 when all match.
"""
from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from gpu_util import DevGraph, bfs, sssp  # noqa: E402
from paper_2201_02789_gb300 import gen  # noqa: E402
from paper_2201_02789_gb300 import nestpar as npb  # noqa: E402


def forms():
    out = []
    for T in (1, 32):
        for cf in (1, 2, 4, 8):
            for cb in (32, 64, 128):
                out.append((f"gridhost-T{T}-C{cf}-cb{cb}", npb.config("tca", threshold=T, cfactor=cf, child_block=cb)))
    out += [("multiblock", npb.config("tca", granularity="multiblock", group_blocks=4)),
            ("grid-device", npb.config("tca", granularity="grid_device", threshold=8)),
            ("block", npb.config("tca", granularity="block", threshold=2, cfactor=2)),
            ("serial-block", npb.config("tca", serial=npb.NP_SERIAL_BLOCK)),
            ("serial-packed", npb.config("tca", serial=npb.NP_SERIAL_PACKED, threshold=64)),
            ("no-small-loop", npb.config("tca", small_parents=0)),
            ("swept-frontier", npb.config("tca", sweep_parents=1, small_parents=0))]
    return out


def main() -> int:
    if not os.environ.get("NESTPAR_LIB"):
        print("NESTPAR_LIB must name the variant library")
        return 2
    ctx = npb.Context(0)
    bad = []
    g = gen.bfs4k()
    dg = DevGraph(g)
    ref_l, ref_d = oracle.bfs(g.row_ptr, g.col, 0), oracle.sssp(g.row_ptr, g.col, g.w, 0)
    for name, cfg in forms():
        if not np.array_equal(bfs(ctx, dg, 0, cfg), ref_l):
            bad.append(f"bfs4k bfs {name}")
        if not np.array_equal(sssp(ctx, dg, 0, cfg), ref_d):
            bad.append(f"bfs4k sssp {name}")
    r = gen.rmat20()
    dr = DevGraph(r)
    if not np.array_equal(bfs(ctx, dr, 0, npb.config("tca")), oracle.bfs(r.row_ptr, r.col, 0)):
        bad.append("rmat20 bfs")
    if not np.array_equal(sssp(ctx, dr, 0, npb.config("tca")), oracle.sssp(r.row_ptr, r.col, r.w, 0)):
        bad.append("rmat20 sssp")
    ctx.close()
    print(f"{npb.LIB_PATH}: {len(forms()) * 2 + 2 - len(bad)} checks exact, mismatches: {bad}")
    return 1 if bad else 0


if __name__ == "__main__":
    sys.exit(main())
