"""Benchmark of the nested-parallel hot path on one GB300 (or N replicas).

Default workload (the headline): single-source shortest paths by frontier
Bellman-Ford on a seeded R-MAT graph, scale 20 (1,048,576 vertices), edge
factor 16 (16,777,216 edges), a,b,c,d = .57/.19/.19/.05, uint32 weights uniform
in [1, 255], source 0. One step = one whole solve (every level of the nested
parent/child work) through the C ABI, graph resident in HBM. Between timed
steps L2 is flushed (a 512 MB write) outside the timed events.

The headline is the aggregated form (threshold + coarsening + grid
aggregation); plain CDP (one device launch per parent), the no-dynamic-
parallelism form and the device-launch aggregation forms are timed beside it
on the same GPU. GTEPS = edges out of reached vertices / solve time (Graph500
convention).

Other workloads (--workload): bfs-rmat20 (BFS on the same graph), bfs4k (the
4096-vertex power-law digraph), road (a 264K-vertex grid road graph with
out-degree <= 8: the low-nested-parallelism case, with the never-taken launch
site measured against the same kernel without it), bt64k (Bezier tessellation
of 65,536 curves, points/s; bt256k: 262,144 curves, whose points exceed L2), tc-rmat17 (triangle counting on the simple
undirected R-MAT scale-17 graph: the second CSR workload, an adjacency-
intersection child; oriented edges/s), batched-sssp / batched-bfs (512 R-MAT instances,
n log-uniform in [2^10, 2^20], edge factor 8..32, in one CUDA graph launch
per step after the per-size-class autotuner; total GTEPS), serving (Poisson
arrivals of BFS/SSSP queries from random sources over seven resident R-MAT
graphs of scales 16..22; queries/s at saturation and p50/p99 latency at
0.5/0.8/0.95 of it).

On one GPU the default run then measures every other workload, each in a
process of its own with few steps and a one-solve CPU leg (the oracle check),
and adds their figures to its JSON line as `other_workloads` (--no-others: not).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload W]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "GTEPS and ms/solve at 1 GB300: aggregated form vs plain CDP; % HBM roofline"
L2_NOTE = "flushed between timed steps (512 MB write)"
RMAT = {"vertices": 1 << 20, "edges": 16 << 20, "rmat_abcd": [0.57, 0.19, 0.19, 0.05],
        "weights": "uint32 uniform [1,255]", "source": 0, "seed": 2}
WORKLOADS = {
    "sssp-rmat20": dict(kind="sssp", graph="rmat20",
                        config=dict(workload="sssp_frontier_bellman_ford_rmat_scale20", **RMAT)),
    "bfs-rmat20": dict(kind="bfs", graph="rmat20", config=dict(workload="bfs_rmat_scale20", **RMAT)),
    "bfs4k": dict(kind="bfs", graph="bfs4k",
                  config=dict(workload="bfs_zipf_digraph_4096", vertices=4096, degrees="Zipf(2.1) on [1,1024]",
                              source=0, seed=1)),
    "road": dict(kind="sssp", graph="road",
                 config=dict(workload="sssp_road_grid_264k", vertices=514 * 514, degrees="2..8 (grid, diagonals p=1/2)",
                             weights="uint32 uniform [1,255]", source=0, seed=6)),
    "batched-sssp": dict(kind="batched", batch_kind=1,
                         config=dict(workload="batched_sssp_512_rmat_instances", instances=512,
                                     vertices="log-uniform [2^10, 2^20]", edge_factor="uniform [8, 32]",
                                     weights="uint32 uniform [1,255]", source=0, seed=4)),
    "batched-bfs": dict(kind="batched", batch_kind=0,
                        config=dict(workload="batched_bfs_512_rmat_instances", instances=512,
                                    vertices="log-uniform [2^10, 2^20]", edge_factor="uniform [8, 32]",
                                    source=0, seed=4)),
    "serving": dict(kind="serving",
                    config=dict(workload="serving_bfs_sssp_queries_rmat_scales_16_22", graphs="R-MAT scales 16..22",
                                edge_factor=16, weights="uint32 uniform [1,255]", mix="50/50 BFS/SSSP",
                                arrivals="Poisson", seed=5)),
    "tc-rmat17": dict(kind="tc", graph=None,
                      config=dict(workload="triangle_count_rmat_scale17_undirected", vertices=1 << 17,
                                  rmat_abcd=[0.57, 0.19, 0.19, 0.05], edge_factor=16, seed=7,
                                  preparation="simple undirected graph, edges oriented by (degree, id)")),
    "bt64k": dict(kind="bezier", graph=None,
                  config=dict(workload="bezier_tessellation_65536_curves", curves=65536,
                              points="ceil(sqrt(kappa)*64) clamped to [4,4096]", seed=3)),
    # four times the curves: about 200 MB of points, more than L2, so the child grid's point
    # stores reach DRAM within the timed kernel
    "bt256k": dict(kind="bezier", graph=None,
                   config=dict(workload="bezier_tessellation_262144_curves", curves=262144,
                               points="ceil(sqrt(kappa)*64) clamped to [4,4096]", seed=3)),
}


# per-workload values of the aggregated form's knobs, from threshold x cfactor x child-block
# sweeps on GB300 (the paper also tunes T and CF per benchmark); other workloads use the defaults
TUNED = {# tessellation: a threshold above every count, so that each curve's points run in its parent
         # warp (a whole warp per curve of 32 points or more) and no child grid is launched: 35 against
         # 42 us with the aggregated child grid below (BT_CHILD_GRID); 512-thread parent CTAs make the
         # output-offset look-back groups 16 tiles long
         "bt64k": dict(threshold=2**31 - 1, parent_block=512),
         # (BT-256K: 448-thread parent CTAs, 66.7 against 68.7 us at 512; BT-64K the same at both)
         "bt256k": dict(threshold=2**31 - 1, parent_block=448),
         "tc-rmat17": dict(threshold=8, child_block=32, cfactor=1),
         # SSSP: every grid level's children only reduce and a sweep over the vertex state forms the
         # next frontier (A/B on GB300: 454 -> 436 us; BFS, whose claims rarely reach the atomic,
         # loses 181 -> 187 us and keeps the appending frontier)
         "sssp-rmat20": dict(sweep_parents=1),
         # BFS: the appending frontier (the library default sweeps levels of 4096 parents or more,
         # 184.6 against 178.5 us here)
         "bfs-rmat20": dict(sweep_parents=0),
         # road grid (out-degree <= 8): a threshold above every degree launches nothing, so no child
         # grid runs at any level; appending frontiers (a sweep reads the whole state for a frontier
         # of about a tenth of it); 16 levels per while body over its 900 levels: 9.5 against 13.2 ms
         # with the defaults
         "road": dict(threshold=2**31 - 1, sweep_parents=0, unroll=16)}
# the tessellation's best form with an aggregated child grid: T 32 (the default), 32-thread child
# blocks of 4 original blocks, 512-thread parent CTAs spreading the serialised points over the CTA
# (serial 2: NP_SERIAL_BLOCK); timed beside the headline
BT_CHILD_GRID = dict(parent_block=512, child_block=32, cfactor=4, serial=2)
# (the 4096-vertex graph, latency-bound, runs almost every level in the while driver's one-CTA
# small-level loop: 115 us, against 150 us on the persistent level loop with 8 CTAs)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _cached(name, make):
    from paper_2201_02789_gb300 import gen
    cache = os.path.join(ROOT, "_cache")
    path = os.path.join(cache, name + ".npz")
    if os.path.exists(path):
        z = np.load(path)
        return gen.Csr(int(z["n"]), z["row_ptr"], z["col"], z["w"])
    g = make()
    try:
        os.makedirs(cache, exist_ok=True)
        np.savez(path + ".tmp.npz", n=g.n, row_ptr=g.row_ptr, col=g.col, w=g.w)
        os.replace(path + ".tmp.npz", path)
    except OSError:
        pass
    return g


def load_graph(which: str = "rmat20"):
    from paper_2201_02789_gb300 import gen
    if which == "rmat20":
        return _cached("rmat20_seed2", gen.rmat20)
    if which == "bfs4k":
        return gen.bfs4k()
    if which == "road":
        return _cached("road514_seed6", lambda: gen.road_grid(514, 514, seed=6))
    raise ValueError(which)


def max_over_ranks(x: float, device=None) -> float:
    """The largest value of x over the ranks of the job (x itself on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, steps: int, units_per_step: int, max_total_ms: float) -> float:
    """Whole-job throughput in G-units/s: every rank processed `steps` solves of
    `units_per_step` units (replicas, weak scaling) within the slowest rank's time."""
    return world * steps * units_per_step / (max_total_ms * 1e-3) / 1e9


def reached_edges(g, reached_mask) -> int:
    return int(np.diff(g.row_ptr.astype(np.int64))[np.asarray(reached_mask)].sum())


# ------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows: list[tuple[float, list[str]]] = []
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.25)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def mark(self, which: str):
        setattr(self, which, time.time())

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        lo, hi = (self.t0 or 0) - 0.15, (self.t1 or time.time()) + 0.15
        sel = [r for t, r in self.rows if lo <= t <= hi] or [r for _, r in self.rows]
        if not sel:
            return None
        sm = [float(r[1]) for r in sel if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in sel if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in sel for k in range(4) if len(r) > 5 + k and "Active" in r[5 + k]
                          and "Not" not in r[5 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sel)}


# --------------------------------------------------------------- roofline

def hbm_peak() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2201_02789_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str) -> float | None:
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if it was
    taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = dict(line.strip("- ").split(":", 1) for line in text.splitlines() if line.startswith("- ") and ":" in line)
    if vals.get("source_hash", "").strip() != source_hash():
        return None
    try:
        return float(vals["traffic_bytes_per_launch"].split()[0])
    except (KeyError, ValueError):
        return None


def kernel_bytes(kind: str, st: dict, W=None) -> dict:
    """Algorithmic bytes of one solve, split by kernel (per the counters `st`).

    SSSP parent grid: per frontier pop the id, the row_ptr pair and dist[u]
    (16 B); per serialised relaxation col + w + dist[v] (12 B); per launching
    parent a 16 B record and a 4 B block offset; per frontier append 4 B.
    SSSP child grid: per relaxation 12 B; per launching parent the record,
    offset and dist[u] it reads back (24 B).
    BFS: as SSSP without weights and dist[u] (pop 12 B, item 8 B, record read
    back 20 B). Bezier parent: per curve its control points and offset
    (28 B), per serialised point 8 B, per launching curve a 20 B record;
    Bezier child: 8 B per point, 44 B per launching curve (record, offset,
    control points)."""
    serial = st["items"] - st["child_items"]
    if kind == "sssp":
        parent = 16 * st["parents"] + 12 * serial + 20 * st["launch_parents"] + 4 * st["pushes"]
        child = 12 * st["child_items"] + 24 * st["launch_parents"]
        solve = 16 * st["parents"] + 12 * st["items"]
    elif kind == "bfs":
        parent = 12 * st["parents"] + 8 * serial + 20 * st["launch_parents"] + 4 * st["pushes"]
        child = 8 * st["child_items"] + 20 * st["launch_parents"]
        solve = 20 * st["parents"] + 8 * st["items"]
    elif kind == "tc":
        # per parent its row bounds (8 B); per oriented edge its column, the head's row
        # bounds and 4 B per walked out-list entry (W.walked / m of them on average)
        per_item = 12 + 4 * W.walked / max(W.dag.m, 1)
        parent = 8 * st["parents"] + per_item * serial + 20 * st["launch_parents"]
        child = per_item * st["child_items"] + 20 * st["launch_parents"]
        solve = W.bytes_per_solve()
    else:
        parent = 28 * st["parents"] + 8 * serial + 20 * st["launch_parents"]
        child = 8 * st["child_items"] + 44 * st["launch_parents"]
        solve = 28 * st["parents"] + 8 * st["items"]
    return {"parent": parent, "child": child, "solve": solve}


# ------------------------------------------------------------------ arms

def run_reference(args, ws, rank):
    """The oracle on the host cores, as the reference arm."""
    if rank != 0:
        return
    import oracle
    wl = WORKLOADS[args.workload]
    if wl["kind"] in ("batched", "serving"):
        return run_reference_multi(args, ws, wl)
    if wl["kind"] == "bezier":
        from paper_2201_02789_gb300 import gen
        ctrl = gen.bezier_curves(wl["config"]["curves"], seed=wl["config"]["seed"])
        run = lambda: oracle.bezier(ctrl)
        units = lambda out: int(out[0][-1])
        unit = "Gpoints/s"
    elif wl["kind"] == "tc":
        from paper_2201_02789_gb300 import gen
        ug, dag = gen.tc_rmat17()
        run = lambda: oracle.triangles(ug.row_ptr, ug.col)
        units = lambda out: dag.m
        unit = "Gedges/s"
        args.steps = min(args.steps, 3)
        args.warmup = min(args.warmup, 1)
    else:
        g = load_graph(wl["graph"])
        if wl["kind"] == "sssp":
            run = lambda: oracle.sssp(g.row_ptr, g.col, g.w, 0)
            units = lambda d: reached_edges(g, d != 0xFFFFFFFF)
        else:
            run = lambda: oracle.bfs(g.row_ptr, g.col, 0)
            units = lambda lv: reached_edges(g, lv >= 0)
        unit = "GTEPS"
    for _ in range(args.warmup):
        out = run()
    ts = []
    for _ in range(args.steps):
        t = time.perf_counter()
        out = run()
        ts.append(time.perf_counter() - t)
    u = units(out)
    total = sum(ts)
    value = args.steps * u / total / 1e9
    line = {"impl": "reference", "metric": METRIC if args.workload == "sssp-rmat20" else f"{unit} ({args.workload})",
            "value": value, "unit": unit, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"bezier": "f32", "tc": "i32"}.get(wl["kind"], "u32"), "data": "synthetic",
            "config": dict(wl["config"], l2="n/a (host)"),
            "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full solves of the workload"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_solves(fn, steps, flush, stream):
    import torch
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms


class GraphWorkload:
    """BFS / SSSP on a resident CSR graph through np_bfs / np_sssp."""

    def __init__(self, kind, g, dev, stream, ctx):
        import torch
        from paper_2201_02789_gb300.devgraph import DevGraph
        from paper_2201_02789_gb300 import nestpar as npb
        self.npb, self.kind, self.g, self.stream, self.ctx = npb, kind, g, stream, ctx
        self.dg = DevGraph(g, device=dev)
        self.out = torch.empty(g.n, dtype=torch.int32, device=dev)
        self.unit = "GTEPS"

    def solve(self, cfg, stats=False):
        f = self.npb.np_sssp if self.kind == "sssp" else self.npb.np_bfs
        return f(self.ctx.handle, self.dg.csr, 0, self.out, cfg, stream=self.stream, stats=stats)

    def result(self):
        r = self.out.cpu().numpy()
        return r.view(np.uint32) if self.kind == "sssp" else r

    def reached(self, r):
        return (r != 0xFFFFFFFF) if self.kind == "sssp" else (r >= 0)

    def units(self):
        return reached_edges(self.g, self.reached(self.result()))

    def oracle(self):
        import oracle
        g = self.g
        return oracle.sssp(g.row_ptr, g.col, g.w, 0) if self.kind == "sssp" else oracle.bfs(g.row_ptr, g.col, 0)

    def e2e(self, cfg, steps, flush, dev):
        import torch
        g = self.g
        rp_h = torch.from_numpy(g.row_ptr).pin_memory()
        col_h = torch.from_numpy(g.col).pin_memory()
        out_h = torch.empty(g.n, dtype=torch.int32).pin_memory()
        w_h = torch.from_numpy(g.w.view(np.int32)).pin_memory() if self.kind == "sssp" else None
        ms = []
        for k in range(steps + 1):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t = time.perf_counter()
            if self.kind == "sssp":
                self.npb.np_sssp_host(self.ctx.handle, rp_h, col_h, w_h, 0, out_h, cfg, stream=self.stream)
            else:
                self.npb.np_bfs_host(self.ctx.handle, rp_h, col_h, 0, out_h, cfg, stream=self.stream)
            if k:
                ms.append((time.perf_counter() - t) * 1e3)
        res = out_h.numpy().view(np.uint32) if self.kind == "sssp" else out_h.numpy().copy()
        h2d = 4 * (g.n + 1) + (8 if self.kind == "sssp" else 4) * g.m
        return ms, h2d, 4 * g.n, res

    def e2e_pipelined(self, cfg, steps, flush, dev):
        """The stream-ordered host calls (np_*_host_async) alternating over two contexts on two
        streams, so that one step's copies run while the other context solves. Every step
        still copies its whole graph in from pinned memory and its result out; the L2 flush
        runs on the step's own stream before its copies. Returns ms per step over the run."""
        import torch
        g = self.g
        ctxs = [self.ctx, self.npb.Context(dev.index)]
        streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
        rp_h = torch.from_numpy(g.row_ptr).pin_memory()
        col_h = torch.from_numpy(g.col).pin_memory()
        w_h = torch.from_numpy(g.w.view(np.int32)).pin_memory() if self.kind == "sssp" else None
        outs = [torch.empty(g.n, dtype=torch.int32).pin_memory() for _ in range(2)]

        def step(k):
            c, s = ctxs[k % 2], streams[k % 2]
            with torch.cuda.stream(s):
                flush.zero_()
            if self.kind == "sssp":
                self.npb.np_sssp_host_async(c.handle, rp_h, col_h, w_h, 0, outs[k % 2], cfg, stream=s)
            else:
                self.npb.np_bfs_host_async(c.handle, rp_h, col_h, 0, outs[k % 2], cfg, stream=s)

        try:
            for k in range(4):   # warm-up: both contexts build their graphs and staging buffers
                step(k)
            torch.cuda.synchronize(dev)
            t = time.perf_counter()
            for k in range(steps):
                step(k)
            torch.cuda.synchronize(dev)
            ms = (time.perf_counter() - t) * 1e3 / steps
            for c, s in zip(ctxs, streams):
                self.npb.np_sync(c.handle, stream=s)
            res = [o.numpy().view(np.uint32) if self.kind == "sssp" else o.numpy().copy() for o in outs]
        finally:
            ctxs[1].close()
        return ms, res


class BezierWorkload:
    """Tessellation of a seeded curve set (65,536 curves by default) through np_bezier."""

    def __init__(self, dev, stream, ctx, ncurves=65536, seed=3):
        import torch
        from paper_2201_02789_gb300 import gen
        from paper_2201_02789_gb300 import nestpar as npb
        self.npb, self.stream, self.ctx, self.kind = npb, stream, ctx, "bezier"
        self.nc = ncurves
        self.ctrl = gen.bezier_curves(ncurves, seed=seed)
        self.c_d = torch.from_numpy(self.ctrl).to(dev)
        self.cap = ncurves * 200
        self.off = torch.empty(ncurves + 1, dtype=torch.int32, device=dev)
        self.pts = torch.empty((self.cap, 2), dtype=torch.float32, device=dev)
        self.unit = "Gpoints/s"

    def solve(self, cfg, stats=False):
        return self.npb.np_bezier(self.ctx.handle, self.c_d, self.nc, self.off, self.pts, self.cap, cfg,
                                  stream=self.stream, stats=stats)

    def result(self):
        return self.off.cpu().numpy()

    def units(self):
        return int(self.result()[-1])

    def oracle(self):
        """The whole tessellation in the oracle: offsets and FP64 points."""
        import oracle
        return oracle.bezier(self.ctrl)

    @staticmethod
    def comparable(ref):
        """The part of an oracle result the device result (the offsets) is compared with."""
        return ref[0]

    def point_errors(self, ref=None):
        """FP32 points against the FP64 oracle (outside any timed region): the largest
        |g - r| / max(|r|, 1) (the tolerance's scale, bound 1e-5), and the largest strict
        relative error |g - r| / |r| over coordinates with |r| >= 1e-3."""
        import oracle
        ref_off, ref_pts = ref if ref is not None else oracle.bezier(self.ctrl)
        total = int(ref_off[-1])
        got = self.pts[:total].cpu().numpy().astype(np.float64)
        err = np.abs(got - ref_pts)
        big = np.abs(ref_pts) >= 1e-3
        return {"points_max_scaled_err": float((err / np.maximum(np.abs(ref_pts), 1.0)).max()),
                "points_within_1e-5_scaled": bool((err <= 1e-5 * np.maximum(np.abs(ref_pts), 1.0)).all()),
                "points_max_abs_err": float(err.max()),
                "points_max_rel_err_where_abs_ge_1e-3": float((err[big] / np.abs(ref_pts[big])).max())}

    def e2e(self, cfg, steps, flush, dev):
        import torch
        c_h = torch.from_numpy(self.ctrl).pin_memory()
        off_h = torch.empty(self.nc + 1, dtype=torch.int32).pin_memory()
        pts_h = torch.empty((self.cap, 2), dtype=torch.float32).pin_memory()
        ms = []
        for k in range(steps + 1):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t = time.perf_counter()
            self.npb.np_bezier_host(self.ctx.handle, c_h, self.nc, off_h, pts_h, self.cap, cfg, stream=self.stream)
            if k:
                ms.append((time.perf_counter() - t) * 1e3)
        total = int(off_h[-1].item())
        return ms, 24 * self.nc, 4 * (self.nc + 1) + 8 * total, off_h.numpy().copy()


class TcWorkload:
    """Triangle counting on the degree-oriented simple undirected R-MAT-17 graph (np_triangles)."""

    def __init__(self, dev, stream, ctx):
        import torch
        from paper_2201_02789_gb300.devgraph import DevGraph
        from paper_2201_02789_gb300 import gen
        from paper_2201_02789_gb300 import nestpar as npb
        self.npb, self.stream, self.ctx, self.kind = npb, stream, ctx, "tc"
        self.u, self.dag = gen.tc_rmat17()
        self.dg = DevGraph(self.dag, device=dev)
        self.out = torch.zeros(1, dtype=torch.int64, device=dev)
        self.unit = "Gedges/s"
        deg = np.diff(self.dag.row_ptr.astype(np.int64))
        src = np.repeat(np.arange(self.dag.n), deg)
        # entries walked by the intersections: the shorter out-list of each oriented edge
        self.walked = int(np.minimum(deg[src], deg[self.dag.col]).sum())

    def solve(self, cfg, stats=False):
        return self.npb.np_triangles(self.ctx.handle, self.dg.csr, self.out, cfg, stream=self.stream, stats=stats)

    def result(self):
        return self.out.cpu().numpy().copy()

    def units(self):
        return self.dag.m

    def oracle(self):
        import oracle
        return np.array([oracle.triangles(self.u.row_ptr, self.u.col)], dtype=np.int64)

    def bytes_per_solve(self):
        """Row bounds per parent (8 B), per oriented edge its column and the row bounds of its
        head (12 B), and 4 B per walked out-list entry (the searched list's reads hit L1/L2)."""
        return 8 * self.dag.n + 12 * self.dag.m + 4 * self.walked

    def e2e(self, cfg, steps, flush, dev):
        import torch
        rp_h = torch.from_numpy(self.dag.row_ptr).pin_memory()
        col_h = torch.from_numpy(self.dag.col).pin_memory()
        out_h = torch.zeros(1, dtype=torch.int64).pin_memory()
        rp = torch.empty_like(rp_h, device=dev)
        col = torch.empty_like(col_h, device=dev)
        csr = self.npb.make_csr(rp, col, None, n=self.dag.n, m=self.dag.m)
        ms = []
        for k in range(steps + 1):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t = time.perf_counter()
            rp.copy_(rp_h, non_blocking=True)
            col.copy_(col_h, non_blocking=True)
            self.npb.np_triangles(self.ctx.handle, csr, self.out, cfg, stream=self.stream)
            out_h.copy_(self.out, non_blocking=True)
            torch.cuda.synchronize(dev)
            if k:
                ms.append((time.perf_counter() - t) * 1e3)
        return ms, 4 * (self.dag.n + 1) + 4 * self.dag.m, 8, out_h.numpy().copy()


def comparison_forms(npb, workload: str, cdp_steps: int):
    """(name, config, timed steps) of the forms timed beside the headline."""
    if workload == "road":
        # low nested parallelism (Section VII-D): no-DP, the same CTA-tiled kernel
        # with and without a launch site that never runs, and the aggregated form
        # the pair below differs only in the launch site: same CTA-tiled kernel,
        # same host-replayed chunk driver
        chunk = dict(driver=npb.NP_DRIVER_CHUNK)
        persist = dict(driver=npb.NP_DRIVER_PERSISTENT)
        return [("nodp", npb.config("nodp"), 5),
                ("nodp_persistent", npb.config("nodp", **persist), 5),
                ("t_c_a_persistent", npb.config("tca", **persist), 5),
                ("nodp_cta_tiles_no_launch_code", npb.config("nodp", granularity="none", **chunk), 5),
                ("cdp_threshold_above_max_degree", npb.config("cdp", threshold=npb.INT32_MAX, **chunk), 5),
                ("plain_cdp", npb.config("cdp"), cdp_steps),
                ("t_c", npb.config("tc"), cdp_steps)]
    bt_only = [("t_c_a_grid_host_child_grid", npb.config("tca", **BT_CHILD_GRID), 20)] \
        if workload in ("bt64k", "bt256k") else []
    graph_only = [] if workload in ("bt64k", "bt256k", "tc-rmat17") else [
        ("t_c_a_persistent", npb.config("tca", driver=npb.NP_DRIVER_PERSISTENT), 5),
        ("nodp_persistent", npb.config("nodp", driver=npb.NP_DRIVER_PERSISTENT), 5)]
    return [("plain_cdp", npb.config("cdp"), cdp_steps), ("nodp", npb.config("nodp"), cdp_steps),
            ("t_c", npb.config("tc"), cdp_steps),
            ("t_c_a_multiblock", npb.config("tca", granularity="multiblock", group_blocks=8), 5),
            ("t_c_a_grid_device", npb.config("tca", granularity="grid_device"), 5),
            ("t_c_a_block", npb.config("tca", granularity="block"), 5)] + bt_only + graph_only


# The other workloads, measured after the default (headline) run and summarised in its JSON line:
# each runs in a process of its own with few steps and a one-solve CPU leg (which still checks the
# result against the oracle). (name, extra arguments)
OTHER_WORKLOADS = [("bfs-rmat20", ["--steps", "50"]), ("bt64k", ["--steps", "100"]), ("bt256k", ["--steps", "50"]),
                   ("bfs4k", ["--steps", "100"]), ("tc-rmat17", ["--steps", "20"]),
                   ("road", ["--steps", "5", "--cdp-steps", "1"]), ("batched-sssp", ["--steps", "5"]),
                   ("batched-bfs", ["--steps", "5"]), ("serving", ["--steps", "5"])]
OTHERS_SECONDS = 420   # no further workload starts after this much time


def compact(d: dict) -> dict:
    """The figures of a workload's JSON line that the headline line carries."""
    out = {k: d[k] for k in ("metric", "value", "unit", "ms_per_step", "gpu_launches") if k in d}
    r = d.get("roofline") or {}
    if r:
        out["roofline"] = {k: r.get(k) for k in ("kernel", "achieved", "peak", "frac", "traffic")}
    if d.get("step_roofline"):
        out["step_roofline_frac"] = d["step_roofline"].get("frac")
    if d.get("e2e"):
        out["e2e"] = {k: d["e2e"].get(k) for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")}
    for k in ("parity_vs_oracle", "parity_vs_oracle_sample", "speedup_vs_plain_cdp", "speedup_vs_nodp",
              "speedup_vs_sequential", "saturation", "poisson"):
        if k in d:
            out[k] = d[k]
    out["clocks"] = d.get("clocks")
    return out


def run_other_workloads() -> dict:
    """Runs OTHER_WORKLOADS one after another (one GPU); per workload its compact figures, the
    command, or the error that stopped it."""
    import subprocess
    res = {}
    t0 = time.perf_counter()
    for name, extra in OTHER_WORKLOADS:
        if time.perf_counter() - t0 > OTHERS_SECONDS:
            res[name] = {"skipped": "time cap of the default run reached"}
            continue
        cmd = ["python", "bench.py", "--workload", name, "--warmup", "3", "--cpu-seconds", "0.1",
               "--e2e-steps", "2", "--no-others"] + extra
        try:
            r = subprocess.run([sys.executable] + cmd[1:], cwd=ROOT, capture_output=True, text=True, timeout=240)
            lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
            if r.returncode != 0 or not lines:
                res[name] = {"command": " ".join(cmd), "error": f"exit {r.returncode}: {r.stderr[-300:]}"}
                continue
            res[name] = dict(compact(json.loads(lines[-1])), command=" ".join(cmd))
        except Exception as e:   # a failed side measurement never costs the headline line
            res[name] = {"command": " ".join(cmd), "error": repr(e)[:300]}
    return res


def run_ours(args, ws, rank, local):
    import torch
    from paper_2201_02789_gb300 import build as nbuild
    from paper_2201_02789_gb300 import nestpar as npb

    nbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    distributed = ws > 1
    if distributed:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = WORKLOADS[args.workload]
    ctx = npb.Context(local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.int8, device=dev)
    if wl["kind"] == "bezier":
        W = BezierWorkload(dev, stream, ctx, wl["config"]["curves"], wl["config"]["seed"])
    elif wl["kind"] == "tc":
        W = TcWorkload(dev, stream, ctx)
    else:
        W = GraphWorkload(wl["kind"], load_graph(wl["graph"]), dev, stream, ctx)
    # the aggregated form; tessellation keeps the child block and coarsening factor
    # its own sweep picked (32-thread child blocks, cfactor 8)
    cfg = npb.config("tca", **TUNED.get(args.workload, {}))

    for _ in range(max(args.warmup, 3)):
        W.solve(cfg)
    _, st = W.solve(cfg, stats=True)
    res_gpu = W.result()
    units = W.units()

    sampler = ClockSampler(local)
    sampler.start()
    if distributed:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    sampler.mark("t0")
    ms = time_solves(lambda: W.solve(cfg), args.steps, flush, stream)
    torch.cuda.synchronize(dev)
    sampler.mark("t1")
    if distributed:
        torch.distributed.barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(ms), dev)
    value = job_value(ws, args.steps, units, total_ms)
    ms_per_step = total_ms / args.steps

    if rank != 0:
        ctx.close()
        if distributed:
            torch.distributed.destroy_process_group()
        return

    # kernels launched per solve: graph solves launch init (+ the small-level loop once before
    # the while loop) + per while-body iteration `unroll` x (parent, child[, sweep]) + the
    # condition kernel (the small-level loop); a tessellation launches init, parent and child
    # (no child when the threshold launches nothing and no children are packed for it)
    if wl["kind"] == "bezier":
        per_solve = 2 if cfg.threshold == npb.INT32_MAX and cfg.serial != npb.NP_SERIAL_PACKED else 3
    elif wl["kind"] == "tc":
        per_solve = 4          # level-state reset, parent, child, partial-count sum
    else:
        # init + while-body iterations x (unroll x (parent, child) + condition) (+ the SSSP
        # distances written from the packed state)
        # (the swept frontier adds its sweep kernel to every grid level)
        # (a threshold that launches nothing runs no child grid, and a level that sweeps adds the sweep)
        child_runs = not (cfg.threshold == npb.INT32_MAX and cfg.serial != npb.NP_SERIAL_PACKED)
        per_level = 1 + (1 if child_runs else 0) + (1 if cfg.sweep_parents > 0 else 0)
        loop = 1 if cfg.driver == npb.NP_DRIVER_PERSISTENT else st["graph_iterations"] * (per_level * cfg.unroll + 1)
        pre = 1 if cfg.driver != npb.NP_DRIVER_PERSISTENT and cfg.small_parents > 0 else 0
        per_solve = 1 + pre + loop + (1 if wl["kind"] == "sssp" else 0)
    gpu_launches = int(per_solve * args.steps)
    metric = METRIC if args.workload == "sssp-rmat20" else \
        f"{W.unit} and ms/solve ({args.workload}): aggregated form vs plain CDP; % HBM roofline"

    if args.only_headline:
        # small run for profiler captures: the headline form, then profile-mode solves
        npb.np_profile_enable(ctx.handle, True)
        for _ in range(3):
            flush.zero_()
            W.solve(cfg, stats=True)
        npb.np_profile_enable(ctx.handle, False)
        print(json.dumps({"metric": metric, "value": value, "unit": W.unit, "ms_per_step": ms_per_step,
                          "gpu_launches": gpu_launches, "only_headline": True}), flush=True)
        ctx.close()
        return

    # forms beside the headline, same GPU, same input
    forms = {}
    for name, c, reps in comparison_forms(npb, args.workload, args.cdp_steps):
        W.solve(c)
        t = time_solves(lambda c=c: W.solve(c), reps, flush, stream)
        m = statistics.median(t)
        _, fst = W.solve(c, stats=True)
        forms[name] = {"ms_per_solve": m, "value": units / (m * 1e-3) / 1e9, "unit": W.unit,
                       "device_launches": fst["device_launches"],
                       "matches_headline": bool(np.array_equal(W.result(), res_gpu))}
    torch.cuda.synchronize(dev)

    # roofline of the dominant kernel: profile mode (separate launches, CUDA events)
    npb.np_profile_enable(ctx.handle, True)
    npb.np_profile_read(ctx.handle, reset=True)
    prof_runs = 3
    for _ in range(prof_runs):
        flush.zero_()
        _, pst = W.solve(cfg, stats=True)
    prof = npb.np_profile_read(ctx.handle, reset=True)
    npb.np_profile_enable(ctx.handle, False)
    kb = kernel_bytes(wl["kind"], pst, W)
    peak, peak_kind = hbm_peak()
    # the grid-host form's parent kernel: warp tiles, or CTA tiles for the CTA-spread / packed
    # serial children (whose child grid is child_agg_pack)
    cta = cfg.serial in (npb.NP_SERIAL_BLOCK, npb.NP_SERIAL_PACKED)
    child_name = "child_agg_pack" if cfg.serial == npb.NP_SERIAL_PACKED else "child_agg"
    kernels = {child_name: (prof["child_ms"], prof["child_launches"], kb["child"]),
               ("parent_cta" if cta else "parent_warp"): (prof["parent_ms"], prof["parent_launches"], kb["parent"])}
    dom = max(kernels, key=lambda k: kernels[k][0])
    k_ms, k_launches, k_bytes = kernels[dom]
    per_launch_bytes = k_bytes * prof_runs / max(k_launches, 1)
    avg_ms = k_ms / max(k_launches, 1)
    achieved = per_launch_bytes / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": ncu_traffic(dom, args.workload),
                "kernel": dom, "peak_kind": f"{peak_kind} (copy bandwidth, burst)",
                "avg_launch_ms": avg_ms, "algorithmic_bytes_per_launch": per_launch_bytes,
                "share_of_profiled_time": k_ms / max(prof["parent_ms"] + prof["child_ms"] + prof["other_ms"], 1e-9)}
    solve_bytes = kb["solve"]
    step_roofline = {"algorithmic_bytes": solve_bytes, "achieved_gbs": solve_bytes / (ms_per_step * 1e-3) / 1e9,
                     "frac": solve_bytes / (ms_per_step * 1e-3) / 1e9 / peak}
    if wl["kind"] == "sssp":
        # the bytes of a solve that relaxes every reached edge once (16 B per reached vertex,
        # 12 B per edge out of one): what redundant relaxations would otherwise hide
        n_r = int(W.reached(W.result()).sum())
        b_min = 16 * n_r + 12 * units
        step_roofline.update({"algorithmic_bytes_min": b_min, "reached_vertices": n_r,
                              "achieved_gbs_min": b_min / (ms_per_step * 1e-3) / 1e9,
                              "frac_min": b_min / (ms_per_step * 1e-3) / 1e9 / peak})
    breakdown = {k: prof[k] for k in ("parent_ms", "child_ms", "other_ms", "parent_launches", "child_launches",
                                      "longest_level_ms", "levels")}
    breakdown["level_parents"] = prof.get("level_parents")

    # end to end through the C ABI from pinned host buffers
    e2e_ms, h2d, d2h, e2e_res = W.e2e(cfg, args.e2e_steps, flush, dev)
    e2e = {"value": units / (statistics.median(e2e_ms) * 1e-3) / 1e9, "unit": W.unit,
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
           "ms_per_step": statistics.median(e2e_ms),
           "matches_device_result": bool(np.array_equal(e2e_res, res_gpu)),
           "mode": "one waiting call per step (np_*_host), median step"}
    if hasattr(W, "e2e_pipelined"):
        # steps overlapped on two contexts (the upload of one with the solve of the other;
        # the L2 flush of every step is inside this timed region); the faster of the two
        # host-buffer modes is the end-to-end figure, the other stays beside it
        p_ms, p_res = W.e2e_pipelined(cfg, max(args.e2e_steps, 8), flush, dev)
        pip = {"value": units / (p_ms * 1e-3) / 1e9, "ms_per_step": p_ms,
               "mode": "stream-ordered calls (np_*_host_async) alternating over 2 contexts and 2 streams"}
        wait = {k: e2e[k] for k in ("value", "ms_per_step", "mode")}
        best, other = (pip, wait) if pip["value"] >= wait["value"] else (wait, pip)
        e2e.update(best)
        e2e["matches_device_result"] = bool(e2e["matches_device_result"] and
                                            all(np.array_equal(r, res_gpu) for r in p_res))
        e2e["other_mode"] = other

    # CPU baseline: the oracle as it stands, one core, bounded sample; also the parity check
    cpu = None
    parity = None
    if ws == 1 and not args.no_cpu:
        ts = []
        ref = None
        t_end = time.perf_counter() + args.cpu_seconds
        while time.perf_counter() < t_end or not ts:
            t = time.perf_counter()
            ref = W.oracle()
            ts.append(time.perf_counter() - t)
        parity = bool(np.array_equal(W.comparable(ref) if hasattr(W, "comparable") else ref, res_gpu))
        if wl["kind"] == "bezier":
            parity = {"offsets_exact": parity, **W.point_errors(ref)}
        cpu = {"value": units / statistics.mean(ts) / 1e9, "unit": W.unit, "cores": 1, "kind": "oracle",
               "sample": f"{len(ts)} full solves of the workload ({sum(ts):.1f} s)",
               "ms_per_solve": statistics.mean(ts) * 1e3}

    line = {"metric": metric, "value": value, "unit": W.unit, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"bezier": "f32", "tc": "i32"}.get(wl["kind"], "u32"), "data": "synthetic",
            "config": dict(wl["config"], l2=L2_NOTE),
            "form": (("threshold INT32_MAX (no child launches: the serialised children run in the parent "
                      "warps, a whole warp per parent of 32 or more), " if wl["kind"] == "bezier" else
                      "threshold INT32_MAX (no child launches: the serialised children spread over the "
                      "parent warps), ") if cfg.threshold == npb.INT32_MAX else
                     f"threshold {cfg.threshold} + coarsening {cfg.cfactor} ({cfg.child_block}-thread child blocks) "
                     "+ grid aggregation (atomic scan), ") + (
                        "one fixed pass replayed as a CUDA graph" if wl["kind"] in ("bezier", "tc") else
                        f"persistent cooperative level loop on {cfg.parent_grid} CTAs"
                        if cfg.driver == npb.NP_DRIVER_PERSISTENT else "while-graph level loop"),
            "ms_per_solve": {"median": statistics.median(ms), "min": min(ms)},
            "units_per_solve": units, "levels": st["levels"], "child_items": st["items"],
            "speedup_vs_plain_cdp": forms["plain_cdp"]["ms_per_solve"] / statistics.median(ms),
            "speedup_vs_nodp": forms["nodp"]["ms_per_solve"] / statistics.median(ms),
            "forms": forms, "roofline": roofline, "step_roofline": step_roofline,
            "cpu_baseline": cpu, "parity_vs_oracle": parity, "e2e": e2e, "clocks": clocks,
            "gpu_launches": gpu_launches, "profile_breakdown": breakdown}
    if ws == 1 and args.workload == "sssp-rmat20" and not args.no_others:
        # the other workloads, each in a process of its own after this one's GPU work
        torch.cuda.synchronize(dev)
        line["other_workloads"] = run_other_workloads()
    print(json.dumps(line), flush=True)
    ctx.close()
    if distributed:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------- batched and serving

def batch_inputs(batch_kind: int):
    from paper_2201_02789_gb300 import build as nbuild
    from paper_2201_02789_gb300 import gen
    nbuild.build_gen()
    specs = gen.batch_specs(512, seed=4)
    graphs = gen.batch_graphs(specs, weights=(1, 255) if batch_kind == 1 else None)
    return specs, graphs


def serving_graphs():
    from paper_2201_02789_gb300 import build as nbuild
    from paper_2201_02789_gb300 import gen
    from concurrent.futures import ThreadPoolExecutor
    nbuild.build_gen()
    with ThreadPoolExecutor(7) as ex:
        return list(ex.map(lambda s: gen.rmat(s, 16, seed=5 * 1000 + s), range(16, 23)))


def serving_queries(graphs, count: int, seed: int):
    """(graph, kind, source) per query: graph and kind uniform, source uniform over vertices with edges."""
    from paper_2201_02789_gb300 import gen
    gi = gen.uniform_int(seed, gen.S_SOURCE + 10, 0, count, 0, len(graphs) - 1)
    kinds = gen.uniform_int(seed, gen.S_SOURCE + 11, 0, count, 0, 1)
    out = []
    for q in range(count):
        g = graphs[int(gi[q])]
        src = int(gen.random_sources(g, 1, seed=seed * 100003 + q)[0])
        out.append((int(gi[q]), int(kinds[q]), src))
    return out


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process: exponential gaps from the seeded uniform stream."""
    from paper_2201_02789_gb300 import gen
    u = gen.uniform_f64(seed, gen.S_SOURCE + 12, 0, count)
    return np.cumsum(-np.log1p(-u) / rate)


def run_reference_multi(args, ws, wl):
    """Reference arm for the batched and serving workloads: the oracle, one query or
    instance after another, on a bounded sample of the workload per step."""
    import oracle
    if wl["kind"] == "batched":
        specs, graphs = batch_inputs(wl["batch_kind"])
        order = np.argsort([g.n for g in graphs], kind="stable")
        sample = [int(order[k]) for k in np.linspace(0, len(order) - 1, 24).astype(int)]

        def run():
            u = 0
            for i in sample:
                g = graphs[i]
                if wl["batch_kind"] == 1:
                    d = oracle.sssp(g.row_ptr, g.col, g.w, 0)
                    u += reached_edges(g, d != 0xFFFFFFFF)
                else:
                    lv = oracle.bfs(g.row_ptr, g.col, 0)
                    u += reached_edges(g, lv >= 0)
            return u
        unit, what = "GTEPS", f"24 of the 512 instances per step, spread over the size range"
    else:
        graphs = serving_graphs()
        qs = serving_queries(graphs, 64, seed=55)

        def run():
            for gi, kind, src in qs:
                g = graphs[gi]
                if kind == 1:
                    oracle.sssp(g.row_ptr, g.col, g.w, src)
                else:
                    oracle.bfs(g.row_ptr, g.col, src)
            return len(qs)
        unit, what = "queries/s", "64 queries per step, answered one after another"
    for _ in range(min(args.warmup, 1)):
        run()
    ts, units = [], 0
    steps = min(args.steps, 5)
    for _ in range(steps):
        t = time.perf_counter()
        units = run()
        ts.append(time.perf_counter() - t)
    total = sum(ts)
    value = steps * units / total / (1e9 if unit == "GTEPS" else 1.0)
    line = {"impl": "reference", "metric": f"{unit} ({args.workload})", "value": value, "unit": unit,
            "n_gpus": ws, "steps": steps, "warmup": args.warmup, "ms_per_step": total / steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": dict(wl["config"], l2="n/a (host)"),
            "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle", "sample": what},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(args, ws, rank, local, wl):
    import torch
    import oracle
    from paper_2201_02789_gb300 import nestpar as npb

    dev = torch.device("cuda", local)
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    bk = wl["batch_kind"]
    t_gen = time.perf_counter()
    specs, graphs = batch_inputs(bk)
    t_gen = time.perf_counter() - t_gen
    log(f"generated {len(graphs)} instances, {sum(g.m for g in graphs)} edges in {t_gen:.1f} s")
    ctx = npb.Context(local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.int8, device=dev)

    def upload():
        tens = []
        for g in graphs:
            rp = torch.from_numpy(g.row_ptr).to(dev, non_blocking=True)
            col = torch.from_numpy(g.col).to(dev, non_blocking=True)
            w = torch.from_numpy(g.w.view(np.int32)).to(dev, non_blocking=True) if bk == 1 else None
            tens.append((rp, col, w))
        return tens, [npb.make_csr(rp, col, w, n=g.n, m=g.m) for (rp, col, w), g in zip(tens, graphs)]

    tens, csrs = upload()
    torch.cuda.synchronize(dev)
    srcs = np.zeros(len(graphs), dtype=np.int32)
    b = npb.np_batch_create(ctx.handle, csrs, srcs, bk, npb.config("tca"))
    offs, total = npb.np_batch_layout(b, len(graphs))
    del tens, csrs
    torch.cuda.empty_cache()
    out = torch.empty((total,), dtype=torch.int32, device=dev)

    def timed(steps):
        return time_solves(lambda: npb.np_batch_run(b, out, stream=stream), steps, flush, stream)

    # untuned (every class on the library default), then the autotuner
    for _ in range(3):
        npb.np_batch_run(b, out, stream=stream)
    ms_default = statistics.median(timed(max(3, args.steps // 4)))
    t_tune = time.perf_counter()
    npb.np_batch_tune(b, out, reps=3, stream=stream)
    t_tune = time.perf_counter() - t_tune
    classes = npb.np_batch_classes(b)
    for _ in range(max(args.warmup, 3)):
        npb.np_batch_run(b, out, stream=stream)
    _, st = npb.np_batch_run(b, out, stream=stream, stats=True)
    res = out.cpu().numpy()
    res = res.view(np.uint32) if bk == 1 else res
    units = 0
    for i, g in enumerate(graphs):
        r = res[offs[i]:offs[i] + g.n]
        units += reached_edges(g, (r != 0xFFFFFFFF) if bk == 1 else (r >= 0))

    sampler = ClockSampler(local)
    sampler.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    sampler.mark("t0")
    ms = timed(args.steps)
    torch.cuda.synchronize(dev)
    sampler.mark("t1")
    if ws > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(ms), dev)
    value = job_value(ws, args.steps, units, total_ms)
    if rank != 0:
        npb.np_batch_destroy(b)
        ctx.close()
        torch.distributed.destroy_process_group()
        return

    # the same instances one solve after another through np_bfs / np_sssp (no batching)
    seq_ms = None
    if not args.only_headline:
        one = torch.empty((max(g.n for g in graphs),), dtype=torch.int32, device=dev)
        devg = []
        for g in graphs:
            rp = torch.from_numpy(g.row_ptr).to(dev)
            col = torch.from_numpy(g.col).to(dev)
            w = torch.from_numpy(g.w.view(np.int32)).to(dev) if bk == 1 else None
            devg.append((npb.make_csr(rp, col, w, n=g.n, m=g.m), rp, col, w))
        f = npb.np_sssp if bk == 1 else npb.np_bfs
        cfg = npb.config("tca")

        def seq():
            for c, *_ in devg:
                f(ctx.handle, c, 0, one, cfg, stream=stream)
        seq()
        seq_ms = statistics.median(time_solves(seq, 3, flush, stream))
        del devg
        torch.cuda.empty_cache()

    # parity on a sample of instances (the oracle, on host cores) and the CPU baseline
    order = np.argsort([g.n for g in graphs], kind="stable")
    sample = sorted({int(order[k]) for k in np.linspace(0, len(order) - 1, 16).astype(int)})
    t_cpu, cpu_units, parity = 0.0, 0, True
    for i in sample:
        g = graphs[i]
        t = time.perf_counter()
        ref = oracle.sssp(g.row_ptr, g.col, g.w, 0) if bk == 1 else oracle.bfs(g.row_ptr, g.col, 0)
        t_cpu += time.perf_counter() - t
        cpu_units += reached_edges(g, (ref != 0xFFFFFFFF) if bk == 1 else (ref >= 0))
        parity = parity and bool(np.array_equal(ref, res[offs[i]:offs[i] + g.n]))
    cpu = {"value": cpu_units / t_cpu / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
           "sample": f"{len(sample)} instances spread over the size range ({t_cpu:.1f} s)"}

    # end to end: host graphs in (pinned), batch build, one launch, results out
    pinned = [(torch.from_numpy(g.row_ptr).pin_memory(), torch.from_numpy(g.col).pin_memory(),
               torch.from_numpy(g.w.view(np.int32)).pin_memory() if bk == 1 else None) for g in graphs]
    out_h = torch.empty((total,), dtype=torch.int32).pin_memory()
    e2e_ms, parts = [], {"upload": [], "np_batch_create": [], "run_and_readback": []}
    for k in range(3):
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        dt = [(rp.to(dev, non_blocking=True), col.to(dev, non_blocking=True),
               w.to(dev, non_blocking=True) if w is not None else None) for rp, col, w in pinned]
        cs = [npb.make_csr(rp, col, w, n=g.n, m=g.m) for (rp, col, w), g in zip(dt, graphs)]
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        b2 = npb.np_batch_create(ctx.handle, cs, srcs, bk, npb.config("tca"))
        for ci, c in enumerate(classes):
            npb.np_batch_set_config(b2, ci, npb.np_config(**c["config"]))
        del dt, cs
        t2 = time.perf_counter()
        npb.np_batch_run(b2, out, stream=stream)
        out_h.copy_(out, non_blocking=True)
        torch.cuda.synchronize(dev)
        t3 = time.perf_counter()
        e2e_ms.append((t3 - t) * 1e3)
        for key, dtm in (("upload", t1 - t), ("np_batch_create", t2 - t1), ("run_and_readback", t3 - t2)):
            parts[key].append(dtm * 1e3)
        npb.np_batch_destroy(b2)
    h2d = sum(4 * (g.n + 1) + (8 if bk == 1 else 4) * g.m for g in graphs)
    e2e = {"value": units / (statistics.median(e2e_ms) * 1e-3) / 1e9, "unit": "GTEPS",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(4 * total),
           "ms_per_step": statistics.median(e2e_ms), "includes": "graph upload, np_batch_create (union copies, "
           "workspaces), tuned configs applied, one np_batch_run, result read-back",
           # np_batch_create allocates and fills the union copies every step: its share apart, and
           # the same figure without it (upload + one launch + read-back)
           "parts_ms": {k: statistics.median(v) for k, v in parts.items()},
           "value_without_create": units / ((statistics.median(parts["upload"]) +
                                             statistics.median(parts["run_and_readback"])) * 1e-3) / 1e9,
           "matches_device_result": bool(np.array_equal(out_h.numpy().view(res.dtype), res))}

    # algorithmic bytes (per instance, as the single-solve model) over the batch time
    kb = kernel_bytes("sssp" if bk == 1 else "bfs", st)
    peak, peak_kind = hbm_peak()
    med = statistics.median(ms)
    step_bytes = kb["solve"]
    groups = sum(c["groups"] for c in classes)
    per_iter = 2 * 4 + 1
    # per group: fill, seed, the small-level loop before the while loop (on by default)
    gpu_launches = int(args.steps * (3 * groups + st["graph_iterations"] * per_iter))
    line = {"metric": f"GTEPS and ms/batch ({args.workload}): 512 instances in one graph launch, autotuned per "
                      f"size class", "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": dict(wl["config"], edges=int(sum(g.m for g in graphs)), vertices_total=int(total),
                           l2="inputs (%.1f GB) larger than L2; also flushed between steps"
                              % (sum(g.m for g in graphs) * (8 if bk == 1 else 4) / 1e9)),
            "ms_per_batch": {"median": med, "min": min(ms)}, "units_per_batch": units,
            "untuned_ms_per_batch": ms_default, "tune_seconds": t_tune,
            "sequential_solves_ms": seq_ms,
            "speedup_vs_sequential": (seq_ms / med) if seq_ms else None,
            "classes": [{"log2_n": [c["log2_lo"], c["log2_lo"] + 2], "instances": c["instances"],
                         "groups": c["groups"], "edges": c["edges"], "tuned_ms": c["tuned_ms"],
                         "threshold": c["config"]["threshold"], "cfactor": c["config"]["cfactor"],
                         "child_block": c["config"]["child_block"],
                         "form": "nodp" if c["config"]["variant"] == 0 else "grid_host_aggregation",
                         "swept_frontier": c["config"]["sweep_parents"] > 0,
                         # the best device-launch granularity, timed outside the graph (not pickable)
                         "device_launch_ms": c["device_launch_ms"],
                         "device_launch_form": {2: "block", 3: "multiblock8", 4: "grid_device"}.get(
                             c["device_launch_granularity"], None),
                         "device_launch_threshold": c["device_launch_threshold"]}
                        for c in classes],
            "step_roofline": {"algorithmic_bytes": step_bytes, "achieved_gbs": step_bytes / (med * 1e-3) / 1e9,
                              "frac": step_bytes / (med * 1e-3) / 1e9 / peak, "peak": peak, "peak_kind": peak_kind},
            "cpu_baseline": cpu, "parity_vs_oracle_sample": parity, "e2e": e2e, "clocks": clocks,
            "gpu_launches": gpu_launches, "generation_seconds": t_gen}
    print(json.dumps(line), flush=True)
    npb.np_batch_destroy(b)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_serving(args, ws, rank, local, wl):
    import torch
    import oracle
    from paper_2201_02789_gb300 import nestpar as npb

    dev = torch.device("cuda", local)
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    graphs = serving_graphs()
    ctx = npb.Context(local)
    devs = []
    for g in graphs:
        rp = torch.from_numpy(g.row_ptr).to(dev)
        col = torch.from_numpy(g.col).to(dev)
        w = torch.from_numpy(g.w.view(np.int32)).to(dev)
        devs.append((npb.make_csr(rp, col, w, n=g.n, m=g.m), rp, col, w))
    lps = 2
    sv = npb.np_server_create(ctx.handle, [d[0] for d in devs], max_slots=64, levels_per_step=lps,
                              bfs_cfg=npb.config("tca"), sssp_cfg=npb.config("tca"))
    slots = {(gi, k): npb.np_server_pool_info(sv, gi, k) for gi in range(len(graphs)) for k in (0, 1)}

    def run_load(queries, arrivals):
        """Submits query q at arrivals[q] (s from the start; None = all at once), steps the
        server until every query is done; returns per-query latency (ms), wall time and steps."""
        outs, tick, t_done, by_ticket = {}, {}, {}, {}
        n = len(queries)
        t0 = time.perf_counter()
        nxt, steps = 0, 0
        live = set()
        while len(t_done) < n:
            now = time.perf_counter() - t0
            while nxt < n and (arrivals is None or arrivals[nxt] <= now):
                gi, kind, src = queries[nxt]
                outs[nxt] = torch.empty((graphs[gi].n,), dtype=torch.int32, device=dev)
                tick[nxt] = npb.np_server_submit(sv, gi, kind, src, outs[nxt])
                by_ticket[tick[nxt]] = nxt
                live.add(nxt)
                nxt += 1
            if not live:
                time.sleep(max(0.0, min(arrivals[nxt] - now, 0.001)) if arrivals is not None else 0)
                continue
            npb.np_server_step(sv)
            steps += 1
            t = time.perf_counter() - t0
            for tk in npb.np_server_finished(sv):
                q = by_ticket.pop(tk)
                t_done[q] = t
                live.discard(q)
                if q >= 24:          # keep a few results for the parity check
                    outs.pop(q)
        wall = time.perf_counter() - t0
        arr = np.zeros(n) if arrivals is None else np.asarray(arrivals)
        lat = np.array([(t_done[q] - arr[q]) * 1e3 for q in range(n)])
        return lat, wall, steps, outs

    # saturation: everything submitted at once (closed loop)
    warm = serving_queries(graphs, 64, seed=51)
    run_load(warm, None)
    sat_q = serving_queries(graphs, 512, seed=52)
    sampler = ClockSampler(local)
    sampler.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    sampler.mark("t0")
    lat_sat, wall_sat, steps_sat, outs = run_load(sat_q, None)
    torch.cuda.synchronize(dev)
    sampler.mark("t1")
    clocks = sampler.stop()
    # every rank served the same number of queries; the job took the slowest rank's time
    wall_job = max_over_ranks(wall_sat, dev)
    qps_sat = len(sat_q) / wall_sat
    qps_job = ws * len(sat_q) / wall_job
    # parity: the first retained results against the oracle, and alone (np_bfs / np_sssp) vs the mix
    parity = True
    alone_eq = True
    for q in sorted(outs)[:24]:
        gi, kind, src = sat_q[q]
        g = graphs[gi]
        got = outs[q].cpu().numpy()
        ref = oracle.sssp(g.row_ptr, g.col, g.w, src) if kind else oracle.bfs(g.row_ptr, g.col, src)
        parity = parity and bool(np.array_equal(got.view(np.uint32) if kind else got, ref))
        alone = torch.empty((g.n,), dtype=torch.int32, device=dev)
        (npb.np_sssp if kind else npb.np_bfs)(ctx.handle, devs[gi][0], src, alone, npb.config("tca"))
        alone_eq = alone_eq and bool(torch.equal(alone, outs[q]))
    loads = {}
    for frac in (0.5, 0.8, 0.95):
        nq = max(64, min(400, int(qps_sat * frac * 2.0)))
        qs = serving_queries(graphs, nq, seed=int(60 + frac * 100))
        arr = poisson_arrivals(qps_sat * frac, nq, seed=int(70 + frac * 100))
        lat, wall, steps, _ = run_load(qs, arr)
        loads[str(frac)] = {"offered_qps": qps_sat * frac, "achieved_qps": nq / wall, "queries": nq,
                            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                            "steps": steps}
    npb.np_server_destroy(sv)
    ctx.close()
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank != 0:
        return
    kernels_per_pool_step = 5 + 2 * lps
    line = {"metric": "queries/s at saturation and p50/p99 latency (serving): continuous batching of BFS/SSSP "
                      "queries over resident R-MAT graphs", "value": qps_job, "unit": "queries/s",
            "n_gpus": ws, "steps": steps_sat, "warmup": 1, "ms_per_step": wall_sat / steps_sat * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": dict(wl["config"], edges=int(sum(g.m for g in graphs)), levels_per_step=lps,
                           max_slots=64, l2="graphs (%.1f GB) larger than L2" % (
                               sum(g.m for g in graphs) * 8 / 1e9)),
            "saturation": {"queries": len(sat_q), "seconds": wall_sat, "p50_ms": float(np.percentile(lat_sat, 50)),
                           "p99_ms": float(np.percentile(lat_sat, 99))},
            "poisson": loads,
            "slots": {f"scale{16 + gi}_{'sssp' if k else 'bfs'}": slots[(gi, k)][0] for (gi, k) in slots},
            "parity_vs_oracle_sample": parity, "alone_equals_mix": alone_eq,
            "e2e": {"value": qps_job, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0, "note": "host-driven loop: every step ends in a host read-back"},
            "clocks": clocks, "gpu_launches_per_pool_step": kernels_per_pool_step}
    print(json.dumps(line), flush=True)


def sweep_variants(npb):
    """(name, config) of the variants the paper compares (Section VII): No CDP, plain CDP, T, C,
    T+C, A at every granularity with and without T and C, and the threshold sweep of T+C+A."""
    out = [("nodp", npb.config("nodp")), ("cdp", npb.config("cdp")), ("t", npb.config("t"))]
    out += [(f"c{cf}", npb.config("c", cfactor=cf)) for cf in (2, 4, 8, 16)]
    out += [("tc", npb.config("tc"))]
    grans = [("warp", dict(granularity="warp")), ("block", dict(granularity="block"))]
    grans += [(f"multiblock{gb}", dict(granularity="multiblock", group_blocks=gb)) for gb in (2, 4, 8, 16, 32)]
    grans += [("grid_device", dict(granularity="grid_device")), ("grid_host", dict(granularity="grid_host"))]
    for gname, kw in grans:
        out.append((f"a_{gname}", npb.config("a", **kw)))
        out.append((f"tca_{gname}", npb.config("tca", **kw)))
    out += [(f"tca_grid_host_T{1 << k}", npb.config("tca", threshold=1 << k)) for k in range(17)]
    out += [(f"tca_grid_host_C{cf}", npb.config("tca", cfactor=cf)) for cf in (1, 2, 8, 16)]
    # the dead-launch-code pair (Section VII-D): the same CTA-tiled parent kernel without and
    # with a launch site that never runs, driven the same way
    chunk = dict(driver=npb.NP_DRIVER_CHUNK)
    out += [("nodp_cta_no_launch_code", npb.config("nodp", granularity="none", **chunk)),
            ("cdp_threshold_above_max_degree", npb.config("cdp", threshold=npb.INT32_MAX, **chunk))]
    # the paper's forms append their frontiers (the library's swept frontier is its own default)
    return [(name, cfg.replace(sweep_parents=0)) for name, cfg in out]


def run_sweep(args, local, wl):
    """Every variant of the comparison on one workload: median ms/solve over a few solves,
    the device-side counters, and equality with the headline form's result."""
    import torch
    from paper_2201_02789_gb300 import build as nbuild
    from paper_2201_02789_gb300 import nestpar as npb
    nbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = npb.Context(local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.int8, device=dev)
    if wl["kind"] == "bezier":
        W = BezierWorkload(dev, stream, ctx, wl["config"]["curves"], wl["config"]["seed"])
    elif wl["kind"] == "tc":
        W = TcWorkload(dev, stream, ctx)
    else:
        W = GraphWorkload(wl["kind"], load_graph(wl["graph"]), dev, stream, ctx)
    head = npb.config("tca", **TUNED.get(args.workload, {}))
    W.solve(head)
    ref = W.result()
    units = W.units()
    only = set(args.variants.split(",")) if args.variants else None
    for name, cfg in sweep_variants(npb):
        if only is not None and name not in only:
            continue
        W.solve(cfg)
        reps = 2 if name in ("cdp", "t") or name.startswith("c") and not name.startswith("c_") else 5
        ms = statistics.median(time_solves(lambda: W.solve(cfg), reps, flush, stream))
        _, st = W.solve(cfg, stats=True)
        print(json.dumps({"workload": args.workload, "variant": name, "config": cfg.as_dict(), "ms_per_solve": ms,
                          "value": units / (ms * 1e-3) / 1e9, "unit": W.unit,
                          "device_launches": st["device_launches"], "launch_failures": st["launch_failures"],
                          "child_items": st["child_items"], "items": st["items"],
                          "matches_headline": bool(np.array_equal(W.result(), ref))}), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="sssp-rmat20")
    ap.add_argument("--cdp-steps", type=int, default=3, help="timed solves of the slow comparison forms")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="time every variant of the paper's comparison on the workload (one JSON line each)")
    ap.add_argument("--variants", default="", help="with --sweep: comma-separated variant names to run")
    ap.add_argument("--no-others", action="store_true",
                    help="default run: do not measure the other workloads after the headline")
    ap.add_argument("--only-headline", action="store_true",
                    help="headline form and three profile-mode solves only (for profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    wl = WORKLOADS[args.workload]
    if args.sweep:
        run_sweep(args, local, wl)
        return
    if wl["kind"] == "batched":
        run_batched(args, ws, rank, local, wl)
    elif wl["kind"] == "serving":
        run_serving(args, ws, rank, local, wl)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
