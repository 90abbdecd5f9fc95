"""Benchmark of the nested-parallel hot path on one GB300 (or N replicas).

Workload: single-source shortest paths by frontier Bellman-Ford on a seeded
R-MAT graph, scale 20 (1,048,576 vertices), edge factor 16 (16,777,216 edges),
a,b,c,d = .57/.19/.19/.05, uint32 weights uniform in [1, 255], source 0. One
step = one whole solve (every level of the nested parent/child work) through
the C ABI, graph resident in HBM. Between timed steps L2 is flushed (a 512 MB
write) outside the timed events.

The headline is the aggregated form (threshold + coarsening + grid aggregation);
plain CDP (one device launch per parent) and the no-dynamic-parallelism form
are timed beside it on the same GPU. GTEPS = edges out of reached vertices /
solve time (Graph500 convention).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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
sys.path.insert(0, os.path.join(ROOT, "tests"))

import numpy as np  # noqa: E402

METRIC = "GTEPS and ms/solve at 1 GB300: aggregated form vs plain CDP; % HBM roofline"
WORKLOAD = "sssp-rmat20"
CONFIG = {"workload": "sssp_frontier_bellman_ford_rmat_scale20", "vertices": 1 << 20, "edges": 16 << 20,
          "rmat_abcd": [0.57, 0.19, 0.19, 0.05], "weights": "uint32 uniform [1,255]", "source": 0,
          "seed": 2, "l2": "flushed between timed steps (512 MB write)"}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_graph():
    from paper_2201_02789_gb300 import gen
    cache = os.path.join(ROOT, "_cache")
    path = os.path.join(cache, "rmat20_seed2.npz")
    if os.path.exists(path):
        z = np.load(path)
        return gen.Csr(int(z["n"]), z["row_ptr"], z["col"], z["w"])
    g = gen.rmat20()
    try:
        os.makedirs(cache, exist_ok=True)
        np.savez(path + ".tmp.npz", n=g.n, row_ptr=g.row_ptr, col=g.col, w=g.w)
        os.replace(path + ".tmp.npz", path)
    except OSError:
        pass
    return g


def reached_edges(g, dist) -> int:
    reached = np.asarray(dist) != 0xFFFFFFFF
    return int(np.diff(g.row_ptr.astype(np.int64))[reached].sum())


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


def ncu_traffic(kernel: str) -> float | None:
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if it was
    taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{WORKLOAD}.md")
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


def sssp_kernel_bytes(st: dict) -> dict:
    """Algorithmic bytes of the SSSP path, split by kernel.

    Parent grid: per frontier pop the id, the row_ptr pair and dist[u] (16 B);
    per serialised relaxation col + w + dist[v] (12 B); per launching parent a
    16 B record and a 4 B block offset; per frontier append 4 B.
    Child grid: per relaxation col + w + dist[v] (12 B); per launching parent the
    record, offset and dist[u] it reads back (24 B)."""
    serial_items = st["items"] - st["child_items"]
    parent = 16 * st["parents"] + 12 * serial_items + 20 * st["launch_parents"] + 4 * st["pushes"]
    child = 12 * st["child_items"] + 24 * st["launch_parents"]
    return {"parent": parent, "child": child, "solve": 16 * st["parents"] + 12 * st["items"]}


# ------------------------------------------------------------------ arms

def run_reference(args, ws, rank):
    """The oracle (serial Dijkstra) on the host cores, as the reference arm."""
    if rank != 0:
        return
    import oracle
    g = load_graph()
    for _ in range(args.warmup):
        d = oracle.sssp(g.row_ptr, g.col, g.w, 0)
    ts = []
    for _ in range(args.steps):
        t = time.perf_counter()
        d = oracle.sssp(g.row_ptr, g.col, g.w, 0)
        ts.append(time.perf_counter() - t)
    mr = reached_edges(g, d)
    total = sum(ts)
    value = args.steps * mr / total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": CONFIG,
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full Dijkstra solves of the workload"},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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


def run_ours(args, ws, rank, local):
    import torch
    from paper_2201_02789_gb300 import build as nbuild
    from paper_2201_02789_gb300 import nestpar as npb
    from gpu_util import DevGraph

    nbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    distributed = ws > 1
    if distributed:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    g = load_graph()
    dg = DevGraph(g, device=dev)
    ctx = npb.Context(local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.int8, device=dev)
    dist_t = torch.empty(g.n, dtype=torch.int32, device=dev)
    cfg = npb.config("tca")

    def solve(c=cfg):
        npb.np_sssp(ctx.handle, dg.csr, 0, dist_t, c, stream=stream)

    for _ in range(max(args.warmup, 3)):
        solve()
    _, st = npb.np_sssp(ctx.handle, dg.csr, 0, dist_t, cfg, stream=stream, stats=True)
    d_gpu = dist_t.cpu().numpy().view(np.uint32)
    mr = reached_edges(g, d_gpu)

    sampler = ClockSampler(local)
    sampler.start()
    if distributed:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    sampler.mark("t0")
    ms = time_solves(solve, args.steps, flush, stream)
    torch.cuda.synchronize(dev)
    sampler.mark("t1")
    if distributed:
        torch.distributed.barrier()
    clocks = sampler.stop()
    total_ms = sum(ms)
    if distributed:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = ws * args.steps * mr / (total_ms * 1e-3) / 1e9
    ms_per_step = total_ms / args.steps

    if rank != 0:
        if distributed:
            torch.distributed.destroy_process_group()
        return

    # kernels launched per solve (while driver): init + per body iteration
    # `unroll` x (parent, child) + the condition kernel
    per_solve = 1 + st["graph_iterations"] * (2 * cfg.unroll + 1)
    gpu_launches = int(per_solve * args.steps)

    if args.only_headline:
        # small run for profiler captures: the headline form, then profile-mode solves
        npb.np_profile_enable(ctx.handle, True)
        for _ in range(3):
            flush.zero_()
            npb.np_sssp(ctx.handle, dg.csr, 0, dist_t, cfg, stream=stream, stats=True)
        npb.np_profile_enable(ctx.handle, False)
        print(json.dumps({"metric": METRIC, "value": value, "unit": "GTEPS", "ms_per_step": ms_per_step,
                          "gpu_launches": gpu_launches, "only_headline": True}), flush=True)
        ctx.close()
        return

    # forms beside the headline, same GPU, same input
    forms = {}
    for name, c, reps in (("plain_cdp", npb.config("cdp"), args.cdp_steps),
                          ("nodp", npb.config("nodp"), args.cdp_steps),
                          ("t_c", npb.config("tc"), args.cdp_steps),
                          ("t_c_a_multiblock", npb.config("tca", granularity="multiblock", group_blocks=8), 5),
                          ("t_c_a_grid_device", npb.config("tca", granularity="grid_device"), 5)):
        solve(c)
        t = time_solves(lambda c=c: solve(c), reps, flush, stream)
        m = statistics.median(t)
        forms[name] = {"ms_per_solve": m, "gteps": mr / (m * 1e-3) / 1e9}
    torch.cuda.synchronize(dev)

    # roofline of the dominant kernel: profile mode (separate launches, CUDA events)
    npb.np_profile_enable(ctx.handle, True)
    npb.np_profile_read(ctx.handle, reset=True)
    prof_runs = 3
    for _ in range(prof_runs):
        flush.zero_()
        _, pst = npb.np_sssp(ctx.handle, dg.csr, 0, dist_t, cfg, stream=stream, stats=True)
    prof = npb.np_profile_read(ctx.handle, reset=True)
    npb.np_profile_enable(ctx.handle, False)
    kb = sssp_kernel_bytes(pst)
    peak, peak_kind = hbm_peak()
    kernels = {"child_agg": (prof["child_ms"], prof["child_launches"], kb["child"]),
               "parent_kernel": (prof["parent_ms"], prof["parent_launches"], kb["parent"])}
    dom = max(kernels, key=lambda k: kernels[k][0])
    k_ms, k_launches, k_bytes = kernels[dom]
    per_launch_bytes = k_bytes * prof_runs / max(k_launches, 1)
    avg_ms = k_ms / max(k_launches, 1)
    achieved = per_launch_bytes / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": ncu_traffic(dom),
                "kernel": dom, "peak_kind": f"{peak_kind} (copy bandwidth, burst)",
                "avg_launch_ms": avg_ms, "algorithmic_bytes_per_launch": per_launch_bytes,
                "share_of_profiled_time": k_ms / max(prof["parent_ms"] + prof["child_ms"] + prof["other_ms"], 1e-9)}
    solve_bytes = kb["solve"]
    step_roofline = {"algorithmic_bytes": solve_bytes, "achieved_gbs": solve_bytes / (ms_per_step * 1e-3) / 1e9,
                     "frac": solve_bytes / (ms_per_step * 1e-3) / 1e9 / peak}

    # end to end through the C ABI from pinned host buffers
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    col_h = torch.from_numpy(g.col).pin_memory()
    w_h = torch.from_numpy(g.w.view(np.int32)).pin_memory()
    out_h = torch.empty(g.n, dtype=torch.int32).pin_memory()
    e2e_ms = []
    for k in range(args.e2e_steps + 1):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        npb.np_sssp_host(ctx.handle, rp_h, col_h, w_h, 0, out_h, cfg, stream=stream)
        dt = (time.perf_counter() - t) * 1e3
        if k:
            e2e_ms.append(dt)
    e2e_ok = bool(np.array_equal(out_h.numpy().view(np.uint32), d_gpu))
    e2e = {"value": mr / (statistics.median(e2e_ms) * 1e-3) / 1e9, "unit": "GTEPS",
           "h2d_bytes_per_step": int(4 * (g.n + 1) + 8 * g.m), "d2h_bytes_per_step": int(4 * g.n),
           "ms_per_step": statistics.median(e2e_ms), "matches_device_result": e2e_ok}

    # CPU baseline: the oracle as it stands, one core, bounded sample; also the parity check
    cpu = None
    parity = None
    if ws == 1 and not args.no_cpu:
        import oracle
        ts = []
        ref = None
        t_end = time.perf_counter() + args.cpu_seconds
        while time.perf_counter() < t_end or not ts:
            t = time.perf_counter()
            ref = oracle.sssp(g.row_ptr, g.col, g.w, 0)
            ts.append(time.perf_counter() - t)
        parity = bool(np.array_equal(ref, d_gpu))
        cpu = {"value": mr / statistics.mean(ts) / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
               "sample": f"{len(ts)} full Dijkstra solves of the workload ({sum(ts):.1f} s)",
               "ms_per_solve": statistics.mean(ts) * 1e3}

    line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": CONFIG,
            "form": "threshold 32 + coarsening 8 (32-thread child blocks) + grid aggregation (atomic scan), "
                    "while-graph level loop",
            "ms_per_solve": {"median": statistics.median(ms), "min": min(ms)},
            "edges_reached": mr, "levels": st["levels"], "relaxations": st["items"],
            "speedup_vs_plain_cdp": forms["plain_cdp"]["ms_per_solve"] / statistics.median(ms),
            "speedup_vs_nodp": forms["nodp"]["ms_per_solve"] / statistics.median(ms),
            "forms": forms, "roofline": roofline, "step_roofline": step_roofline,
            "cpu_baseline": cpu, "parity_vs_oracle": parity, "e2e": e2e, "clocks": clocks,
            "gpu_launches": gpu_launches, "profile_breakdown": prof}
    print(json.dumps(line), flush=True)
    ctx.close()
    if distributed:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cdp-steps", type=int, default=3, help="timed solves of the slow comparison forms")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--only-headline", action="store_true",
                    help="headline form and three profile-mode solves only (for profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
