"""GPU parity: every form of the nested-parallel engine against the CPU oracle.

Integer work (BFS levels, SSSP distances, tessellation offsets) must match
bit for bit; tessellation points must satisfy |g - r| <= 1e-5 * max(|r|, 1)
against the FP64 oracle (FP32 evaluation of a quadratic with coefficients in
[0, 1] errs by a few ulp of 1, about 1e-7). Stats are checked where the
definition of the form fixes them (threshold above every degree: no launch;
plain CDP: one launch per parent with children).
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import DevGraph, bezier, bfs, form_grid, sssp
from invariants import (bezier_relative_error, bezier_tolerance_ok, check_bfs_levels, check_sssp_dist,
                        csr_from_edges)
from paper_2201_02789_gb300 import gen
from paper_2201_02789_gb300 import nestpar as npb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2201_02789_gb300 import build as nbuild
    nbuild.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = npb.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def g4k():
    g = gen.bfs4k()
    return g, DevGraph(g), oracle.bfs(g.row_ptr, g.col, 0), oracle.sssp(g.row_ptr, g.col, g.w, 0)


FORMS = form_grid()


@pytest.mark.parametrize("name,cfg", FORMS, ids=[f[0] for f in FORMS])
def test_bfs_sssp_all_forms_bitexact(ctx, g4k, name, cfg):
    g, dg, ref_l, ref_d = g4k
    lv, st = bfs(ctx, dg, 0, cfg, stats=True)
    np.testing.assert_array_equal(lv, ref_l)
    d, st2 = sssp(ctx, dg, 0, cfg, stats=True)
    np.testing.assert_array_equal(d, ref_d)
    for s in (st, st2):
        assert s["error"] == 0 and s["launch_failures"] == 0 and s["timeouts"] == 0
        if cfg.variant == npb.NP_VARIANT_NODP or cfg.threshold == npb.INT32_MAX:
            assert s["device_launches"] == 0
    reached = ref_l >= 0
    assert st["parents"] == reached.sum()
    assert st["items"] == np.diff(g.row_ptr)[reached].sum()
    if cfg.variant == npb.NP_VARIANT_CDP and cfg.granularity == npb.NP_GRAN_NONE and cfg.threshold <= 1:
        has_children = (np.diff(g.row_ptr)[reached] > 0).sum()
        assert st["launch_parents"] == has_children
        assert st["device_launches"] == has_children


EXTRA = [
    ("atomic-mb2", dict(granularity="multiblock", group_blocks=2, scan=npb.NP_SCAN_ATOMIC)),
    ("atomic-griddev", dict(granularity="grid_device", scan=npb.NP_SCAN_ATOMIC)),
    ("atomic-gridhost", dict(granularity="grid_host", scan=npb.NP_SCAN_ATOMIC, threshold=1)),
    ("aggthr-warp", dict(granularity="warp", agg_threshold=4, threshold=2)),
    ("aggthr-block", dict(granularity="block", agg_threshold=16, threshold=2)),
    ("child32", dict(child_block=32, threshold=1, cfactor=16)),
    ("child1024", dict(child_block=1024, threshold=1, cfactor=1)),
    ("parent64", dict(parent_block=64, granularity="multiblock", group_blocks=5)),
    ("parent512", dict(parent_block=512, granularity="grid_device")),
    ("grid1", dict(parent_grid=1, granularity="multiblock", group_blocks=2)),
    ("grid3-host", dict(parent_grid=3, threshold=1)),
    ("driver-host", dict(driver=npb.NP_DRIVER_HOST, granularity="block")),
    ("driver-chunk1", dict(driver=npb.NP_DRIVER_CHUNK, unroll=1, granularity="warp")),
    ("driver-chunk7", dict(driver=npb.NP_DRIVER_CHUNK, unroll=7)),
    ("driver-while1", dict(driver=npb.NP_DRIVER_WHILE, unroll=1)),
    ("driver-while16", dict(driver=npb.NP_DRIVER_WHILE, unroll=16, threshold=0)),
    ("nodp-host", dict(variant=npb.NP_VARIANT_NODP, driver=npb.NP_DRIVER_HOST)),
    ("persistent", dict(driver=npb.NP_DRIVER_PERSISTENT)),
    ("persistent-T1-C1", dict(driver=npb.NP_DRIVER_PERSISTENT, threshold=1, cfactor=1)),
    ("persistent-T0-C16", dict(driver=npb.NP_DRIVER_PERSISTENT, threshold=0, cfactor=16)),
    ("persistent-lb", dict(driver=npb.NP_DRIVER_PERSISTENT, scan=npb.NP_SCAN_LOOKBACK, threshold=4)),
    ("persistent-cb1024", dict(driver=npb.NP_DRIVER_PERSISTENT, child_block=1024, threshold=1)),
    ("persistent-pb512-cb128", dict(driver=npb.NP_DRIVER_PERSISTENT, parent_block=512, child_block=128,
                                    threshold=2)),
    ("persistent-pb384-cb256", dict(driver=npb.NP_DRIVER_PERSISTENT, parent_block=384, child_block=256,
                                    threshold=2)),
    ("persistent-nodp", dict(variant=npb.NP_VARIANT_NODP, driver=npb.NP_DRIVER_PERSISTENT)),
    ("persistent-grid1", dict(driver=npb.NP_DRIVER_PERSISTENT, parent_grid=1)),
    ("persistent-grid3-T1", dict(driver=npb.NP_DRIVER_PERSISTENT, parent_grid=3, threshold=1)),
    ("persistent-grid8-nodp", dict(variant=npb.NP_VARIANT_NODP, driver=npb.NP_DRIVER_PERSISTENT, parent_grid=8)),
    # children below the threshold packed into the child grid: CTA shapes, drivers, scans
    ("pack-pb64", dict(serial=npb.NP_SERIAL_PACKED, parent_block=64, threshold=8)),
    ("pack-pb512-cb32", dict(serial=npb.NP_SERIAL_PACKED, parent_block=512, child_block=32, threshold=64)),
    ("pack-cb1024", dict(serial=npb.NP_SERIAL_PACKED, child_block=1024, cfactor=1, threshold=16)),
    ("pack-cb512-lb", dict(serial=npb.NP_SERIAL_PACKED, child_block=512, scan=npb.NP_SCAN_LOOKBACK, threshold=256)),
    ("pack-grid1", dict(serial=npb.NP_SERIAL_PACKED, parent_grid=1, threshold=32)),
    ("pack-grid3-lb", dict(serial=npb.NP_SERIAL_PACKED, parent_grid=3, scan=npb.NP_SCAN_LOOKBACK, threshold=128)),
    ("pack-T1024-C16", dict(serial=npb.NP_SERIAL_PACKED, threshold=1024, cfactor=16)),
    ("pack-T1025", dict(serial=npb.NP_SERIAL_PACKED, threshold=1025)),
    ("pack-driver-host", dict(serial=npb.NP_SERIAL_PACKED, driver=npb.NP_DRIVER_HOST, threshold=32)),
    ("pack-driver-chunk3", dict(serial=npb.NP_SERIAL_PACKED, driver=npb.NP_DRIVER_CHUNK, unroll=3, threshold=32)),
    ("pack-driver-while1", dict(serial=npb.NP_SERIAL_PACKED, driver=npb.NP_DRIVER_WHILE, unroll=1, threshold=64)),
    # children below the threshold spread over the parent CTA
    ("block-pb64", dict(serial=npb.NP_SERIAL_BLOCK, parent_block=64, threshold=8)),
    ("block-pb512", dict(serial=npb.NP_SERIAL_BLOCK, parent_block=512, threshold=64)),
    ("block-pb96-lb", dict(serial=npb.NP_SERIAL_BLOCK, parent_block=96, scan=npb.NP_SCAN_LOOKBACK, threshold=4)),
    ("block-grid1", dict(serial=npb.NP_SERIAL_BLOCK, parent_grid=1, threshold=32)),
    ("block-grid3-lb", dict(serial=npb.NP_SERIAL_BLOCK, parent_grid=3, scan=npb.NP_SCAN_LOOKBACK, threshold=128)),
    ("block-never", dict(serial=npb.NP_SERIAL_BLOCK, threshold=npb.INT32_MAX)),
    ("block-driver-host", dict(serial=npb.NP_SERIAL_BLOCK, driver=npb.NP_DRIVER_HOST, threshold=32)),
    ("block-driver-while1", dict(serial=npb.NP_SERIAL_BLOCK, driver=npb.NP_DRIVER_WHILE, unroll=1)),
    # the swept frontier: drivers, the small-level loop around it, forms that fall back to the queue
    ("sweep-small", dict(sweep_parents=1)),
    ("sweep-small1", dict(sweep_parents=1, small_parents=1, unroll=1)),
    ("sweep-driver-host", dict(sweep_parents=1, driver=npb.NP_DRIVER_HOST, small_parents=0)),
    ("sweep-driver-chunk5", dict(sweep_parents=1, driver=npb.NP_DRIVER_CHUNK, unroll=5)),
    ("sweep-grid1-lb", dict(sweep_parents=1, parent_grid=1, scan=npb.NP_SCAN_LOOKBACK,
                            small_parents=0)),
    ("sweep-cb1024", dict(sweep_parents=1, child_block=1024, cfactor=1, small_parents=0)),
    ("sweep-persistent", dict(sweep_parents=1, driver=npb.NP_DRIVER_PERSISTENT)),
    ("sweep-block", dict(sweep_parents=1, serial=npb.NP_SERIAL_BLOCK, small_parents=0)),
    # levels above the limit sweep, the others append, in one solve
    ("sweep-mixed100", dict(sweep_parents=100, small_parents=0)),
    ("sweep-mixed400-lb-T4", dict(sweep_parents=400, small_parents=0, scan=npb.NP_SCAN_LOOKBACK, threshold=4)),
    ("spread-driver-while", dict(serial=npb.NP_SERIAL_SPREAD, driver=npb.NP_DRIVER_WHILE, threshold=32)),
    ("spread-grid3", dict(serial=npb.NP_SERIAL_SPREAD, parent_grid=3, threshold=16)),
]


@pytest.mark.parametrize("name,kw", EXTRA, ids=[e[0] for e in EXTRA])
def test_extra_settings_bitexact(ctx, g4k, name, kw):
    g, dg, ref_l, ref_d = g4k
    cfg = npb.config("tca", **kw)
    lv, st = bfs(ctx, dg, 0, cfg, stats=True)
    np.testing.assert_array_equal(lv, ref_l)
    d, st2 = sssp(ctx, dg, 0, cfg, stats=True)
    np.testing.assert_array_equal(d, ref_d)
    assert st["error"] == 0 and st2["error"] == 0


@pytest.mark.parametrize("driver", [npb.NP_DRIVER_WHILE, npb.NP_DRIVER_PERSISTENT])
def test_graph_drivers_refuse_device_launch_forms(ctx, g4k, driver):
    _, dg, _, _ = g4k
    level = torch.empty(dg.n, dtype=torch.int32, device="cuda:0")
    for gran in ("none", "block", "multiblock", "grid_device"):
        cfg = npb.config("tca", granularity=gran, driver=driver)
        assert npb.np_bfs(ctx.handle, dg.csr, 0, level, cfg, check=False) == npb.NP_ERR_UNSUPPORTED
    # the dead-launch-code baseline (NODP, CTA tiles) has no persistent loop either
    if driver == npb.NP_DRIVER_PERSISTENT:
        cfg = npb.config("nodp", granularity="none", driver=driver)
        assert npb.np_bfs(ctx.handle, dg.csr, 0, level, cfg, check=False) == npb.NP_ERR_UNSUPPORTED


# ------------------------------------------------------------------ edge cases

def _graph_from_edges(n, edges, ws=None):
    if edges:
        rp, col, w = csr_from_edges(n, edges, ws or [1 + (i * 37) % 255 for i in range(len(edges))])
    else:
        rp, col, w = np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint32)
    return gen.Csr(n, rp, col, w)


def _edge_graphs():
    out = {}
    out["single_vertex"] = _graph_from_edges(1, [])
    out["isolated_source"] = _graph_from_edges(5, [(1, 2), (2, 3), (3, 4)])
    # hub with a ragged degree well above a child grid: 70001 children
    hub = [(0, 1 + i) for i in range(70001)] + [(5, 0), (70001, 2)]
    out["hub"] = _graph_from_edges(70002, hub)
    # long path: thousands of levels through the level loop
    out["path"] = _graph_from_edges(3000, [(i, i + 1) for i in range(2999)])
    # duplicates and self-loops
    out["dups"] = _graph_from_edges(6, [(0, 1), (0, 1), (1, 1), (1, 2), (2, 0), (2, 3), (3, 3), (3, 4), (0, 4)])
    out["road"] = gen.road_grid(60, 70, seed=6)
    out["rmat12"] = gen.rmat(12, 8, seed=13)
    out["switch"] = _switch_graph()
    return out


def _switch_graph():
    """Levels that cross the one-CTA small-level loop's limits (1024 or 2048 parents,
    16384 children) in both directions, twice: a short path, a vertex with 20000
    children, a level of 20000 parents funnelling into 600, a path again, a fan-out of
    30000, a path, and a level of 1500 parents (above 1024, within 2048)."""
    rng = np.random.default_rng(77)
    edges = [(0, 1), (1, 2)]
    a0 = 3
    edges += [(2, a0 + i) for i in range(20000)]               # 1 parent, 20000 children
    b0 = a0 + 20000
    edges += [(a0 + i, b0 + int(rng.integers(0, 600))) for i in range(20000)]   # 20000 parents
    c0 = b0 + 600
    edges += [(b0 + i, c0) for i in range(600)]                 # 600 parents, 600 children
    edges += [(c0 + i, c0 + i + 1) for i in range(5)]           # path
    d0 = c0 + 6
    edges += [(c0 + 5, d0 + i) for i in range(30000)]           # 1 parent, 30000 children
    e0 = d0 + 30000
    edges += [(d0 + i, e0 + i % 40) for i in range(30000)]      # 30000 parents, 40 children each way
    edges += [(e0 + i, e0 + 40) for i in range(40)]
    edges += [(e0 + 40 + i, e0 + 41 + i) for i in range(8)]     # path
    f0 = e0 + 49
    edges += [(e0 + 48, f0 + i) for i in range(1500)]           # 1 parent, 1500 children
    edges += [(f0 + i, f0 + 1500 + i % 7) for i in range(1500)]  # 1500 parents: one thread, two parents
    edges += [(f0 + 1500 + i, f0 + 1507) for i in range(7)]
    n = f0 + 1508
    ws = [int(x) for x in rng.integers(1, 256, size=len(edges))]
    return _graph_from_edges(n, edges, ws)


EDGE = _edge_graphs()


@pytest.mark.parametrize("gname", list(EDGE))
@pytest.mark.parametrize("form", ["nodp", "cdp", "tc", "tca", "mb", "block", "persist", "persist-nodp",
                                  "tca-nosmall", "tca-small1", "tca-small1024", "tca-small33-cta", "tca-sweep"])
def test_edge_graphs(ctx, gname, form):
    g = EDGE[gname]
    kw = {"mb": dict(granularity="multiblock", group_blocks=2, threshold=4),
          "tca-nosmall": dict(small_parents=0),
          "tca-small1": dict(small_parents=1, unroll=1),
          "tca-small1024": dict(small_parents=1024),
          "tca-small33-cta": dict(small_parents=33, serial=npb.NP_SERIAL_BLOCK, unroll=3),
          "tca-sweep": dict(sweep_parents=1, small_parents=64),
          "block": dict(granularity="block", threshold=1, cfactor=2),
          "persist": dict(driver=npb.NP_DRIVER_PERSISTENT, threshold=2),
          "persist-nodp": dict(driver=npb.NP_DRIVER_PERSISTENT)}.get(form, {})
    base = {"persist": "tca", "persist-nodp": "nodp"}.get(form, form.split("-")[0])
    cfg = npb.config(base if base in ("nodp", "cdp", "tc", "tca") else "tca", **kw)
    dg = DevGraph(g)
    for src in sorted({0, g.n - 1, g.n // 2}):
        np.testing.assert_array_equal(bfs(ctx, dg, src, cfg), oracle.bfs(g.row_ptr, g.col, src))
        np.testing.assert_array_equal(sssp(ctx, dg, src, cfg), oracle.sssp(g.row_ptr, g.col, g.w, src))


def test_hand_worked_fixture(ctx, tiny_graph):
    rp, col, w, level, dist = tiny_graph
    dg = DevGraph(gen.Csr(7, rp, col, w))
    for form in ("nodp", "cdp", "tca"):
        np.testing.assert_array_equal(bfs(ctx, dg, 0, npb.config(form)), level)
        np.testing.assert_array_equal(sssp(ctx, dg, 0, npb.config(form)), dist)


def test_invalid_arguments(ctx, g4k):
    _, dg, _, _ = g4k
    level = torch.empty(dg.n, dtype=torch.int32, device="cuda:0")
    cfg = npb.config("tca")
    assert npb.np_bfs(ctx.handle, dg.csr, -1, level, cfg, check=False) == npb.NP_ERR_INVALID
    assert npb.np_bfs(ctx.handle, dg.csr, dg.n, level, cfg, check=False) == npb.NP_ERR_INVALID
    assert npb.np_bfs(ctx.handle, dg.csr, 0, None, cfg, check=False) == npb.NP_ERR_INVALID
    for bad in (dict(cfactor=3), dict(child_block=48), dict(parent_block=1024), dict(unroll=0),
                dict(granularity=9), dict(granularity="multiblock", group_blocks=0)):
        assert npb.np_bfs(ctx.handle, dg.csr, 0, level, cfg.replace(**bad), check=False) == npb.NP_ERR_INVALID
    nw = npb.make_csr(dg.row_ptr, dg.col, None, n=dg.n, m=dg.m)
    assert npb.np_sssp(ctx.handle, nw, 0, level, cfg, check=False) == npb.NP_ERR_INVALID


def test_repeat_and_context_reuse(ctx, g4k):
    g, dg, ref_l, ref_d = g4k
    other = gen.rmat(13, 16, seed=17)
    dgo = DevGraph(other)
    ref_o = oracle.sssp(other.row_ptr, other.col, other.w, 3)
    for _ in range(3):
        for cfg in (npb.config("tca"), npb.config("cdp"), npb.config("tca", granularity="multiblock")):
            np.testing.assert_array_equal(bfs(ctx, dg, 0, cfg), ref_l)
            np.testing.assert_array_equal(sssp(ctx, dgo, 3, cfg), ref_o)
            np.testing.assert_array_equal(sssp(ctx, dg, 0, cfg), ref_d)


# ---------------------------------------------------------------- tessellation

BT_FORMS = [("nodp", {}), ("cdp", {}), ("t", {}), ("tc", {}), ("tca", {}),
            ("tca", dict(granularity="block")), ("tca", dict(granularity="warp", threshold=8)),
            ("tca", dict(granularity="multiblock", group_blocks=4, cfactor=2)),
            ("tca", dict(granularity="grid_device", scan=npb.NP_SCAN_ATOMIC)),
            ("tca", dict(granularity="grid_host", threshold=0, cfactor=16, child_block=64)),
            ("tca", dict(threshold=npb.INT32_MAX)),
            ("tca", dict(serial=npb.NP_SERIAL_SPREAD)),
            ("tca", dict(serial=npb.NP_SERIAL_PACKED, threshold=1024, scan=npb.NP_SCAN_LOOKBACK, parent_block=512,
                         child_block=32)),
            ("tca", dict(serial=npb.NP_SERIAL_PACKED, threshold=200, child_block=1024, cfactor=1)),
            ("tca", dict(serial=npb.NP_SERIAL_BLOCK, threshold=64)),
            ("tca", dict(serial=npb.NP_SERIAL_BLOCK, threshold=npb.INT32_MAX, parent_block=64,
                         scan=npb.NP_SCAN_LOOKBACK)),
            # serialised curves of 32 points or more run with the whole parent warp, the rest spread
            # over its lanes: every curve in the parent warps, or all three kinds in one pass
            ("tca", dict(threshold=npb.INT32_MAX, parent_block=512)),
            ("tca", dict(threshold=npb.INT32_MAX, parent_block=64, scan=npb.NP_SCAN_LOOKBACK)),
            ("tca", dict(threshold=40, child_block=32)),
            ("tca", dict(threshold=1024, cfactor=2))]


@pytest.mark.parametrize("form,kw", BT_FORMS, ids=[f"{f}-{i}" for i, (f, _) in enumerate(BT_FORMS)])
def test_bezier_forms(ctx, form, kw):
    ctrl = gen.bezier_curves(3000, seed=31)
    ref_off, ref_pts = oracle.bezier(ctrl)
    status, off, pts, st = bezier(ctx, ctrl, npb.config(form, **kw))
    assert status == npb.NP_OK
    np.testing.assert_array_equal(off, ref_off)
    ok, worst = bezier_tolerance_ok(pts[: ref_off[-1]], ref_pts)
    assert ok, worst
    assert st["items"] == ref_off[-1] and st["parents"] == 3000


def _curves_around_a_warp():
    """Curves with exactly 31, 32 and 33 points and the longest of a large random draw,
    interleaved, so that a warp tile holds some of each."""
    pool = gen.bezier_curves(40000, seed=35)
    n = np.diff(oracle.bezier_offsets(pool))
    pick = [np.flatnonzero(n == k)[:40] for k in (31, 32, 33)] + [np.argsort(n)[-40:]]
    idx = np.stack([p[:min(len(q) for q in pick)] for p in pick], 1).reshape(-1)
    return np.ascontiguousarray(pool[idx]), n[idx]


@pytest.mark.parametrize("kw", [dict(threshold=npb.INT32_MAX), dict(threshold=33), dict(threshold=32),
                                dict(threshold=npb.INT32_MAX, parent_block=512, scan=npb.NP_SCAN_LOOKBACK)],
                         ids=["never", "T33", "T32", "never-pb512-lookback"])
def test_bezier_whole_warp_curves(ctx, kw):
    ctrl, counts = _curves_around_a_warp()
    assert {31, 32, 33} <= set(counts.tolist()) and counts.max() > 1000
    ref_off, ref_pts = oracle.bezier(ctrl)
    status, off, pts, st = bezier(ctx, ctrl, npb.config("tca", **kw))
    assert status == npb.NP_OK and st["error"] == 0
    np.testing.assert_array_equal(off, ref_off)
    ok, worst = bezier_tolerance_ok(pts[: ref_off[-1]], ref_pts)
    assert ok, worst
    assert st["items"] == ref_off[-1]
    launching = int((counts >= kw["threshold"]).sum()) if kw["threshold"] != npb.INT32_MAX else 0
    assert st["launch_parents"] == launching and st["serial_parents"] == len(counts) - launching
    if launching == 0:
        # a threshold that launches nothing: no child grid runs at all
        assert st["child_blocks"] == 0 and st["child_items"] == 0


@pytest.mark.parametrize("pb", [64, 128, 512])
@pytest.mark.parametrize("nc", [1, 33, 3001])
def test_bezier_offset_groups_of_any_size(ctx, pb, nc):
    """The output offsets are scanned per CTA group of tiles (2 to 16 warps): ragged curve
    counts leave the last group partial and some warps past the last tile."""
    ctrl = gen.bezier_curves(nc, seed=33)
    ref_off, ref_pts = oracle.bezier(ctrl)
    for scan in (npb.NP_SCAN_ATOMIC, npb.NP_SCAN_LOOKBACK):
        status, off, pts, st = bezier(ctx, ctrl, npb.config("tca", parent_block=pb, scan=scan))
        assert status == npb.NP_OK and st["error"] == 0
        np.testing.assert_array_equal(off, ref_off)
        ok, worst = bezier_tolerance_ok(pts[: ref_off[-1]], ref_pts)
        assert ok, worst


def test_bezier_hand_counts_on_gpu(ctx):
    from conftest import read_golden
    rows = read_golden("bezier_counts.txt")["rows"]
    ctrl = np.array([[float(x) for x in r[:6]] for r in rows], np.float32).reshape(-1, 3, 2)
    status, off, pts, _ = bezier(ctx, ctrl, npb.config("tca"))
    assert status == npb.NP_OK
    np.testing.assert_array_equal(np.diff(off), [int(r[6]) for r in rows])


def _tie_curves():
    """Curves on the 2^-24 grid whose exact t = 64 (S/C)^(1/4) is an integer m (P0 = (0, m^2),
    P1 = (4096, 0), P2 = (8192, m^2) in units of 2^-24), and the same with the apex moved by
    one unit either way (t within about 1/m^2 of m)."""
    rows = []
    for m in (3, 4, 5, 17, 64, 100, 1000, 4095, 4096):
        for d in (0, -1, 1):
            y = m * m + d
            if not 0 <= y < (1 << 24):
                continue
            rows.append([0, y, 4096, 0, 8192, y])
    return np.array(rows, np.float64).astype(np.float32).reshape(-1, 3, 2) * np.float32(2.0 ** -24)


@pytest.mark.parametrize("form", ["tca", "nodp"])
def test_bezier_counts_at_ties_and_off_grid(ctx, form):
    """The point count takes an exact integer path for coordinates on the 2^-24 grid and the
    FP64 sequence elsewhere and at near-ties; both must give the oracle's FP64 counts."""
    ties = _tie_curves()
    u = gen.uniform_f64(77, 1, 0, 600 * 6)
    off_grid = np.concatenate([
        ((u[:1800] - 0.5) * 6.0).astype(np.float32),          # negative and > 1 coordinates
        (u[1800:] * 0.3 + 0.1).astype(np.float32)]).reshape(-1, 3, 2)   # values off the 2^-24 grid
    straight = np.array([[[0.25, 0.25], [0.5, 0.5], [0.75, 0.75]], [[0.5, 0.5]] * 3,
                         [[0.0, 0.0], [0.0, 0.5], [0.0, 0.0]]], np.float32)
    for ctrl in (ties, off_grid, straight, np.concatenate([ties, gen.bezier_curves(300, seed=78)])):
        status, off, pts, _ = bezier(ctx, ctrl, npb.config(form))
        assert status == npb.NP_OK
        np.testing.assert_array_equal(off, oracle.bezier_offsets(ctrl))


def test_bezier_capacity_and_empty(ctx):
    ctrl = gen.bezier_curves(200, seed=32)
    ref_off, ref_pts = oracle.bezier(ctrl)
    cap = int(ref_off[100])            # room for the first 100 curves only
    status, off, pts, st = bezier(ctx, ctrl, npb.config("tca"), cap=cap, check=False)
    assert status == npb.NP_ERR_CAPACITY
    np.testing.assert_array_equal(off, ref_off)
    ok, _ = bezier_tolerance_ok(pts[:cap], ref_pts[:cap])
    assert ok
    status, off, _, _ = bezier(ctx, np.zeros((0, 3, 2), np.float32), npb.config("tca"))
    assert status == npb.NP_OK and off[0] == 0


# ------------------------------------------------------------ one nesting pass

def test_run_nested_bfs_levels(ctx, g4k):
    g, dg, ref_l, _ = g4k
    dev = "cuda:0"
    level = torch.full((g.n,), -1, dtype=torch.int32, device=dev)
    level[0] = 0
    cur = torch.tensor([0], dtype=torch.int32, device=dev)
    host_level = np.full(g.n, -1, np.int32)
    host_level[0] = 0
    host_cur = np.array([0], np.int32)
    L = 0
    while host_cur.size:
        nxt = torch.empty(g.n, dtype=torch.int32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int32, device=dev)
        body = npb.np_body(kind=npb.NP_BODY_BFS_VISIT, next_level=L + 1, level=level.data_ptr(),
                           next=nxt.data_ptr(), next_count=cnt.data_ptr())
        parents = npb.np_parents(cur.data_ptr(), cur.shape[0])
        cfg = npb.config("tca", granularity=["grid_host", "multiblock", "block", "none"][L % 4], threshold=2)
        npb.np_run_nested(ctx.handle, parents, npb.NP_COUNT_CSR_DEGREE, dg.csr, body, cfg)
        got = np.sort(nxt[: int(cnt.item())].cpu().numpy())
        ref = np.sort(oracle.bfs_expand(g.row_ptr, g.col, host_cur, L, host_level))
        np.testing.assert_array_equal(got, ref)
        host_cur, cur, L = ref, nxt[: int(cnt.item())].clone(), L + 1
    np.testing.assert_array_equal(level.cpu().numpy(), ref_l)


def test_run_nested_sssp_pass_sandwich(ctx):
    """One chaotic relaxation pass lies between the synchronous pass and the
    final distances, and appends exactly the vertices whose distance dropped."""
    g = gen.rmat(12, 16, seed=19)
    dg = DevGraph(g)
    final = oracle.sssp(g.row_ptr, g.col, g.w, 0)
    rng = np.random.default_rng(4)
    dist0 = final.astype(np.int64) + rng.integers(0, 40, g.n)
    dist0 = np.where(final == 0xFFFFFFFF, 0xFFFFFFFF, dist0).astype(np.uint32)
    dist0[0] = 0
    frontier = np.nonzero(dist0 != 0xFFFFFFFF)[0].astype(np.int32)[::3].copy()
    dev = "cuda:0"
    d_dist = torch.from_numpy(dist0.view(np.int32).copy()).to(dev)
    stamp = torch.full((g.n,), -1, dtype=torch.int32, device=dev)
    nxt = torch.empty(g.n, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    fr = torch.from_numpy(frontier).to(dev)
    body = npb.np_body(kind=npb.NP_BODY_SSSP_RELAX, iteration=1, dist=d_dist.data_ptr(), stamp=stamp.data_ptr(),
                       next=nxt.data_ptr(), next_count=cnt.data_ptr())
    npb.np_run_nested(ctx.handle, npb.np_parents(fr.data_ptr(), len(frontier)), npb.NP_COUNT_CSR_DEGREE, dg.csr,
                      body, npb.config("tca", threshold=8))
    got = d_dist.cpu().numpy().view(np.uint32)
    sync = oracle.sssp_relax_pass(g.row_ptr, g.col, g.w, frontier, dist0)
    assert np.all(got <= sync) and np.all(got >= final)
    pushed = np.sort(nxt[: int(cnt.item())].cpu().numpy())
    np.testing.assert_array_equal(pushed, np.nonzero(got < dist0)[0])


def test_run_nested_bezier_subset(ctx):
    ctrl = gen.bezier_curves(1000, seed=33)
    ids = np.arange(999, -1, -7, dtype=np.int32)       # reversed, strided subset
    ref_counts = np.array([oracle.bezier_count(ctrl[i]) for i in ids])
    dev = "cuda:0"
    c_d = torch.from_numpy(ctrl).to(dev)
    off = torch.empty(len(ids) + 1, dtype=torch.int32, device=dev)
    cap = int(ref_counts.sum())
    pts = torch.empty((cap, 2), dtype=torch.float32, device=dev)
    idt = torch.from_numpy(ids).to(dev)
    body = npb.np_body(kind=npb.NP_BODY_BEZIER_EVAL, ctrl=c_d.data_ptr(), offsets=off.data_ptr(),
                       points=pts.data_ptr(), cap=cap)
    npb.np_run_nested(ctx.handle, npb.np_parents(idt.data_ptr(), len(ids)), npb.NP_COUNT_BEZIER, None, body,
                      npb.config("tca", threshold=64))
    o = off.cpu().numpy()
    np.testing.assert_array_equal(np.diff(o), ref_counts)
    p = pts.cpu().numpy()
    for k in range(0, len(ids), 11):
        N = ref_counts[k]
        for j in (0, N // 2, N - 1):
            ref = oracle.bezier_point(ctrl[ids[k]], N, j)
            assert bezier_tolerance_ok(p[o[k] + j], ref)[0]


# ------------------------------------------------------------ full-size configs

@pytest.fixture(scope="module")
def rmat20():
    g = gen.rmat20()
    return g, DevGraph(g)


@pytest.mark.parametrize("form", ["tca", "nodp", "tca-mb", "tca-atomic", "tca-persistent", "nodp-persistent",
                                  "tca-block", "tca-packed", "tca-block-lookback", "tca-sweep",
                                  "tca-sweep-nosmall", "tca-sweep-mixed"])
def test_rmat20_sssp_bfs_full(ctx, rmat20, form):
    g, dg = rmat20
    kw = {"tca-mb": dict(granularity="multiblock", group_blocks=8),
          "tca-atomic": dict(scan=npb.NP_SCAN_ATOMIC),
          "tca-block": dict(serial=npb.NP_SERIAL_BLOCK),
          "tca-packed": dict(serial=npb.NP_SERIAL_PACKED),
          "tca-block-lookback": dict(serial=npb.NP_SERIAL_BLOCK, scan=npb.NP_SCAN_LOOKBACK, threshold=256),
          "tca-sweep": dict(sweep_parents=1),
          "tca-sweep-nosmall": dict(sweep_parents=1, small_parents=0),
          "tca-sweep-mixed": dict(sweep_parents=100000, small_parents=0),
          "tca-persistent": dict(driver=npb.NP_DRIVER_PERSISTENT),
          "nodp-persistent": dict(driver=npb.NP_DRIVER_PERSISTENT)}.get(form, {})
    cfg = npb.config(form.split("-")[0], **kw)
    ref_l = oracle.bfs(g.row_ptr, g.col, 0)
    np.testing.assert_array_equal(bfs(ctx, dg, 0, cfg), ref_l)
    d, st = sssp(ctx, dg, 0, cfg, stats=True)
    np.testing.assert_array_equal(d, oracle.sssp(g.row_ptr, g.col, g.w, 0))
    assert st["error"] == 0


def test_rmat20_plain_cdp_full(ctx, rmat20):
    g, dg = rmat20
    lv, st = bfs(ctx, dg, 0, npb.config("cdp"), stats=True)
    np.testing.assert_array_equal(lv, oracle.bfs(g.row_ptr, g.col, 0))
    assert st["device_launches"] + st["launch_failures"] == st["launch_parents"]


def test_bt64k_full(ctx):
    """Full size, offsets exact and points within the scaled tolerance; the strict relative
    error where |r| >= 1e-3 is reported. FP32 evaluation of B(t) errs by a few units of
    2^-24 of the largest term (coordinates in [0, 1]), about 1e-7 absolute, so a coordinate
    near 1e-3 can be off by about 1e-4 relative: the bound asserted there is the absolute
    one, 16 * 2^-24 (about 1e-6), divided by |r|."""
    ctrl = gen.bt64k()
    ref_off, ref_pts = oracle.bezier(ctrl)
    status, off, pts, st = bezier(ctx, ctrl, npb.config("tca"), cap=int(ref_off[-1]))
    assert status == npb.NP_OK
    np.testing.assert_array_equal(off, ref_off)
    ok, worst = bezier_tolerance_ok(pts, ref_pts)
    assert ok, worst
    err = np.abs(pts.astype(np.float64) - ref_pts)
    assert err.max() <= 16 * 2.0 ** -24, err.max()
    rel = bezier_relative_error(pts, ref_pts, 1e-3)
    print(f"bt64k: max |g - r| = {err.max():.3e}, max relative error where |r| >= 1e-3: {rel:.3e}")
    assert rel <= 16 * 2.0 ** -24 / 1e-3


def test_bt256k_full(ctx):
    """262,144 curves (about 25 M points, more than L2 holds) in the benchmark's setting:
    offsets exact, points within the tolerance."""
    import bench
    ctrl = gen.bezier_curves(262144, seed=3)
    ref_off, ref_pts = oracle.bezier(ctrl)
    status, off, pts, st = bezier(ctx, ctrl, npb.config("tca", **bench.TUNED["bt256k"]), cap=int(ref_off[-1]))
    assert status == npb.NP_OK and st["error"] == 0
    np.testing.assert_array_equal(off, ref_off)
    ok, worst = bezier_tolerance_ok(pts, ref_pts)
    assert ok, worst


def test_bench_tuned_configs_full(ctx, g4k):
    """The configurations bench.py times where they differ from the library default (BT-64K
    with 512-thread parent CTAs, 32-thread child blocks, CF 4 and the serial children spread
    over the parent CTA; the SSSP setting, the swept frontier, runs in test_rmat20_sssp_bfs_full
    and the triangle-counting one in its own tests), and the 4096-vertex graph on the
    persistent loop with 8 CTAs, at full size, against the oracle."""
    import bench
    cfg = npb.config("tca", **bench.TUNED["bt64k"])
    ctrl = gen.bt64k()
    ref_off, ref_pts = oracle.bezier(ctrl)
    status, off, pts, st = bezier(ctx, ctrl, cfg, cap=int(ref_off[-1]))
    assert status == npb.NP_OK and st["error"] == 0
    np.testing.assert_array_equal(off, ref_off)
    ok, worst = bezier_tolerance_ok(pts, ref_pts)
    assert ok, worst
    g, dg, ref_l, ref_d = g4k
    cfg = npb.config("tca", driver=npb.NP_DRIVER_PERSISTENT, parent_grid=8)
    lv, st = bfs(ctx, dg, 0, cfg, stats=True)
    np.testing.assert_array_equal(lv, ref_l)
    d, st2 = sssp(ctx, dg, 0, cfg, stats=True)
    np.testing.assert_array_equal(d, ref_d)
    assert st["error"] == 0 and st2["error"] == 0


# ------------------------------------------------------------------ stress

@pytest.mark.parametrize("scan", [npb.NP_SCAN_LOOKBACK, npb.NP_SCAN_ATOMIC], ids=["lookback", "atomic"])
def test_multiblock_repeated_runs(ctx, scan):
    """Group counters and accumulators are reset by each group's last block;
    repeated solves on alternating graphs and group sizes must stay exact."""
    graphs = [gen.bfs4k(), gen.rmat(13, 12, seed=23)]
    devs = [DevGraph(g) for g in graphs]
    refs = [(oracle.bfs(g.row_ptr, g.col, 0), oracle.sssp(g.row_ptr, g.col, g.w, 0)) for g in graphs]
    for rep in range(6):
        for gi, (dg, (rl, rd)) in enumerate(zip(devs, refs)):
            cfg = npb.config("tca", granularity="multiblock", group_blocks=1 + (rep + gi) % 4, scan=scan,
                             threshold=[8, 32, 128][rep % 3], child_block=[32, 256][gi])
            np.testing.assert_array_equal(bfs(ctx, dg, 0, cfg), rl)
            np.testing.assert_array_equal(sssp(ctx, dg, 0, cfg), rd)


# ------------------------------------------------------------ bounded waits

@pytest.mark.parametrize("which,limit_ns", [(0, 0), (1, 50_000_000)])
def test_bounded_waits_time_out_and_context_survives(ctx, g4k, which, limit_ns):
    """A look-back whose predecessor never publishes, and a grid barrier one CTA never
    reaches, both give up with NP_ERR_TIMEOUT; the next solve on the context is exact."""
    import time
    g, dg, ref_l, ref_d = g4k
    t = time.perf_counter()
    assert npb.np_selftest_wait(ctx.handle, which, limit_ns) == npb.NP_ERR_TIMEOUT
    assert time.perf_counter() - t < 30.0
    np.testing.assert_array_equal(bfs(ctx, dg, 0, npb.config("tca")), ref_l)
    cfg = npb.config("tca", driver=npb.NP_DRIVER_PERSISTENT)
    d, st = sssp(ctx, dg, 0, cfg, stats=True)
    np.testing.assert_array_equal(d, ref_d)
    assert st["error"] == 0
