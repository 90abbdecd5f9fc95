"""GPU tests of the host-buffer entry points and of the execution-time breakdown.

np_bfs_host / np_sssp_host / np_bezier_host copy host inputs in and results
out on the caller's stream; their results must equal the oracle's. The
breakdown (np_profile_*) must describe the solve it times: one record per
level, the first level holding the source, frontier sizes summing to the
solve's frontier pops.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import DevGraph
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


@pytest.mark.parametrize("form", ["tca", "nodp", "cdp"])
def test_graph_host_entry_points(ctx, form):
    cfg = npb.config(form)
    for g, src in ((gen.bfs4k(), 0), (gen.rmat(12, 8, seed=91), 7), (gen.road_grid(20, 30, seed=6), 599)):
        lv = np.full(g.n, 9, np.int32)
        _, st = npb.np_bfs_host(ctx.handle, g.row_ptr, g.col, src, lv, cfg, stats=True)
        np.testing.assert_array_equal(lv, oracle.bfs(g.row_ptr, g.col, src))
        assert st["error"] == 0
        d = np.full(g.n, 9, np.uint32)
        npb.np_sssp_host(ctx.handle, g.row_ptr, g.col, g.w, src, d, cfg)
        np.testing.assert_array_equal(d, oracle.sssp(g.row_ptr, g.col, g.w, src))


def test_graph_host_entry_edge_cases(ctx):
    one = gen.Csr(1, np.zeros(2, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint32))
    lv = np.full(1, 9, np.int32)
    npb.np_bfs_host(ctx.handle, one.row_ptr, one.col, 0, lv, npb.config("tca"))
    assert lv.tolist() == [0]
    d = np.full(1, 9, np.uint32)
    npb.np_sssp_host(ctx.handle, one.row_ptr, one.col, one.w, 0, d, npb.config("tca"))
    assert d.tolist() == [0]
    g = gen.bfs4k()
    bad = np.zeros(g.n, np.int32)
    assert npb.np_bfs_host(ctx.handle, g.row_ptr, g.col, g.n, bad, npb.config("tca"), check=False) == \
        npb.NP_ERR_INVALID


def test_async_host_entry_points_on_two_contexts(ctx):
    """The stream-ordered host calls on two contexts and two streams, issued back to back so
    that one context's copies can overlap the other's solve, over graphs of different sizes
    (the staging buffers grow between calls): every result equals the oracle's and np_sync
    reports no device error."""
    ctx2 = npb.Context(0)
    try:
        ctxs, streams = [ctx, ctx2], [torch.cuda.Stream(), torch.cuda.Stream()]
        graphs = [(gen.rmat(14, 8, seed=93), 3), (gen.bfs4k(), 0), (gen.road_grid(30, 20, seed=7), 11),
                  (gen.rmat(12, 16, seed=94), 0), (gen.rmat(15, 4, seed=95), 5)]
        bufs = []
        for g, _ in graphs:
            pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            bufs.append((pin(g.row_ptr), pin(g.col), pin(g.w.view(np.int32)),
                         torch.full((g.n,), 9, dtype=torch.int32).pin_memory(),
                         torch.full((g.n,), 9, dtype=torch.int32).pin_memory()))
        cfg = npb.config("tca")
        for rep in range(2):
            for k, ((g, src), (rp, col, w, lv, d)) in enumerate(zip(graphs, bufs)):
                c, s = ctxs[(k + rep) % 2], streams[(k + rep) % 2]
                npb.np_bfs_host_async(c.handle, rp, col, src, lv, cfg, stream=s)
                npb.np_sssp_host_async(c.handle, rp, col, w, src, d, cfg, stream=s)
            for c, s in zip(ctxs, streams):
                s.synchronize()
                _, st = npb.np_sync(c.handle, stream=s)
                assert st["error"] == 0
            for (g, src), (rp, col, w, lv, d) in zip(graphs, bufs):
                np.testing.assert_array_equal(lv.numpy(), oracle.bfs(g.row_ptr, g.col, src))
                np.testing.assert_array_equal(d.numpy().view(np.uint32), oracle.sssp(g.row_ptr, g.col, g.w, src))
                lv.fill_(9)
                d.fill_(9)
    finally:
        ctx2.close()


def test_async_host_entry_points_pageable_and_degenerate(ctx):
    """The stream-ordered calls with pageable numpy buffers (the runtime copies synchronously)
    and on a single vertex without edges; argument errors come back at once."""
    s = torch.cuda.Stream()
    g = gen.rmat(12, 8, seed=96)
    lv = np.full(g.n, 9, np.int32)
    d = np.full(g.n, 9, np.uint32)
    npb.np_bfs_host_async(ctx.handle, g.row_ptr, g.col, 5, lv, npb.config("tca"), stream=s)
    npb.np_sssp_host_async(ctx.handle, g.row_ptr, g.col, g.w, 5, d, npb.config("tca"), stream=s)
    s.synchronize()
    assert npb.np_sync(ctx.handle, stream=s)[1]["error"] == 0
    np.testing.assert_array_equal(lv, oracle.bfs(g.row_ptr, g.col, 5))
    np.testing.assert_array_equal(d, oracle.sssp(g.row_ptr, g.col, g.w, 5))
    one = gen.Csr(1, np.zeros(2, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint32))
    lv1, d1 = np.full(1, 9, np.int32), np.full(1, 9, np.uint32)
    npb.np_bfs_host_async(ctx.handle, one.row_ptr, one.col, 0, lv1, npb.config("tca"), stream=s)
    npb.np_sssp_host_async(ctx.handle, one.row_ptr, one.col, one.w, 0, d1, npb.config("tca"), stream=s)
    s.synchronize()
    assert lv1.tolist() == [0] and d1.tolist() == [0]
    assert npb.np_bfs_host_async(ctx.handle, g.row_ptr, g.col, g.n, lv, npb.config("tca"), stream=s,
                                 check=False) == npb.NP_ERR_INVALID


@pytest.mark.parametrize("form", ["tca", "nodp"])
def test_bezier_host_entry_point(ctx, form):
    ctrl = gen.bezier_curves(700, seed=92)
    ref_off, ref_pts = oracle.bezier(ctrl)
    total = int(ref_off[-1])
    off = np.zeros(701, np.int32)
    pts = np.full((total, 2), np.nan, np.float32)
    _, st = npb.np_bezier_host(ctx.handle, ctrl, 700, off, pts, total, npb.config(form), stats=True)
    np.testing.assert_array_equal(off, ref_off)
    assert np.all(np.abs(pts - ref_pts) <= 1e-5 * np.maximum(np.abs(ref_pts), 1.0))
    # too small an output: the offsets stay complete and the status says so
    off2 = np.zeros(701, np.int32)
    pts2 = np.zeros((total // 2, 2), np.float32)
    s = npb.np_bezier_host(ctx.handle, ctrl, 700, off2, pts2, total // 2, npb.config(form), check=False)
    assert s == npb.NP_ERR_CAPACITY
    np.testing.assert_array_equal(off2, ref_off)
    # no curves
    off3 = np.full(1, 5, np.int32)
    npb.np_bezier_host(ctx.handle, np.zeros((0, 3, 2), np.float32), 0, off3, np.zeros((1, 2), np.float32), 0,
                       npb.config(form))
    assert off3.tolist() == [0]


@pytest.mark.parametrize("kind", ["bfs", "sssp"])
def test_profile_breakdown_describes_the_solve(ctx, kind):
    g = gen.rmat(14, 16, seed=93)
    dg = DevGraph(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda:0")
    npb.np_profile_enable(ctx.handle, True)
    try:
        npb.np_profile_read(ctx.handle, reset=True)
        f = npb.np_bfs if kind == "bfs" else npb.np_sssp
        _, st = f(ctx.handle, dg.csr, 0, out, npb.config("tca"), stats=True)
        prof = npb.np_profile_read(ctx.handle, reset=True)
    finally:
        npb.np_profile_enable(ctx.handle, False)
    ref = oracle.bfs(g.row_ptr, g.col, 0) if kind == "bfs" else oracle.sssp(g.row_ptr, g.col, g.w, 0)
    got = out.cpu().numpy()
    np.testing.assert_array_equal(got.view(np.uint32) if kind == "sssp" else got, ref)
    levels = prof["levels"]
    assert levels >= st["levels"] >= 1
    lp = list(prof["level_parents"])[:levels]
    assert lp[0] == 1                                  # the source
    assert sum(lp) == st["parents"]                    # every frontier pop is in one level's record
    assert prof["parent_launches"] == levels and prof["child_launches"] == levels
    assert prof["parent_ms"] > 0 and prof["child_ms"] > 0
    assert prof["longest_level_ms"] <= prof["parent_ms"] + prof["child_ms"]
    if kind == "bfs":
        assert lp[1:st["levels"]] == [int((ref == L).sum()) for L in range(1, st["levels"])]
