"""The allocation-free tessellation entry point against the oracle and the regular one.

np_bezier_noalloc is for callers that cannot allocate device memory when they
call the library (all their device memory belongs to their own pool or a budget
fixed at start-up, or an allocation would stall a latency-critical loop). It
keeps its scratch in a static device array. These tests call it through the C
ABI twice in a row (the second call reuses the array the first one left behind)
and compare each call with the FP64 oracle (offsets bit for bit, points within
the tessellation tolerance used everywhere else: |g - r| <= 1e-5 * max(|r|, 1))
and with np_bezier on the same input. They also cover an empty input and a
capacity shortfall. This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes alone in a fresh
process.
"""
import numpy as np
import pytest
import torch

import oracle
from invariants import bezier_tolerance_ok
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


def _regular(ctx, c_d, nc, cap, cfg):
    off = torch.empty(nc + 1, dtype=torch.int32, device="cuda:0")
    pts = torch.zeros((cap, 2), dtype=torch.float32, device="cuda:0")
    npb.np_bezier(ctx.handle, c_d, nc, off, pts, cap, cfg, stats=True)
    return off.cpu().numpy(), pts.cpu().numpy()


def _noalloc(c_d, nc, cap, cfg, spare=0):
    """Runs the entry point into buffers of cap + spare points (NaN-filled)."""
    off = torch.full((nc + 1,), -7, dtype=torch.int32, device="cuda:0")
    pts = torch.full((cap + spare, 2), float("nan"), dtype=torch.float32, device="cuda:0")
    assert npb.np_bezier_noalloc(c_d, nc, off, pts, cap, cfg) == npb.NP_OK
    torch.cuda.synchronize()
    return off.cpu().numpy(), pts.cpu().numpy()


FORMS = [("tca", {}), ("tca", dict(scan=npb.NP_SCAN_ATOMIC, threshold=0, cfactor=2)),
         ("tca", dict(serial=npb.NP_SERIAL_BLOCK, parent_block=512)), ("nodp", {}),
         ("nodp", dict(granularity="none")),
         # every curve in its parent warp (the tessellation benchmark's form)
         ("tca", dict(threshold=npb.INT32_MAX, parent_block=512))]


@pytest.mark.parametrize("form,kw", FORMS, ids=["grid-host", "grid-host-atomic", "grid-host-cta-serial", "nodp",
                                                "nodp-cta-tiles", "grid-host-no-child"])
def test_noalloc_matches_oracle_and_np_bezier_two_calls(ctx, form, kw):
    cfg = npb.config(form, **kw)
    # first call: the largest input the static scratch allows; second call: a
    # different, smaller input on the array the first call left behind
    for nc, seed in ((npb.NP_NOALLOC_MAX_CURVES, 3), (5003, 41)):
        ctrl = gen.bezier_curves(nc, seed=seed)
        ref_off, ref_pts = oracle.bezier(ctrl)
        c_d = torch.from_numpy(ctrl).to("cuda:0")
        cap = nc * 200
        off, pts = _noalloc(c_d, nc, cap, cfg)
        np.testing.assert_array_equal(off, ref_off)
        total = int(ref_off[-1])
        assert total <= cap
        ok, worst = bezier_tolerance_ok(pts[:total], ref_pts)
        assert ok, worst
        reg_off, reg_pts = _regular(ctx, c_d, nc, cap, cfg)
        np.testing.assert_array_equal(off, reg_off)
        ok, worst = bezier_tolerance_ok(pts[:total], reg_pts[:total])
        assert ok, worst


def test_noalloc_empty_input():
    c_d = torch.zeros((1, 3, 2), dtype=torch.float32, device="cuda:0")
    off, _ = _noalloc(c_d, 0, 0, npb.config("tca"))
    assert off.tolist() == [0]


def test_noalloc_capacity_shortfall():
    """cap below the total: offsets are still exact, the total exceeds cap, and no point
    is written at or beyond cap (the curves that do not fit are skipped)."""
    nc = 3001
    ctrl = gen.bezier_curves(nc, seed=43)
    ref_off, ref_pts = oracle.bezier(ctrl)
    cap = int(ref_off[nc // 2]) + 17
    c_d = torch.from_numpy(ctrl).to("cuda:0")
    off, pts = _noalloc(c_d, nc, cap, npb.config("tca"), spare=4096)
    np.testing.assert_array_equal(off, ref_off)
    assert off[-1] > cap
    assert np.isnan(pts[cap:]).all()
    fit = int(np.searchsorted(ref_off[1:], cap, side="right"))   # curves that end within cap
    end = int(ref_off[fit])
    ok, worst = bezier_tolerance_ok(pts[:end], ref_pts[:end])
    assert ok, worst


def test_noalloc_rejects_what_it_cannot_run(ctx):
    c_d = torch.zeros((npb.NP_NOALLOC_MAX_CURVES + 1, 3, 2), dtype=torch.float32, device="cuda:0")
    off = torch.empty(npb.NP_NOALLOC_MAX_CURVES + 2, dtype=torch.int32, device="cuda:0")
    pts = torch.empty((16, 2), dtype=torch.float32, device="cuda:0")
    cfg = npb.config("tca")
    too_many = npb.np_bezier_noalloc(c_d, npb.NP_NOALLOC_MAX_CURVES + 1, off, pts, 16, cfg, check=False)
    assert too_many == npb.NP_ERR_INVALID
    device_launch = npb.np_bezier_noalloc(c_d, 10, off, pts, 16, npb.config("tca", granularity="block"), check=False)
    assert device_launch == npb.NP_ERR_UNSUPPORTED
    packed = npb.np_bezier_noalloc(c_d, 10, off, pts, 16, npb.config("tca", serial=npb.NP_SERIAL_PACKED),
                                   check=False)
    assert packed == npb.NP_ERR_UNSUPPORTED
    # the configuration checks of np_bezier
    for bad in (dict(agg_threshold=-1), dict(unroll=0), dict(driver=9), dict(serial=7)):
        assert npb.np_bezier_noalloc(c_d, 10, off, pts, 16, npb.config("tca", **bad),
                                     check=False) == npb.NP_ERR_INVALID
    cfg_res = npb.config("tca")
    cfg_res.reserved[0] = 1
    assert npb.np_bezier_noalloc(c_d, 10, off, pts, 16, cfg_res, check=False) == npb.NP_ERR_INVALID
