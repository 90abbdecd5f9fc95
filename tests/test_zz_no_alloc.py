"""The allocation-free tessellation entry point against the regular one.

np_bezier_noalloc is for callers that cannot allocate device memory when they
call the library (for example while they capture a CUDA graph, or when all
device memory belongs to their own pool). It keeps its scratch in a static
device array. These tests call it through the C ABI twice in a row (the second
call reuses the array the first one left behind) and compare with np_bezier:
offsets bit for bit, points within the tessellation tolerance used everywhere
else (|g - r| <= 1e-5 * max(|r|, 1)). This file is collected last so that a
run stopping at the first failure has already run every other test; it also
passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

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


def _noalloc(c_d, nc, cap, cfg):
    off = torch.full((nc + 1,), -1, dtype=torch.int32, device="cuda:0")
    pts = torch.full((cap, 2), float("nan"), dtype=torch.float32, device="cuda:0")
    assert npb.np_bezier_noalloc(c_d, nc, off, pts, cap, cfg) == npb.NP_OK
    torch.cuda.synchronize()
    return off.cpu().numpy(), pts.cpu().numpy()


@pytest.mark.parametrize("form,kw", [("tca", {}), ("tca", dict(scan=npb.NP_SCAN_ATOMIC, threshold=0, cfactor=2)),
                                     ("nodp", {})], ids=["grid-host", "grid-host-atomic", "nodp"])
def test_noalloc_matches_np_bezier_two_calls(ctx, form, kw):
    cfg = npb.config(form, **kw)
    # first call: the largest input the static scratch allows; second call: a
    # different, smaller input on the array the first call left behind
    for nc, seed in ((npb.NP_NOALLOC_MAX_CURVES, 3), (5003, 41)):
        ctrl = gen.bezier_curves(nc, seed=seed)
        c_d = torch.from_numpy(ctrl).to("cuda:0")
        cap = nc * 200
        ref_off, ref_pts = _regular(ctx, c_d, nc, cap, cfg)
        off, pts = _noalloc(c_d, nc, cap, cfg)
        np.testing.assert_array_equal(off, ref_off)
        total = int(ref_off[-1])
        assert total <= cap
        ok, worst = bezier_tolerance_ok(pts[:total], ref_pts[:total])
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
