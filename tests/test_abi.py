"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every
function include/nestpar.h declares, and the Python structures match the C
layouts (checked against gcc's sizeof/offsetof of the header itself)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2201_02789_gb300 import build as nbuild
from paper_2201_02789_gb300 import nestpar as npb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nestpar.h")


@pytest.fixture(scope="module")
def lib():
    nbuild.build()
    return npb.lib()


def declared_functions() -> list[str]:
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(np_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("np_create", "np_destroy", "np_bfs", "np_sssp", "np_bezier", "np_run_nested",
                     "np_workspace_size", "np_sync", "np_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    out = subprocess.run(["nm", "-D", "--defined-only", npb.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)
    assert set(npb.exported_symbols()) == set(names)
    # nothing but the C ABI leaks out of the library
    assert all(s.startswith("np_") for s in exported), sorted(s for s in exported if not s.startswith("np_"))[:5]


def test_struct_layouts_match_header(tmp_path):
    probe = tmp_path / "layout.c"
    probe.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "nestpar.h"
int main(void) {
  printf("np_config %zu %zu %zu\n", sizeof(np_config), offsetof(np_config, unroll), offsetof(np_config, reserved));
  printf("np_csr %zu %zu %zu\n", sizeof(np_csr), offsetof(np_csr, n), offsetof(np_csr, m));
  printf("np_stats %zu %zu %zu\n", sizeof(np_stats), offsetof(np_stats, timeouts), offsetof(np_stats, error));
  printf("np_parents %zu %zu %zu\n", sizeof(np_parents), offsetof(np_parents, ids), offsetof(np_parents, count));
  printf("np_body %zu %zu %zu\n", sizeof(np_body), offsetof(np_body, level), offsetof(np_body, cap));
  printf("np_profile %zu %zu %zu\n", sizeof(np_profile), offsetof(np_profile, levels), offsetof(np_profile, level_child_ms));
  printf("np_batch_options %zu %zu %zu\n", sizeof(np_batch_options), offsetof(np_batch_options, max_group_edges), offsetof(np_batch_options, config));
  printf("np_batch_class %zu %zu %zu\n", sizeof(np_batch_class), offsetof(np_batch_class, config), offsetof(np_batch_class, device_launch_threshold));
  printf("np_server_options %zu %zu %zu\n", sizeof(np_server_options), offsetof(np_server_options, levels_per_step), offsetof(np_server_options, sssp_config));
  printf("np_query_info %zu %zu %zu\n", sizeof(np_query_info), offsetof(np_query_info, slot), offsetof(np_query_info, finish_step));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)])
    rows = {l.split()[0]: [int(x) for x in l.split()[1:]] for l in subprocess.check_output([str(exe)], text=True).splitlines()}
    py = {
        "np_config": (npb.np_config, "unroll", "reserved"),
        "np_csr": (npb.np_csr, "n", "m"),
        "np_stats": (npb.np_stats, "timeouts", "error"),
        "np_parents": (npb.np_parents, "ids", "count"),
        "np_body": (npb.np_body, "level", "cap"),
        "np_profile": (npb.np_profile, "levels", "level_child_ms"),
        "np_batch_options": (npb.np_batch_options, "max_group_edges", "config"),
        "np_batch_class": (npb.np_batch_class, "config", "device_launch_threshold"),
        "np_server_options": (npb.np_server_options, "levels_per_step", "sssp_config"),
        "np_query_info": (npb.np_query_info, "slot", "finish_step"),
    }
    for name, (cls, f1, f2) in py.items():
        assert rows[name] == [ctypes.sizeof(cls), getattr(cls, f1).offset, getattr(cls, f2).offset], name


def test_host_only_entry_points(lib):
    assert npb.np_version() == 10200
    assert npb.np_status_string(npb.NP_ERR_INVALID) == "invalid argument"
    cfg = npb.np_config_default()
    assert (cfg.variant, cfg.threshold, cfg.cfactor, cfg.granularity, cfg.scan) == (1, 32, 4, npb.NP_GRAN_GRID_HOST, npb.NP_SCAN_ATOMIC)
    assert cfg.child_block == 64
    assert (cfg.small_parents, cfg.sweep_parents) == (npb.NP_SMALL_PARENTS_MAX, 4096)
    assert npb.np_workspace_size(1 << 20, cfg) > (1 << 20) * 16
    with pytest.raises(npb.NestparError):
        npb.np_workspace_size(-1, cfg)
    bad = cfg.replace(cfactor=3)
    with pytest.raises(npb.NestparError):
        npb.np_workspace_size(10, bad)


def test_host_argument_errors_of_new_entry_points(lib):
    """Argument checks that return before any device work (NULL handles, bad sizes)."""
    L = npb.lib()
    assert L.np_batch_destroy(None) == npb.NP_ERR_INVALID
    assert L.np_server_destroy(None) == npb.NP_ERR_INVALID
    assert L.np_server_step(None, None) == npb.NP_ERR_INVALID
    assert L.np_server_finished(None, None, 0, None) == npb.NP_ERR_INVALID
    assert L.np_batch_run(None, None, None, None) == npb.NP_ERR_INVALID
    assert L.np_batch_create(None, 0, None, None, None, None) == npb.NP_ERR_INVALID
    assert L.np_server_create(None, None, 0, None, None) == npb.NP_ERR_INVALID
    assert L.np_bfs_multi(None, None, 0, None, None, 0, None, None, None) == npb.NP_ERR_INVALID
    assert L.np_bfs_host_async(None, 0, 0, None, None, 0, None, None, None) == npb.NP_ERR_INVALID
    assert L.np_sssp_host_async(None, 1, 0, None, None, None, 0, None, None, None) == npb.NP_ERR_INVALID
    assert npb.multi_stride(1) == 1 and npb.multi_stride(4096) == 4096 and npb.multi_stride(4097) == 8192


def test_named_forms():
    f = {k: npb.config(k) for k in ("nodp", "cdp", "t", "c", "tc", "a", "ta", "ca", "tca")}
    assert f["nodp"].variant == npb.NP_VARIANT_NODP
    assert (f["cdp"].threshold, f["cdp"].cfactor, f["cdp"].granularity) == (0, 1, npb.NP_GRAN_NONE)
    assert f["tca"].granularity == npb.NP_GRAN_GRID_HOST and f["tca"].threshold == 32
    assert npb.config("tca", granularity="multiblock").granularity == npb.NP_GRAN_MULTIBLOCK


def test_create_without_gpu_reports_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(npb.NestparError):
        npb.np_create(0)
