"""Build options that select another code path than the default, built and checked
against the oracle.

NP_TMA_STAGE=1 stages each aggregated child block's edge lists in shared memory
with the bulk-copy engine (cp.async.bulk into an mbarrier), one block ahead.
NP_PDL=0 launches the level loop's kernels without programmatic dependent
launch; NP_FILTER_L1=0 reads the child items' filter values through L2 only.
Each variant library is built in-tree beside the default one and exercised in
its own process by tests/option_check.py, bit-exact against the oracle.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
OPTIONS = {"tma_stage": ("NP_TMA_STAGE=1",), "no_pdl_l2_filter": ("NP_PDL=0", "NP_FILTER_L1=0")}


@pytest.mark.parametrize("name", list(OPTIONS))
def test_build_option_matches_oracle(name):
    from paper_2201_02789_gb300 import build
    lib = build.build(defines=OPTIONS[name], out_dir=os.path.join(build.BUILD, "opt_" + name))
    env = dict(os.environ, NESTPAR_LIB=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "option_check.py")], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-4000:], r.stderr[-4000:])
    assert "mismatches: []" in r.stdout
