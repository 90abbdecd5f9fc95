"""Host-side checks of bench.py: the reference arm (the CPU oracle) and the
replica timing of a multi-rank job, run as two gloo ranks on the CPU."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run_bench(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          env=env, timeout=600)


def test_reference_arm_prints_one_json_line():
    r = _run_bench({}, "--impl", "reference", "--workload", "bfs4k", "--steps", "2", "--warmup", "3")
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "cpu_baseline", "e2e", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_other_ranks_stay_silent():
    r = _run_bench({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--impl", "reference", "--workload", "bfs4k",
                   "--steps", "1", "--warmup", "3")
    assert r.returncode == 0 and r.stdout.strip() == ""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _replica(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [12.0, 20.0][rank]
    mx = bench.max_over_ranks(local_ms)
    q.put((rank, mx, bench.job_value(world, 10, 1_000_000, mx)))
    dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [20.0, 20.0]
    # 2 ranks x 10 steps x 1e6 units in 20 ms = 1.0 G units/s
    assert out[0][2] == pytest.approx(1.0)


def test_traffic_is_reported_only_for_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    """A committed ncu summary counts only while its source hash is the current one."""
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "child_agg_w.md").write_text(
        "# x\n\n- kernel: child_agg\n- traffic_bytes_per_launch: 1234\n- source_hash: abc\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda: "abc")
    assert bench.ncu_traffic("child_agg", "w") == 1234.0
    monkeypatch.setattr(bench, "source_hash", lambda: "def")
    assert bench.ncu_traffic("child_agg", "w") is None
    assert bench.ncu_traffic("parent_warp", "w") is None   # no summary at all


def test_source_hash_follows_every_kernel_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2201_02789_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cuh").write_text("int a;\n")
    (csrc / "notes.txt").write_text("ignored\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.source_hash()
    (csrc / "notes.txt").write_text("still ignored\n")
    assert bench.source_hash() == h0
    (csrc / "b.cu").write_text("int b;\n")
    h1 = bench.source_hash()
    assert h1 != h0
    (csrc / "a.cuh").write_text("int a2;\n")
    assert bench.source_hash() not in (h0, h1)


def test_poisson_arrivals_are_seeded_and_have_the_offered_rate():
    a = bench.poisson_arrivals(500.0, 20000, seed=5)
    assert np.array_equal(a, bench.poisson_arrivals(500.0, 20000, seed=5))
    assert not np.array_equal(a, bench.poisson_arrivals(500.0, 20000, seed=6))
    gaps = np.diff(np.concatenate([[0.0], a]))
    assert (gaps > 0).all()
    # exponential gaps: mean 1/rate, coefficient of variation 1 (20,000 samples: within 3%)
    assert abs(gaps.mean() * 500.0 - 1.0) < 0.03
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.03


def test_other_workloads_of_the_default_run():
    """Every workload the default run adds is a bench workload other than the headline, run with
    a one-solve CPU leg (which keeps the oracle check) and without recursing into further runs;
    compact() keeps the figures a reader checks and drops the rest."""
    names = [n for n, _ in bench.OTHER_WORKLOADS]
    assert len(set(names)) == len(names) and "sssp-rmat20" not in names
    assert set(names) == set(bench.WORKLOADS) - {"sssp-rmat20"}
    line = {"metric": "m", "value": 2.0, "unit": "GTEPS", "ms_per_step": 1.5, "gpu_launches": 10,
            "roofline": {"kernel": "child_agg", "achieved": 1.0, "peak": 2.0, "frac": 0.5, "traffic": None,
                         "avg_launch_ms": 0.1},
            "step_roofline": {"frac": 0.25, "algorithmic_bytes": 3},
            "e2e": {"value": 1.0, "unit": "GTEPS", "h2d_bytes_per_step": 4, "d2h_bytes_per_step": 5, "mode": "x"},
            "parity_vs_oracle": True, "forms": {"nodp": {}}, "clocks": {"sm_mhz": 2070.0}}
    c = bench.compact(line)
    assert c["value"] == 2.0 and c["roofline"]["frac"] == 0.5 and "avg_launch_ms" not in c["roofline"]
    assert c["step_roofline_frac"] == 0.25 and c["e2e"]["h2d_bytes_per_step"] == 4 and "mode" not in c["e2e"]
    assert c["parity_vs_oracle"] is True and "forms" not in c and c["clocks"]["sm_mhz"] == 2070.0
