"""bench.py's host logic on the CPU: the formula count of the roofline, the
traffic record's tie to the kernel sources, and the reference arm's JSON
line (the FP64 oracle timed on the host, the same metric and config keys as
the GPU arm)."""

import json
import os
import subprocess
import sys

import pytest

import ra_scenes as rs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_formula_count_is_consistent():
    import bench

    for name in ("c1_plain", "c2_closed_loop", "c5_stress", "c4_gradient", "paper_sim", "linear_test"):
        p = rs.preset(name)
        d_bf, n_bf = bench.algorithmic_ops(p)
        d0, n0 = bench.algorithmic_ops(p, tested_obstacles=0.0)
        assert d_bf > 0 and n_bf > 0
        # culling only removes indicator obstacle tests (6 per tested obstacle)
        if int(p["obs_mode"]) == 0:
            assert d_bf - d0 == pytest.approx(6 * int(p["n_obs"]))
        else:
            assert d_bf == d0
        assert n0 == n_bf
    # the dynamic model's six Heun sub-steps dominate its count
    dyn, _ = bench.algorithmic_ops(rs.preset("c2_closed_loop"), tested_obstacles=0.0)
    kin, _ = bench.algorithmic_ops(rs.preset("c1_plain"), tested_obstacles=0.0)
    assert dyn > 4 * kin


def test_traffic_record_needs_matching_sources(monkeypatch):
    import bench

    rec = json.load(open(os.path.join(ROOT, "profiles", "rollout_cvar_c2.json")))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "not the recorded sources")
    assert bench.load_traffic("c2") is None
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: rec["source_sha"])
    assert bench.load_traffic("c2") == rec["dram_bytes_per_launch"] > 0
    assert bench.load_traffic("no_such_workload") is None


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c1",
                          "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == "rollout-steps/s (K*M*T)" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["warmup"] >= 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["K"] == 256 and line["config"]["M"] == 32
