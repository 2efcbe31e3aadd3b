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
        d_bf, n_bf = bench.pipe_counts(p)
        d0, n0 = bench.pipe_counts(p, tested=0.0)
        for pipe in ("fp32", "xu", "int", "issue"):
            assert d_bf[pipe] >= 0 and n_bf[pipe] > 0
        # culling only removes indicator obstacle tests (6 fp32 per tested obstacle)
        if int(p["obs_mode"]) == 0 and int(p["risk_mask"]) & 4 and int(p["model"]) != 2:
            assert d_bf["fp32"] - d0["fp32"] == pytest.approx(6 * int(p["n_obs"]))
        else:
            assert d_bf == d0
        assert n0 == n_bf
    # the dynamic model's six Heun sub-steps dominate its count: 6 x (2 derivatives
    # of 48 fp32 + 7 special-function ops, + 18 for the trapezoid), plus the
    # heading wrap and the control terms once per control step
    dyn, _ = bench.pipe_counts(rs.preset("c2_closed_loop"), tested=0.0)
    kin, _ = bench.pipe_counts(rs.preset("c1_plain"), tested=0.0)
    assert dyn["fp32"] > 4 * kin["fp32"]
    assert bench._dyn_substep() == {"fp32": 114, "xu": 14, "int": 0}
    # paired FP32 halves the dynamics' share of the issue count only
    d1, _ = bench.pipe_counts(rs.preset("c5_stress"), tested=3.0, ilp=2, paired=False)
    d2, _ = bench.pipe_counts(rs.preset("c5_stress"), tested=3.0, ilp=2, paired=True)
    assert d1["fp32"] == d2["fp32"] and d1["issue"] - d2["issue"] == pytest.approx((6 * 114 + 4 + 1) / 2)


def test_pipe_roofline_picks_the_binding_pipe():
    import bench

    p = rs.preset("c5_stress")
    units = p["K"] * p["M"] * p["T"]
    rates = {"fp32": 128.0, "xu": 32.0, "issue": 128.0}
    bound, pipes = bench.pipe_roofline(p, units, 0.030, 3.0, 2, True, rates, 152, 2070.0)
    assert bound == max(("fp32", "xu", "issue"), key=lambda k: pipes[k]["frac"])
    for k in ("fp32", "xu", "issue"):
        assert pipes[k]["frac"] == pytest.approx(pipes[k]["achieved"] / pipes[k]["peak"])
    # twice the time, half of every fraction
    _, slow = bench.pipe_roofline(p, units, 0.060, 3.0, 2, True, rates, 152, 2070.0)
    assert slow["fp32"]["frac"] == pytest.approx(pipes["fp32"]["frac"] / 2)


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


def test_cpu_baseline_reports_all_cores_and_one():
    import bench

    p = rs.preset("c1_plain")
    obs = rs.scene_obstacles(p)
    x0 = rs.initial_state(int(p["model"]))
    V = rs.random_controls(int(p["model"]), int(p["T"]), p["u_lo"], p["u_hi"], 3)
    cb = bench.cpu_baseline(p, x0, V, obs, 2, 0.5)
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] > 0
    st = cb["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0 and st["unit"] == cb["unit"]
