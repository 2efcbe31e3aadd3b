"""Benchmark of the RA-MPPI control update on GB300.

Metric: rollout-steps/s, one rollout-step being one disturbed step of one
of the K x M rollouts (K M T per update); the K T nominal steps are extra
work that is not counted.  A "step" of this benchmark is one complete
update (sampling, nominal and disturbed rollouts, CVaR, softmin update) on
the paper-scale closed-loop workload: dynamic single-track vehicle,
K = 4096 samples, M = 128 disturbed rollouts, T = 40 steps, 50 obstacles.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own instance (seed + rank): weak scaling,
no collective on the data path.  `--impl reference` times the FP64 CPU
oracle on the host cores over bounded samples of the same workload.
"""

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ra_scenes as rs  # noqa: E402

WORKLOADS = {
    "c2": "c2_closed_loop",
    "c1": "c1_plain",
    "c5": "c5_stress",
    "c4": "c4_gradient",
    "paper": "paper_sim",
}
N_SMS = 152
LANES_PER_SM = 128


# ---------------------------------------------------------------- op counts
def algorithmic_ops(p, tested_obstacles=None):
    """Formula count of ALU lane-operations per disturbed step and per nominal
    step: FP32 add/mul/FMA/min/max/compare/select and INT32 ops count 1 each,
    every special-function evaluation (sin, cos, tan, atan, atan2, log, exp,
    sqrt, rsqrt, division) counts 1.  The indicator obstacle term of a
    disturbed step counts the obstacles actually tested (`tested_obstacles`
    per rollout-step, after the kernel's exact bounding-box cull) when given,
    else all of them."""
    model, n_obs, sub = int(p["model"]), int(p["n_obs"]), int(p["substeps"])
    philox = 100  # 10 rounds x (2 mullo + 2 mulhi + 4 xor + 2 key adds)
    n_test = n_obs if tested_obstacles is None else tested_obstacles
    obs_ind = 6 * n_test  # 2 sub, mul, fma, compare-select, add
    obs_sp = 10 * n_obs  # 2 sub, mul, fma, sqrt, sub, mul, exp, log1p, add
    obs = obs_ind if int(p["obs_mode"]) == 0 else obs_sp
    if model == 1:
        deriv = 38  # slip angles 7, two tyres 10, sincos 2, six derivatives 19
        dyn = sub * (2 * deriv + 6 + 12)
        # mixture: per slot the tail mass (3), ln, the Laplace value (1), the
        # Gaussian radius and angle (sqrt, cos, 4), select and sign (2)
        noise = (2 * philox + 3 * 12) if int(p["noise_type"]) == 1 else (philox + 2 * 10 + 3)
    elif model == 0:
        dyn = sub * 7
        noise = philox + 2 * 10 + 4
    else:
        dyn, noise = sub, philox + 10 + 1
    risk = 1 + obs
    disturbed = dyn + noise + risk
    # nominal: control draw (Philox + Box-Muller + clip ~ 120), dynamics, full q
    # (the nominal rollout tests every obstacle)
    nominal = 120 + dyn + (6 * n_obs if int(p["obs_mode"]) == 0 else obs_sp) + 30
    return disturbed, nominal


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------- oracle timing
def oracle_rate(p, x0, V, obs, target_s, threads, iteration=0):
    """Oracle rollout-steps/s on a bounded sample of the workload's samples."""
    import oracle

    K, M, T = int(p["K"]), int(p["M"]), int(p["T"])
    n = max(threads, 8)
    while True:
        ks = np.arange(min(n, K), dtype=np.int32)
        t0 = time.perf_counter()
        out = oracle.samples(p, x0, V, obs, ks=ks, iteration=iteration, n_threads=threads)
        oracle.update(out["S_tilde"], out["U"], float(np.float32(p["lam"])))
        dt = time.perf_counter() - t0
        if dt >= target_s or len(ks) >= K:
            return len(ks) * M * T / dt, len(ks), dt
        n = int(min(K, max(2 * n, n * target_s / max(dt, 1e-3) * 1.1)))


def run_reference(args, p, x0, V, obs):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    # calibrate the per-step sample to about 1.5 s of CPU work
    _, n_cal, dt_cal = oracle_rate(p, x0, V, obs, 0.3, threads)
    per = n_cal / max(dt_cal, 1e-6)
    ks_n = int(max(threads, min(int(p["K"]), per * 1.5)))
    import oracle

    K, M, T = int(p["K"]), int(p["M"]), int(p["T"])
    ks = np.arange(ks_n, dtype=np.int32)
    for i in range(args.warmup):
        oracle.samples(p, x0, V, obs, ks=ks[: max(1, ks_n // 4)], iteration=i, n_threads=threads)
    times = []
    for i in range(args.steps):
        t0 = time.perf_counter()
        out = oracle.samples(p, x0, V, obs, ks=ks, iteration=args.warmup + i, n_threads=threads)
        oracle.update(out["S_tilde"], out["U"], float(np.float32(p["lam"])))
        times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    value = ks_n * M * T / t
    line = {
        "impl": "reference", "metric": "rollout-steps/s (K*M*T)", "value": value,
        "unit": "rollout-steps/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": config_dict(p, args),
        "cpu_baseline": {"value": value, "unit": "rollout-steps/s", "cores": threads, "kind": "oracle",
                         "sample": f"{ks_n} of {K} samples x M={M} x T={T} per step (FP64 C oracle, "
                                   f"OpenMP over samples), then the softmin update over them"},
        "e2e": {"value": value, "unit": "rollout-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_dict(p, args):
    return {"workload": f"{args.workload}: {p['K']} samples x {p['M']} rollouts x {p['T']} steps, "
                        f"{['kinematic bicycle', 'dynamic single-track', 'linear'][int(p['model'])]}, "
                        f"{p['n_obs']} obstacles",
            "K": int(p["K"]), "M": int(p["M"]), "T": int(p["T"]), "model": int(p["model"]),
            "substeps": int(p["substeps"]), "n_obs": int(p["n_obs"]), "alpha": float(p["alpha"]),
            "step": f"one receding-horizon iteration (update, plant step, warm start) after a "
                    f"{args.preroll}-iteration untimed pre-roll from the track origin",
            "l2": "flushed before every timed step (256 MB write, outside the step's events)"}


# ---------------------------------------------------------------- GPU arm
def run_ours(args, p, x0, V, obs):
    import torch
    import torch.distributed as dist

    from paper_2209_12842_gb300 import RaMppi
    from paper_2209_12842_gb300 import binding as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    p = dict(p, seed=int(p["seed"]) + rank, instance_id=rank)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    ctl = RaMppi(p, obs)
    x0_d = torch.from_numpy(x0).to(dev)
    V_d = torch.from_numpy(V).to(dev)
    V_out = torch.empty_like(V_d)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kv_b = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kv_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]

    # The timed step is one receding-horizon iteration of Algorithm 1 (update,
    # execute v0+ on the simulated plant, warm start), from the state the loop
    # reaches after an untimed pre-roll, so the rollouts meet the obstacles.
    x_d = x0_d.clone()
    hits = torch.zeros(2, dtype=torch.int32, device=dev)
    for i in range(args.preroll):
        ctl.closed_loop_step(x_d, V_d, hits)
    torch.cuda.synchronize()
    tune_ms = ctl.tune(x_d, V_d, 3)  # launch-shape autotuner (results do not depend on it)
    warps, ilp, wps = ctl.get_launch()
    for i in range(args.warmup):
        ctl.closed_loop_step(x_d, V_d, hits)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
        time.sleep(0.4)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler select exactly these launches
    for i in range(args.steps):
        flush.fill_(float(i))
        ctl.set_timing_events(kv_b[i], kv_e[i])
        ev_b[i].record(stream)
        ctl.closed_loop_step(x_d, V_d, hits)
        ev_e[i].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - t0
    ctl.set_timing_events(None)
    clk = clocks.stop() if rank == 0 else None
    status = ctl.status()
    # obstacles tested exactly per rollout-step (one extra, untimed update)
    cand = torch.zeros(1, dtype=torch.int64, device=dev)
    B.ra_mppi_set_diagnostics(ctl.h, cand.data_ptr())
    ctl.step(x_d, V_d, V_out)
    torch.cuda.synchronize()
    B.ra_mppi_set_diagnostics(ctl.h, None)
    tested = float(cand.item()) / (int(p["K"]) * ((int(p["M"]) + 31) // 32) * int(p["T"]))

    step_ms = np.array([b.elapsed_time(e) for b, e in zip(ev_b, ev_e)])
    kern_ms = np.array([b.elapsed_time(e) for b, e in zip(kv_b, kv_e)])
    t_step = aggregate_over_ranks(dist if world > 1 else None, torch, float(step_ms.sum()) / 1e3, dev)
    K, M, T = int(p["K"]), int(p["M"]), int(p["T"])
    units = K * M * T
    value = job_value(world, units, args.steps, t_step)

    # end to end through the C ABI with host buffers (pinned), copies inside
    nx = x0.size
    x0_h = x_d.cpu().pin_memory()
    V_h = torch.from_numpy(V).pin_memory()
    Vo_h = torch.empty_like(V_h).pin_memory()
    for i in range(2):
        B.ra_mppi_step_host(ctl.h, x0_h.data_ptr(), V_h.data_ptr(), Vo_h.data_ptr(), None, stream.cuda_stream)
    e2e_ms = []
    for i in range(args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        B.ra_mppi_step_host(ctl.h, x0_h.data_ptr(), V_h.data_ptr(), Vo_h.data_ptr(), None, stream.cuda_stream)
        e2e_ms.append(1e3 * (time.perf_counter() - t1))
    e2e_t = aggregate_over_ranks(dist if world > 1 else None, torch, float(np.mean(e2e_ms)) / 1e3, dev)
    ctl.close()

    if rank == 0:
        d_ops, n_ops = algorithmic_ops(p, tested)
        d_ops_bf, _ = algorithmic_ops(p)
        ops_per_launch = units * d_ops + K * T * n_ops
        k_mean = float(kern_ms.mean()) / 1e3
        achieved = ops_per_launch / k_mean / 1e9
        sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
        peak = N_SMS * LANES_PER_SM * sm_mhz * 1e6 / 1e9
        traffic = load_traffic(args.workload)
        line = {
            "metric": "rollout-steps/s (K*M*T)", "value": value, "unit": "rollout-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_step / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(p, args),
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                           "rollout_kernel_mean": 1e3 * k_mean},
            "wall_ms_per_step_incl_flush": 1e3 * wall / args.steps,
            "gpu_launches": 3 * args.steps,
            "launch": {"warps_per_block": warps, "rollouts_interleaved": ilp, "warps_per_sample": wps,
                       "tune_ms": tune_ms},
            "status": B.STATUS_NAMES.get(status, status),
            "clocks": clk,
            "e2e": {"value": world * units / e2e_t, "unit": "rollout-steps/s",
                    "h2d_bytes_per_step": 4 * (nx + V.size), "d2h_bytes_per_step": 4 * V.size,
                    "ms_per_step": 1e3 * e2e_t},
            "roofline": {"bound": "alu", "kernel": "rollout_cvar_kernel", "achieved": achieved, "peak": peak,
                         "unit": "Gop/s (ALU lane-ops, formula count)", "frac": achieved / peak,
                         "ops_per_launch": ops_per_launch, "ops_per_disturbed_step": d_ops,
                         "ops_per_nominal_step": n_ops,
                         "obstacles_tested_per_rollout_step": tested,
                         "ops_per_disturbed_step_brute_force": d_ops_bf,
                         "frac_brute_force_count": (units * d_ops_bf + K * T * n_ops) / k_mean / 1e9 / peak,
                         "peak_basis": f"{N_SMS} SMs x {LANES_PER_SM} lanes x median SM clock {sm_mhz:.0f} MHz",
                         "traffic": traffic},
        }
        if world == 1 and not args.no_studies:
            line["closed_loop"] = closed_loop_study(torch, args.loop_updates)
            line["closed_loop_paper_preset"] = closed_loop_study(
                torch, args.loop_updates, "paper_sim", [("mppi", dict(A=0.0)), ("ra_alpha0.7", {})])
            line["batched"] = batched_study(torch, 10)
            line["adjoint"] = adjoint_study(torch, 10)
            line["importance"] = importance_study(torch)
        if world == 1 and not args.no_cpu_baseline:
            threads = os.cpu_count() or 1
            rate, n_s, dt = oracle_rate(p, x0, V, obs, args.cpu_seconds, threads)
            line["cpu_baseline"] = {"value": rate, "unit": "rollout-steps/s", "cores": threads,
                                    "kind": "oracle",
                                    "sample": f"{n_s} of {K} samples x M={M} x T={T} "
                                              f"({dt:.1f} s, FP64 C oracle, OpenMP over samples)"}
        else:
            line["cpu_baseline"] = None
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def kernel_source_sha():
    """Hash of the sources of the rollout kernel (names and bytes), to tie ncu
    counters to a kernel version."""
    import hashlib

    csrc = os.path.join(ROOT, "paper_2209_12842_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(csrc)):
        if f.startswith(("ra_rollout", "ra_device", "ra_api")):
            h.update(f.encode())
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def aggregate_over_ranks(dist, torch, seconds, device):
    """Max over ranks of a per-rank duration (the slowest rank sets the job
    time); identity without a process group."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, units_per_rank, steps, seconds):
    """Whole-job rollout-steps/s: every rank processes its own problem."""
    return world * units_per_rank * steps / seconds


def ev_time(torch, fn, n, stream):
    """Median and p99 of n CUDA-event timings of fn (ms), after 2 warm-ups."""
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for b, e in evs:
        b.record(stream)
        fn()
        e.record(stream)
    torch.cuda.synchronize()
    t = np.array([b.elapsed_time(e) for b, e in evs])
    return float(np.median(t)), float(np.percentile(t, 99))


def closed_loop_study(torch, n_updates, preset="c2_closed_loop", runs=None, seeds=(12842, 12843, 12844)):
    """Receding-horizon loop on the simulated plant (Alg. 1 outer loop): update
    rate, plant steps inside an obstacle and steps off the track, for plain
    MPPI (A = 0) and RA-MPPI, each over the same obstacle field with several
    noise seeds (the counts of one 1000-update run vary a lot with the
    noise).  Config 2 compares alpha in {0.5, 0.9, 0.99} with its risk cost
    l = obstacle term; the paper's preset uses l = q (boundary, obstacles,
    deviation) with A = 10, C_u = 0.6, alpha = 0.7."""
    from paper_2209_12842_gb300 import RaMppi

    p0 = rs.preset(preset)
    obs = rs.scene_obstacles(p0)
    out = {"preset": preset, "updates": n_updates, "seeds": list(seeds)}
    if runs is None:
        runs = [("mppi", dict(A=0.0))] + [(f"ra_alpha{a}", dict(alpha=a)) for a in (0.5, 0.9, 0.99)]
    for name, ov in runs:
        hits_per_seed, exits_per_seed, hz, status = [], [], None, 0
        for seed in seeds:
            p = rs.preset(preset, seed=seed, **ov)
            ctl = RaMppi(p, obs)
            x = torch.from_numpy(rs.scene_initial_state(p)).cuda()
            V = torch.zeros((p["T"], 2), dtype=torch.float32, device="cuda")
            hits = torch.zeros(2, dtype=torch.int32, device="cuda")  # obstacle hits, track exits
            stream = torch.cuda.current_stream()
            b, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            b.record(stream)
            for _ in range(n_updates):
                ctl.closed_loop_step(x, V, hits)
            e.record(stream)
            torch.cuda.synchronize()
            if hz is None:
                hz = 1e3 * n_updates / b.elapsed_time(e)
            h2 = hits.cpu().numpy()
            hits_per_seed.append(int(h2[0]))
            exits_per_seed.append(int(h2[1]))
            status |= ctl.status()
            ctl.close()
        out[name] = {"obstacle_hits": hits_per_seed, "obstacle_hits_mean": float(np.mean(hits_per_seed)),
                     "track_exits": exits_per_seed, "track_exits_mean": float(np.mean(exits_per_seed)),
                     "update_hz": hz, "status": status}
    return out


def batched_study(torch, steps):
    """Config 3: B = 256 uneven kinematic problems, one graph replay per round
    against a loop of 256 plain per-problem updates on the same stream."""
    from paper_2209_12842_gb300 import RaMppi
    from paper_2209_12842_gb300.controller import RaMppiBatch

    insts = rs.batched_instances(256)
    for d in insts:
        d["max_obstacles"] = d["n_obs"]
    p = rs.preset("c3_instance")
    batch = RaMppiBatch(p, insts)
    x0s, Vs, obs = [], [], []
    for i, d in enumerate(insts):
        o = rs.make_obstacles(d["seed"], d["n_obs"], 0.3, 0.3)
        obs.append(o)
        batch.set_obstacles(i, o)
        x0s.append(rs.initial_state(0))
        Vs.append(rs.random_controls(0, d["T"], p["u_lo"], p["u_hi"], d["seed"]))
    batch.set_inputs(x0s, Vs)
    units = sum(d["K"] * d["M"] * d["T"] for d in insts)
    stream = torch.cuda.current_stream()
    tuned_ms = batch.tune(3)
    g50, g99 = ev_time(torch, lambda: batch.step(graph=True), steps, stream)
    ctls = []
    for i, d in enumerate(insts):
        q = dict(p, K=d["K"], M=d["M"], T=d["T"], seed=d["seed"], instance_id=d["instance_id"], n_obs=d["n_obs"])
        c = RaMppi(q, obs[i], max_obstacles=max(d["n_obs"], 1))
        ctls.append((c, torch.from_numpy(x0s[i]).cuda(), torch.from_numpy(Vs[i]).cuda(),
                     torch.empty((d["T"], 2), dtype=torch.float32, device="cuda")))

    def loop():
        for c, x, v, o in ctls:
            c.step(x, v, o, want_cvar=False)

    l50, l99 = ev_time(torch, loop, max(3, steps // 2), stream)
    launch = batch.get_launch()
    for c, *_ in ctls:
        c.close()
    batch.close()
    return {"problems": 256, "rollout_steps_per_round": units,
            "batched_graph": {"p50_ms": g50, "p99_ms": g99, "rollout_steps_per_s": units / g50 * 1e3},
            "loop_of_plain_launches": {"p50_ms": l50, "p99_ms": l99, "rollout_steps_per_s": units / l50 * 1e3},
            "speedup_p50": l50 / g50, "tuned_launch": {"warps_per_block": launch[0], "ilp": launch[1],
                                                       "grid": launch[2], "tune_ms": tuned_ms}}


def adjoint_study(torch, steps):
    """Config 4: forward update and hand-written adjoint latency (kinematic,
    K = 1024, M = 64, T = 30, softplus barrier)."""
    from paper_2209_12842_gb300 import RaMppi

    p = rs.preset("c4_gradient")
    obs = rs.make_obstacles(p["seed"], p["n_obs"], *p["obs_r"])
    ctl = RaMppi(p, obs, differentiable=True)
    x0 = torch.tensor([0.0, -4.0, 0.0, 1.5], device="cuda")
    V = torch.from_numpy(rs.random_controls(0, p["T"], p["u_lo"], p["u_hi"], 5)).cuda()
    gVp, gS = rs.random_cotangents(p["T"], 2, p["K"], 11)
    gVp, gS = torch.from_numpy(gVp).cuda(), torch.from_numpy(gS).cuda()
    stream = torch.cuda.current_stream()
    f50, f99 = ev_time(torch, lambda: ctl.step(x0, V), steps, stream)
    ctl.step(x0, V)
    b50, b99 = ev_time(torch, lambda: ctl.backward(gVp, gS), steps, stream)
    ctl.close()
    units = p["K"] * p["M"] * p["T"]
    return {"forward_p50_ms": f50, "forward_p99_ms": f99, "backward_p50_ms": b50, "backward_p99_ms": b99,
            "backward_rollout_steps_per_s": units / b50 * 1e3}


def importance_study(torch, scales=((1.5, 0.5), (1.1, 0.5)), alpha=0.99):
    """Importance-sampled CVaR at alpha = 0.99: the spread of the estimate
    over K independent samples with identical controls (sigma_u = 0), plain
    Monte Carlo against the scaled-proposal, deterministic-mixture weights at
    the same M.  (a) The linear-Gaussian test system (T = 10 noise draws per
    rollout), whose CVaR has a closed form; (b) the config 2 vehicle (dynamic
    model, 120 noise draws per rollout, obstacle risk cost) driving straight
    between two obstacles that its nominal path clears by 1 cm, so that only
    about one rollout in a thousand collides, with plain Monte Carlo at 4x
    the rollouts as the reference mean."""
    from statistics import NormalDist

    from paper_2209_12842_gb300 import RaMppi

    def estimates(p, obs, x0, V):
        ctl = RaMppi(p, obs)
        x0t, Vt = torch.from_numpy(x0).cuda(), torch.from_numpy(V).cuda()
        ctl.step(x0t, Vt)
        ms, _ = ev_time(torch, lambda: ctl.step(x0t, Vt), 5, torch.cuda.current_stream())
        cv = ctl.cvar.cpu().numpy().astype(np.float64)
        ctl.close()
        return cv, ms

    out = {"alpha": alpha}
    T, sw = 10, float(np.float32(0.5))
    a32 = float(np.float32(alpha))
    V = (np.arange(T) * 0.1 - 0.3).astype(np.float32).reshape(T, 1)
    x0 = np.array([0.25], np.float32)
    xs = 0.25 + np.concatenate([[0.0], np.cumsum(V[:, 0].astype(np.float64))])[:T]
    sd = sw * np.sqrt((T - 1) * T * (2 * T - 1) / 6.0)
    truth = xs.sum() + sd * NormalDist().pdf(NormalDist().inv_cdf(a32)) / (1 - a32)
    p = rs.preset("linear_test", K=4096, M=128, T=T, w_scale=(sw, 0, 0, 0), alpha=alpha)
    lin = {"closed_form": truth, "M": 128, "K": 4096, "is_scale": scales[0][0], "is_frac": scales[0][1]}
    for name, ov in (("plain", {}), ("importance", dict(is_scale=scales[0][0], is_frac=scales[0][1]))):
        cv, ms = estimates(dict(p, **ov), np.zeros((0, 3), np.float32), x0, V)
        lin[name] = {"mean": float(cv.mean()), "sd": float(cv.std()),
                     "rmse": float(np.sqrt(np.mean((cv - truth) ** 2))), "update_ms": ms}
    lin["variance_ratio"] = (lin["plain"]["sd"] / lin["importance"]["sd"]) ** 2
    out["linear_gaussian"] = lin
    p = rs.preset("c2_closed_loop", sigma_u=(0.0, 0.0), alpha=alpha)
    x0 = rs.initial_state(1)
    obs = np.array([[0.8, x0[1] + 0.21, 0.2], [1.2, x0[1] - 0.21, 0.2]], np.float32)
    V = np.tile(np.array([[0.0, 1.0]], np.float32), (p["T"], 1))  # straight, accelerating
    ref, _ = estimates(dict(p, M=512), obs, x0, V)
    dyn = {"reference_mean_M512": float(ref.mean()), "M": p["M"], "K": p["K"], "is_scale": scales[1][0],
           "is_frac": scales[1][1]}
    for name, ov in (("plain", {}), ("importance", dict(is_scale=scales[1][0], is_frac=scales[1][1]))):
        cv, ms = estimates(dict(p, **ov), obs, x0, V)
        dyn[name] = {"mean": float(cv.mean()), "sd": float(cv.std()), "update_ms": ms}
    dyn["variance_ratio"] = (dyn["plain"]["sd"] / dyn["importance"]["sd"]) ** 2 if dyn["importance"]["sd"] > 0 else None
    out["config2"] = dyn
    return out


def stress_sweep(args):
    """Config 5: dynamic single-track, K = 65536, T = 50, 200 obstacles; M in
    {32, 64, 128, 256} x alpha in {0.8, 0.95}; update latency p50/p99 over
    `--steps` updates per point and the rollout kernel's roofline fraction."""
    import torch

    from paper_2209_12842_gb300 import RaMppi
    from paper_2209_12842_gb300 import binding as B

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    base = rs.preset("c5_stress")
    obs = rs.make_obstacles(base["seed"], base["n_obs"], *base["obs_r"])
    x0 = torch.from_numpy(rs.initial_state(base["model"])).cuda()
    V = torch.from_numpy(rs.random_controls(base["model"], base["T"], base["u_lo"], base["u_hi"], 3)).cuda()
    clocks = ClockSampler(0)
    clocks.start()
    points = []
    for M in (32, 64, 128, 256):
        for alpha in (0.8, 0.95):
            p = rs.preset("c5_stress", M=M, alpha=alpha)
            ctl = RaMppi(p, obs)
            Vo = torch.empty_like(V)
            ctl.tune(x0, V, 2)
            warps, ilp, wps = ctl.get_launch()
            kb = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            ke = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            sb = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            se = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            for _ in range(args.warmup):
                ctl.step(x0, V, Vo)
            torch.cuda.synchronize()
            for i in range(args.steps):
                ctl.set_timing_events(kb[i], ke[i])
                sb[i].record(stream)
                ctl.step(x0, V, Vo)
                se[i].record(stream)
            torch.cuda.synchronize()
            ctl.set_timing_events(None)
            cand = torch.zeros(1, dtype=torch.int64, device="cuda")
            B.ra_mppi_set_diagnostics(ctl.h, cand.data_ptr())
            ctl.step(x0, V, Vo)
            torch.cuda.synchronize()
            B.ra_mppi_set_diagnostics(ctl.h, None)
            tested = float(cand.item()) / (p["K"] * ((M + 31) // 32) * p["T"])
            step_ms = np.array([a.elapsed_time(b) for a, b in zip(sb, se)])
            k_ms = float(np.mean([a.elapsed_time(b) for a, b in zip(kb, ke)]))
            d_ops, n_ops = algorithmic_ops(p, tested)
            ops = p["K"] * M * p["T"] * d_ops + p["K"] * p["T"] * n_ops
            points.append({"M": M, "alpha": alpha, "p50_ms": float(np.percentile(step_ms, 50)),
                           "p99_ms": float(np.percentile(step_ms, 99)), "rollout_kernel_ms": k_ms,
                           "rollout_steps_per_s": p["K"] * M * p["T"] / (float(np.median(step_ms)) / 1e3),
                           "obstacles_tested_per_rollout_step": tested, "ops_per_launch": ops,
                           "achieved_gops": ops / (k_ms / 1e3) / 1e9, "launch": [warps, ilp, wps]})
            ctl.close()
    clk = clocks.stop()
    peak = N_SMS * LANES_PER_SM * (clk.get("sm_mhz") or 2070.0) * 1e6 / 1e9
    for pt in points:
        pt["roofline_frac"] = pt["achieved_gops"] / peak
    top = [pt for pt in points if pt["M"] == 256 and pt["alpha"] == 0.95][0]
    line = {"metric": "rollout-steps/s (K*M*T)", "value": top["rollout_steps_per_s"], "unit": "rollout-steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": top["p50_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c5 stress: dynamic single-track, K=65536, T=50, 200 obstacles, sweep of M and alpha",
                       "l2": "inputs resident; per-update working set below L2 (compute bound)"},
            "clocks": clk, "roofline_peak_gops": peak, "sweep": points}
    print(json.dumps(line), flush=True)


def load_traffic(workload):
    """DRAM bytes per rollout-kernel launch from the committed ncu summary, or
    None when none exists or it was taken on a different kernel version."""
    path = os.path.join(ROOT, "profiles", f"rollout_cvar_{workload}.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("source_sha") != kernel_source_sha():
        return None
    return rec.get("dram_bytes_per_launch")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-studies", action="store_true",
                    help="skip the closed-loop, batched and adjoint sections of the line")
    ap.add_argument("--loop-updates", type=int, default=1000)
    ap.add_argument("--preroll", type=int, default=200,
                    help="untimed receding-horizon iterations before timing (the state leaves the start area)")
    ap.add_argument("--sweep", action="store_true", help="config 5 stress sweep over M and alpha")
    ap.add_argument("--K", type=int, default=0,
                    help="run the workload with this many samples instead (a smaller case for ncu captures; "
                         "not a bench line of the named workload)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.sweep:
        stress_sweep(args)
        return
    p = rs.preset(WORKLOADS[args.workload], **({"K": args.K} if args.K > 0 else {}))
    obs = rs.scene_obstacles(p)
    x0 = rs.scene_initial_state(p)
    V = rs.random_controls(p["model"], p["T"], p["u_lo"], p["u_hi"], 3)
    if args.impl == "reference":
        run_reference(args, p, x0, V, obs)
    else:
        run_ours(args, p, x0, V, obs)


if __name__ == "__main__":
    main()
