"""Benchmark of the RA-MPPI control update on GB300.

Metric: rollout-steps/s, one rollout-step being one disturbed step of one
of the K x M rollouts (K M T per update); the K T nominal steps are extra
work that is not counted.  A "step" of this benchmark is one complete
update (sampling, nominal and disturbed rollouts, CVaR, softmin update;
ra_mppi_step) on the stress workload by default: dynamic single-track
vehicle, K = 65536 samples, M = 256 disturbed rollouts, T = 50 steps, 200
obstacles (`--workload` picks another; the line's sections carry the
others).

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
# Formula counts of the rollout kernel's work, by pipe, per disturbed
# rollout-step and per nominal step (lane-operations).  Each count follows
# the source of the device functions it names:
#   fp32  FP32 add, multiply, FMA, min/max, compare-select, rounding;
#   xu    special-function unit: every rsqrt, rcp, sin, cos, log, exp, sqrt,
#         tan the kernel calls (a math-library call counts as one operation,
#         whatever it expands to);
#   int   32-bit integer and logic operations, int <-> float conversions
#         (64 per SM per clock on GB300, not the special-function rate), warp
#         votes and reductions;
#   issue warp instructions x 32 of the three, where the dynamic model's
#         FP32 arithmetic counts half when the launch steps rollouts in
#         paired FP32 instructions (loads, moves and branches are not
#         counted, so this is a lower bound of what the kernel issues).
PHILOX_INT = 60  # 10 rounds x (2 wide multiplies, 2 three-input xors, 2 key adds)


DYN_DERIV_FP32 = 1 + 4 + 1 + 18 + 2 + 10 + 1 + 11
# one obstacle of the softplus barrier (softplus_fast): offsets 2, squared
# distance 2, distance 2, argument 2, the exponential's scaling 1, the series
# 5, the logarithm's sum and scaling 2, select, max, sum and accumulation 4
SOFTPLUS_FP32 = 20
DYN_SUBSTEP_FP32 = 2 * DYN_DERIV_FP32 + 18


def _dyn_substep():
    """One Heun sub-step of the dynamic single-track model (Model<1>):
    two derivative evaluations and the trapezoid update.  Per derivative:
    the floored 1/vx (1 fp32 + rcp), slip arguments (4), the warp's range
    vote (1), two arctangent polynomials (2 x 9), Pacejka arguments (2), two
    closed-form C = 3/2 shapes (2 x (5 fp32 + 2 rsqrt)), the heading sincos
    of a heading near [-pi, pi] (its argument scaling, 1 fp32, + sin + cos)
    and the six derivatives (11)."""
    return dict(fp32=DYN_SUBSTEP_FP32, xu=2 * (1 + 4 + 2), int=0)


def _dyn_step_extra(ilp):
    """Once per control step of the dynamic model: the heading wrapped to
    [-pi, pi] (4 fp32) and the front axle's two control terms (2 fp32, shared
    by the ILP rollouts of a lane)."""
    return 4 + 2 / ilp


def _kin_substep():
    """One Euler sub-step of the kinematic bicycle: heading sincos (5 fp32 +
    sin + cos), h v (1) and four FMAs."""
    return dict(fp32=10, xu=2, int=0)


def _noise(p):
    """Process noise of one rollout-step (add_process_noise)."""
    model, nt = int(p["model"]), int(p["noise_type"])
    slots = {0: 4, 1: 3, 2: 1}[model]
    if nt == 1:  # mixture: two Philox calls; per slot mix_value (log, rsqrt, cos, 2 conversions)
        return dict(fp32=14 * slots, xu=3 * slots, int=2 * PHILOX_INT + 6 * slots)
    if nt == 0:  # Gaussian: one Philox call, ceil(slots / 2) Box-Muller pairs (log, rsqrt, sin, cos)
        bm = (slots + 1) // 2
        return dict(fp32=9 * bm + slots, xu=4 * bm, int=PHILOX_INT + 2 * bm)
    if nt == 2:  # uniform: one conversion per slot
        return dict(fp32=2 * slots, xu=0, int=PHILOX_INT + slots)
    return dict(fp32=slots + 2, xu=0, int=PHILOX_INT + 2)  # impulse (mostly no jump)


def pipe_counts(p, tested=None, ilp=1, paired=False):
    """(disturbed, nominal): per-pipe lane-operation counts per disturbed
    rollout-step and per nominal step, and the issue count.

    tested: obstacles tested exactly per rollout-step after the kernel's
    bounding-box cull (measured by the diagnostic counter); None counts all
    of them (brute force).  ilp: rollouts a lane interleaves (the cull's box
    and its obstacle rounds are shared by them).  paired: the dynamic model's
    FP32 arithmetic runs in paired instructions."""
    model, n_obs, sub = int(p["model"]), int(p["n_obs"]), int(p["substeps"])
    ind = int(p["obs_mode"]) == 0
    if model == 1:
        step = {k: v * sub for k, v in _dyn_substep().items()}
        step["fp32"] += _dyn_step_extra(ilp)
    elif model == 0:
        step = {k: v * sub for k, v in _kin_substep().items()}
    else:
        step = dict(fp32=sub, xu=0, int=0)
    dyn_fp32 = step["fp32"]
    nz = _noise(p)
    d = {k: step[k] + nz[k] for k in ("fp32", "xu", "int")}
    risk_obs = int(p["risk_mask"]) & 4
    if risk_obs and ind and model != 2:
        n_test = n_obs if tested is None else tested
        windowed = model == 1 and n_obs > 64
        rounds = 1 if windowed else max(1, -(-n_obs // 32))
        # box of the warp's states: min/max, shift, warp reductions, unshift;
        # per 32-obstacle round: the box test (8 fp32) and its ballot and loop
        # (4 int); per candidate: the exact test (6 fp32) per state and the
        # candidate loop (3 int, shared); the x window's two searches (10 int)
        d["fp32"] += (2 * (ilp - 1) + 8 + 8 * rounds) / ilp + 6 * n_test + 1
        d["int"] += (4 + 4 * rounds + (10 if windowed else 0)) / ilp + 3 * n_test / ilp
    elif risk_obs and model != 2:  # softplus barrier: per obstacle 20 fp32, rsqrt + ex2 + lg2
        d["fp32"] += SOFTPLUS_FP32 * n_obs + 1
        d["xu"] += 3 * n_obs
    if int(p["risk_mask"]) & ~4:
        d["fp32"] += 8
        d["xu"] += 1
    fp32_instr = d["fp32"] - (dyn_fp32 / 2 if paired and model == 1 else 0)
    d["issue"] = fp32_instr + d["xu"] + d["int"]
    # nominal step: control draw (Philox, accurate Box-Muller, clip: 11 fp32,
    # log + sqrt + sin + cos, 2 conversions), the per-step control
    # quantities, the dynamics, the full running cost (track 6 fp32 + sqrt,
    # deviation, speed, every obstacle) and the control cost
    n = dict(fp32=11 + step["fp32"] + 6 + 2 + 3 + (6 * n_obs if ind else SOFTPLUS_FP32 * n_obs) + 3 + 2,
             xu=4 + 2 + step["xu"] + 1 + (0 if ind else 3 * n_obs),
             int=PHILOX_INT + step["int"] + 6)
    n["issue"] = n["fp32"] + n["xu"] + n["int"]
    return d, n


def pipe_roofline(p, units, kernel_s, tested, ilp, paired, rates, n_sms, sm_mhz):
    """Per-pipe roofline of one rollout-kernel launch: achieved lane-ops/s of
    each pipe from the formula counts over the measured kernel time, against
    n_sms x (measured lane-ops per SM per clock) x the sampled SM clock."""
    d, n = pipe_counts(p, tested, ilp, paired)
    K, T = int(p["K"]), int(p["T"])
    clk = sm_mhz * 1e6
    out = {}
    for pipe in ("fp32", "xu", "issue"):
        ops = units * d[pipe] + K * T * n[pipe]
        peak = n_sms * rates[pipe] * clk
        out[pipe] = {"ops_per_launch": ops, "achieved": ops / kernel_s / 1e9, "peak": peak / 1e9,
                     "frac": ops / kernel_s / peak, "per_disturbed_step": d[pipe], "per_nominal_step": n[pipe]}
    out["int_ops_per_disturbed_step"] = d["int"]
    bound = max(("fp32", "xu", "issue"), key=lambda k: out[k]["frac"])
    return bound, out


def adjoint_counts(p):
    """Per-pipe formula counts of the adjoint's main kernel (bwd_main_kernel):
    per reversed disturbed rollout-step and per reversed nominal step.  A
    reversed step replays 7 of 8 forward steps from the checkpoints (dynamics
    and, disturbed, the process noise), then takes the step's transposed
    Jacobian and the gradient of the cost terms; the softplus barrier's
    gradient takes per obstacle 12 fp32 and a reciprocal square root, an
    exponential, a logarithm and a reciprocal."""
    model, n_obs, sub = int(p["model"]), int(p["n_obs"]), int(p["substeps"])
    if model == 1:
        fwd = {k: v * sub for k, v in _dyn_substep().items()}
        # the sub-steps recomputed from the step's start (sub (sub - 1) / 2),
        # then per sub-step one derivative and two transposed derivatives
        # (each about 80 fp32, 10 special-function operations)
        vjp = dict(fp32=(sub * (sub - 1) // 2) * DYN_SUBSTEP_FP32 + sub * (DYN_DERIV_FP32 + 2 * 80 + 18),
                   xu=(sub * (sub - 1) // 2) * 14 + sub * (7 + 2 * 10), int=0)
    elif model == 0:
        fwd = {k: v * sub for k, v in _kin_substep().items()}
        vjp = dict(fp32=sub * 17, xu=sub * 2, int=0)
    else:
        fwd, vjp = dict(fp32=sub, xu=0, int=0), dict(fp32=sub, xu=0, int=0)
    soft = int(p["obs_mode"]) == 1
    obs_g = dict(fp32=(12 if soft else 6) * n_obs, xu=(4 if soft else 0) * n_obs, int=0)
    nz = _noise(p)
    rep = 7.0 / 8.0
    d = {k: rep * (fwd[k] + nz[k]) + vjp[k] + (obs_g[k] if int(p["risk_mask"]) & 4 else 0)
         for k in ("fp32", "xu", "int")}
    d["int"] += 10  # the control cotangents' warp sums
    n = {k: rep * fwd[k] + vjp[k] + obs_g[k] for k in ("fp32", "xu", "int")}
    n["fp32"] += 8 + 5 + 4 + 12  # track gradient, deviation, speed, control cost and clip
    n["xu"] += 2 + (2 if model == 0 else 0)  # track sqrt and division; tan(steer) and its /L
    for c in (d, n):
        c["issue"] = c["fp32"] + c["xu"] + c["int"]
    return d, n


def tail_rollouts(p):
    """Rollouts with a nonzero cotangent of a fractional-tail CVaR: ranks
    ceil(alpha M) .. M (without ties at VaR)."""
    M = int(p["M"])
    j = int(np.ceil(float(np.float32(p["alpha"])) * M))
    return M - max(1, min(M, j)) + 1


def adjoint_roofline(p, kernel_s, rates, n_sms, sm_mhz):
    d, n = adjoint_counts(p)
    K, T = int(p["K"]), int(p["T"])
    n_tail = tail_rollouts(p)
    clk = sm_mhz * 1e6
    out = {}
    for pipe in ("fp32", "xu", "issue"):
        ops = K * n_tail * T * d[pipe] + K * T * n[pipe]
        peak = n_sms * rates[pipe] * clk
        out[pipe] = {"ops_per_launch": ops, "achieved": ops / kernel_s / 1e9, "peak": peak / 1e9,
                     "frac": ops / kernel_s / peak}
    bound = max(("fp32", "xu", "issue"), key=lambda k: out[k]["frac"])
    return {"kernel": "bwd_main_kernel", "bound": "alu", "pipe": bound, "frac": out[bound]["frac"],
            "kernel_ms_mean": 1e3 * kernel_s, "tail_rollouts_per_sample": n_tail, "pipes": out,
            "note": "latency bound: one warp per sample on sequential reverse sweeps"}


def algorithmic_ops(p, tested_obstacles=None):
    """All counted lane-operations (fp32 + xu + int) per disturbed and per
    nominal step, one number each (the blended count)."""
    d, n = pipe_counts(p, tested_obstacles)
    return d["fp32"] + d["xu"] + d["int"], n["fp32"] + n["xu"] + n["int"]


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
        "config": config_dict(p, args, reference=True),
        "cpu_baseline": {"value": value, "unit": "rollout-steps/s", "cores": threads, "kind": "oracle",
                         "sample": f"{ks_n} of {K} samples x M={M} x T={T} per step (FP64 C oracle, "
                                   f"OpenMP over samples), then the softmin update over them"},
        "e2e": {"value": value, "unit": "rollout-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_dict(p, args, reference=False):
    return {"workload": f"{args.workload}: {p['K']} samples x {p['M']} rollouts x {p['T']} steps, "
                        f"{['kinematic bicycle', 'dynamic single-track', 'linear'][int(p['model'])]}, "
                        f"{p['n_obs']} obstacles",
            "K": int(p["K"]), "M": int(p["M"]), "T": int(p["T"]), "model": int(p["model"]),
            "substeps": int(p["substeps"]), "n_obs": int(p["n_obs"]), "alpha": float(p["alpha"]),
            "step": ("one RA-MPPI update (the FP64 oracle's per-sample stage over a bounded sample of the "
                     "K samples, then its softmin update) from the track origin" if reference else
                     f"one RA-MPPI update (ra_mppi_step: sampling, nominal and disturbed rollouts, CVaR, "
                     f"softmin update) of the state that an untimed {args.preroll}-iteration receding-horizon "
                     f"pre-roll from the track origin reaches"),
            "l2": ("not applicable: the oracle runs on the host cores" if reference else
                   "flushed before every timed step (256 MB write, outside the step's events)")}


# ---------------------------------------------------------------- GPU arm
# Default per-SM-per-clock lane-operation rates, used when the probes cannot
# run: 128 FP32 lanes, 4 schedulers x 32 lanes of issue, and the special-
# function rate the probe measured on GB300 (see measure_pipe_rates).
DEFAULT_RATES = {"fp32": 128.0, "issue": 128.0, "xu": 16.0}
PROBE_KINDS = {"ffma": (0, 400000), "ffma2": (1, 200000), "rsqrt": (2, 60000), "cos": (3, 60000),
               "ex2": (4, 60000), "lg2": (5, 60000), "sin": (6, 60000), "i2f": (7, 60000),
               "imad": (8, 200000)}


def measure_pipe_rates(torch, reps=3):
    """Lane-operations per SM per clock of each pipe from the library's
    probe kernels (CUDA events, best of `reps`), converted with the median SM
    clock sampled while they ran.  The special-function rate of the roofline
    is the median over the six unit operations."""
    from paper_2209_12842_gb300 import binding as B

    n_sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    raw = {}
    for name, (kind, iters) in PROBE_KINDS.items():
        best = None
        for _ in range(reps):
            ms, ops = B.ra_mppi_pipe_probe(kind, iters)
            rate = ops / (ms / 1e3)
            best = rate if best is None or rate > best else best
        raw[name] = best
    clk = clocks.stop()
    mhz = clk.get("sm_mhz") or 2070.0
    per = {k: v / (n_sms * mhz * 1e6) for k, v in raw.items()}
    xu = float(np.median([per[k] for k in ("rsqrt", "cos", "ex2", "lg2", "sin")]))
    rates = {"fp32": per["ffma"], "issue": DEFAULT_RATES["issue"], "xu": xu}
    return {"per_sm_per_clock": per, "rates_used": rates, "n_sms": n_sms, "clocks": clk,
            "basis": "probe kernels, 8 independent chains per thread, 4 x 256 threads per SM; "
                     "issue rate = 4 schedulers x 32 lanes"}


def measure_update(torch, p, obs, x0, V, steps, warmup, preroll, rates, clocks=None, flush=None, tune=True):
    """Device-timed updates of one problem (ra_mppi_step on HBM-resident
    inputs, fresh noise every update) from the state an untimed receding-
    horizon pre-roll reaches: per-update CUDA events on the launching stream
    with an L2 flush before each, the rollout kernel timed by the library's
    event hook, and the per-pipe roofline of that kernel."""
    from paper_2209_12842_gb300 import RaMppi
    from paper_2209_12842_gb300 import binding as B

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    ctl = RaMppi(p, obs)
    x_d = torch.from_numpy(x0).to(dev)
    V_d = torch.from_numpy(V).to(dev)
    hits = torch.zeros(2, dtype=torch.int32, device=dev)
    for _ in range(preroll):
        ctl.closed_loop_step(x_d, V_d, hits)
    torch.cuda.synchronize()
    tune_ms = ctl.tune(x_d, V_d, 3) if tune else None
    warps, ilp, wps = ctl.get_launch()
    plan = ctl.launch_plan()
    V_out = torch.empty_like(V_d)
    for _ in range(warmup):
        ctl.step(x_d, V_d, V_out, want_cvar=False)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(steps)] for _ in range(4)]
    if clocks is not None:
        clocks.start()
        time.sleep(0.4)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler select exactly these launches
    for i in range(steps):
        if flush is not None:
            flush.fill_(float(i))
        ctl.set_timing_events(ev[2][i], ev[3][i])
        ev[0][i].record(stream)
        ctl.step(x_d, V_d, V_out, want_cvar=False)
        ev[1][i].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks is not None else None
    ctl.set_timing_events(None)
    status = ctl.status()
    # obstacles tested exactly per rollout-step (one extra, untimed update)
    cand = torch.zeros(1, dtype=torch.int64, device=dev)
    B.ra_mppi_set_diagnostics(ctl.h, cand.data_ptr())
    ctl.step(x_d, V_d, V_out)
    torch.cuda.synchronize()
    B.ra_mppi_set_diagnostics(ctl.h, None)
    K, M, T = int(p["K"]), int(p["M"]), int(p["T"])
    tested = float(cand.item()) / (K * ((M + 31) // 32) * T)
    step_ms = np.array([b.elapsed_time(e) for b, e in zip(ev[0], ev[1])])
    kern_ms = np.array([b.elapsed_time(e) for b, e in zip(ev[2], ev[3])])
    units = K * M * T
    sm_mhz = ((clk or {}).get("sm_mhz")) or 2070.0
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    paired = int(p["model"]) == 1 and ilp % 2 == 0
    k_s = float(kern_ms.mean()) / 1e3
    bound, pipes = pipe_roofline(p, units, k_s, tested, ilp, paired, rates, n_sms, sm_mhz)
    _, pipes_bf = pipe_roofline(p, units, k_s, None, ilp, paired, rates, n_sms, sm_mhz)
    out = {"ctl": ctl, "x": x_d, "V": V_d, "step_ms": step_ms, "kern_ms": kern_ms, "clocks": clk,
           "status": status, "tested": tested, "units": units, "launch": (warps, ilp, wps), "tune_ms": tune_ms,
           "plan": {"grid": plan[0], "tail_first_block": plan[1], "tail_warps_per_sample": plan[2],
                    "blocks_per_sm": plan[3]},
           "roofline": {
               "bound": "alu", "kernel": "rollout_cvar_kernel", "pipe": bound,
               "achieved": pipes[bound]["achieved"], "peak": pipes[bound]["peak"],
               "unit": f"G lane-ops/s ({bound} pipe, formula count)", "frac": pipes[bound]["frac"],
               "pipes": pipes, "obstacles_tested_per_rollout_step": tested,
               "frac_brute_force_count": {k: pipes_bf[k]["frac"] for k in ("fp32", "xu", "issue")},
               "peak_basis": f"{n_sms} SMs x measured lane-ops per SM per clock "
                             f"(fp32 {rates['fp32']:.1f}, xu {rates['xu']:.1f}, issue {rates['issue']:.0f}) "
                             f"x median SM clock {sm_mhz:.0f} MHz during the timed region",
               "kernel_ms_mean": 1e3 * k_s}}
    return out


def run_ours(args, p, x0, V, obs):
    import torch
    import torch.distributed as dist

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
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peaks = None
    rates = dict(DEFAULT_RATES)
    if rank == 0 and world == 1 and not args.no_probes:
        peaks = measure_pipe_rates(torch)
        rates = peaks["rates_used"]

    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local) if rank == 0 else None
    t0 = time.perf_counter()
    m = measure_update(torch, p, obs, x0, V, args.steps, args.warmup, args.preroll, rates, clocks, flush)
    wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    ctl, x_d = m["ctl"], m["x"]
    K, M, T = int(p["K"]), int(p["M"]), int(p["T"])
    t_step = aggregate_over_ranks(dist if world > 1 else None, torch, float(m["step_ms"].sum()) / 1e3, dev)
    value = job_value(world, m["units"], args.steps, t_step)

    # end to end through the C ABI with host buffers (pinned): the same update
    # of the same state, its inputs copied in and V+ copied out inside the call
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
        step_ms = m["step_ms"]
        warps, ilp, wps = m["launch"]
        roof = m["roofline"]
        roof["traffic"] = load_traffic(args.workload)
        line = {
            "metric": "rollout-steps/s (K*M*T)", "value": value, "unit": "rollout-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_step / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(p, args),
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                           "rollout_kernel_mean": float(m["kern_ms"].mean())},
            "wall_s_timed_section": wall,
            "gpu_launches": LAUNCHES_PER_UPDATE * args.steps,
            "launch": {"warps_per_block": warps, "rollouts_interleaved": ilp, "warps_per_sample": wps,
                       "tune_ms": m["tune_ms"], **m["plan"]},
            "status": B.STATUS_NAMES.get(m["status"], m["status"]),
            "clocks": m["clocks"],
            "e2e": {"value": world * m["units"] / e2e_t, "unit": "rollout-steps/s",
                    "h2d_bytes_per_step": 4 * (nx + V.size), "d2h_bytes_per_step": 4 * V.size,
                    "ms_per_step": 1e3 * e2e_t,
                    "call": "ra_mppi_step_host: the same update, copies in and out and a stream sync inside"},
            "roofline": roof,
            "pipe_peaks": peaks,
        }
        if world == 1 and not args.no_studies:
            line["sections"] = sections(torch, args, rates, flush)
        if world == 1 and not args.no_cpu_baseline:
            threads = os.cpu_count() or 1
            line["cpu_baseline"] = cpu_baseline(p, x_d.cpu().numpy(), V, obs, threads, args.cpu_seconds)
        else:
            line["cpu_baseline"] = None
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


LAUNCHES_PER_UPDATE = 2  # rollout_cvar_kernel and softmin_update_kernel


def cpu_baseline(p, x0, V, obs, threads, seconds):
    """The FP64 oracle on the host cores (OpenMP over samples) on K/64 of the
    workload's samples (at least the thread count), repeated for about
    `seconds`; reported as rollout-steps/s and the full update's
    extrapolated time."""
    import oracle

    K, M, T = int(p["K"]), int(p["M"]), int(p["T"])
    n = max(threads, K // 64)
    ks = np.arange(min(n, K), dtype=np.int32)
    reps, spent = 0, 0.0
    while spent < seconds or reps == 0:
        t0 = time.perf_counter()
        out = oracle.samples(p, x0, V, obs, ks=ks, iteration=reps, n_threads=threads)
        oracle.update(out["S_tilde"], out["U"], float(np.float32(p["lam"])))
        spent += time.perf_counter() - t0
        reps += 1
    rate = reps * len(ks) * M * T / spent
    # the same oracle on one core, over K/1024 of the samples for about a
    # fifth of the time
    ks1 = ks[: max(1, K // 1024)]
    reps1, spent1 = 0, 0.0
    while spent1 < seconds / 5 or reps1 == 0:
        t0 = time.perf_counter()
        out = oracle.samples(p, x0, V, obs, ks=ks1, iteration=reps1, n_threads=1)
        oracle.update(out["S_tilde"], out["U"], float(np.float32(p["lam"])))
        spent1 += time.perf_counter() - t0
        reps1 += 1
    rate1 = reps1 * len(ks1) * M * T / spent1
    return {"value": rate, "unit": "rollout-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(ks)} of {K} samples (K/64) x M={M} x T={T}, {reps} updates in {spent:.1f} s "
                      f"(FP64 C oracle, OpenMP over samples); the full update extrapolates to "
                      f"{K * M * T / rate:.1f} s",
            "single_thread": {"value": rate1, "unit": "rollout-steps/s", "cores": 1,
                              "sample": f"{len(ks1)} of {K} samples (K/1024) x M={M} x T={T}, {reps1} updates "
                                        f"in {spent1:.1f} s on one core"}}


def roofline_summary(m):
    r = m["roofline"]
    return {"pipe": r["pipe"], "frac": r["frac"], "fracs": {k: r["pipes"][k]["frac"] for k in ("fp32", "xu", "issue")},
            "kernel_ms_mean": r["kernel_ms_mean"], "obstacles_tested_per_rollout_step": r[
                "obstacles_tested_per_rollout_step"]}


SECTIONS = ("c2_update", "paper_preset_update", "c1_update", "c2_closed_loop", "batched", "adjoint", "importance")


def sections(torch, args, rates, flush):
    """The other workloads of the same line: config 2 (update rate and
    roofline, and its 1000-update closed loop), the paper's simulation preset
    (update rate only), config 1, config 3 (batched), config 4 (adjoint), and
    the importance-sampling study (`--sections` picks a subset)."""
    out = {}
    want = set(args.sections.split(",")) if args.sections else set(SECTIONS)
    for name, preset in (("c2_update", "c2_closed_loop"), ("paper_preset_update", "paper_sim"),
                         ("c1_update", "c1_plain")):
        if name not in want:
            continue
        q = rs.preset(preset)
        m = measure_update(torch, q, rs.scene_obstacles(q), rs.scene_initial_state(q),
                           rs.random_controls(q["model"], q["T"], q["u_lo"], q["u_hi"], 3), 20, 5,
                           args.preroll, rates, None, flush)
        m["ctl"].close()
        out[name] = {"K": q["K"], "M": q["M"], "T": q["T"], "p50_ms": float(np.percentile(m["step_ms"], 50)),
                     "p99_ms": float(np.percentile(m["step_ms"], 99)),
                     "rollout_steps_per_s": m["units"] / (float(np.median(m["step_ms"])) / 1e3),
                     "update_hz": 1e3 / float(np.median(m["step_ms"])), "launch": m["launch"], "plan": m["plan"],
                     "roofline": roofline_summary(m)}
    if "c2_closed_loop" in want:
        out["c2_closed_loop"] = closed_loop_study(torch, args.loop_updates)
    if "batched" in want:
        out["batched"] = batched_study(torch, 10, rates)
    if "adjoint" in want:
        out["adjoint"] = adjoint_study(torch, 10, rates)
    if "importance" in want:
        out["importance"] = importance_study(torch)
    return out


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
    l = obstacle term, and alpha in {0.5, 0.9} with l = obstacle term +
    squared deviation from the centreline at A = 3 (a risk cost that sees
    the track edges, which the obstacle term does not)."""
    from paper_2209_12842_gb300 import RaMppi

    p0 = rs.preset(preset)
    obs = rs.scene_obstacles(p0)
    out = {"preset": preset, "updates": n_updates, "seeds": list(seeds)}
    if runs is None:
        runs = [("mppi", dict(A=0.0))] + [(f"ra_alpha{a}", dict(alpha=a)) for a in (0.5, 0.9, 0.99)] + \
            [(f"ra_alpha{a}_obs_dev_A3", dict(alpha=a, A=3.0, risk_mask=rs.RISK_OBS | rs.RISK_DEV)) for a in (0.5, 0.9)]
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


def batched_study(torch, steps, rates=None):
    """Config 3: B = 256 uneven kinematic problems, one graph replay per round
    against a loop of 256 plain per-problem updates on the same stream; and
    the persistent rollout kernel's per-pipe roofline (its eager launch timed
    by the library's event hook, the obstacles tested counted once)."""
    from paper_2209_12842_gb300 import RaMppi
    from paper_2209_12842_gb300.controller import RaMppiBatch

    rates = rates or dict(DEFAULT_RATES)
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
    # the rollout kernel alone (eager launches with the event hook)
    kb, ke = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    batch.set_timing_events(kb, ke)
    kms = []
    torch.cuda.nvtx.range_push("batched_eager")  # lets a profiler select these launches
    for _ in range(max(3, steps // 2)):
        batch.step(graph=False)
        torch.cuda.synchronize()
        kms.append(kb.elapsed_time(ke))
    torch.cuda.nvtx.range_pop()
    batch.set_timing_events(None)
    cand = torch.zeros(1, dtype=torch.int64, device="cuda")
    batch.set_diagnostics(cand)
    batch.step(graph=False)
    torch.cuda.synchronize()
    batch.set_diagnostics(None)
    rows = sum(d["K"] * ((d["M"] + 31) // 32) * d["T"] for d in insts)
    tested = float(cand.item()) / rows
    launch = batch.get_launch()
    k_s = float(np.median(kms)) / 1e3
    n_sms = torch.cuda.get_device_properties(0).multi_processor_count
    sm_mhz = 2070.0
    ops = {"fp32": 0.0, "xu": 0.0, "issue": 0.0}
    for d in insts:
        q = dict(p, K=d["K"], M=d["M"], T=d["T"], n_obs=d["n_obs"])
        dd, nn = pipe_counts(q, tested, launch[1], False)
        for pipe in ops:
            ops[pipe] += d["K"] * d["M"] * d["T"] * dd[pipe] + d["K"] * d["T"] * nn[pipe]
    pipes = {k: {"ops_per_launch": v, "achieved": v / k_s / 1e9, "peak": n_sms * rates[k] * sm_mhz * 1e6 / 1e9,
                 "frac": v / k_s / (n_sms * rates[k] * sm_mhz * 1e6)} for k, v in ops.items()}
    bound = max(pipes, key=lambda k: pipes[k]["frac"])
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
    for c, *_ in ctls:
        c.close()
    batch.close()
    return {"problems": 256, "rollout_steps_per_round": units,
            "batched_graph": {"p50_ms": g50, "p99_ms": g99, "rollout_steps_per_s": units / g50 * 1e3},
            "loop_of_plain_launches": {"p50_ms": l50, "p99_ms": l99, "rollout_steps_per_s": units / l50 * 1e3},
            "speedup_p50": l50 / g50, "tuned_launch": {"warps_per_block": launch[0], "ilp": launch[1],
                                                       "grid": launch[2], "tune_ms": tuned_ms},
            "roofline": {"kernel": "batch_rollout_kernel", "bound": "alu", "pipe": bound,
                         "frac": pipes[bound]["frac"], "kernel_ms_median": 1e3 * k_s,
                         "obstacles_tested_per_rollout_step": tested, "pipes": pipes,
                         "peak_basis": f"{n_sms} SMs x measured lane-ops per SM per clock x {sm_mhz:.0f} MHz"}}


def adjoint_study(torch, steps, rates=None):
    """Config 4: forward update and hand-written adjoint latency (kinematic,
    K = 1024, M = 64, T = 30, softplus barrier), and the main adjoint
    kernel's per-pipe roofline (timed alone by the library's event hook)."""
    from paper_2209_12842_gb300 import RaMppi

    rates = rates or dict(DEFAULT_RATES)
    p = rs.preset("c4_gradient")
    obs = rs.make_obstacles(p["seed"], p["n_obs"], *p["obs_r"])
    ctl = RaMppi(p, obs, differentiable=True)
    x0 = torch.tensor([0.0, -4.0, 0.0, 1.5], device="cuda")
    V = torch.from_numpy(rs.random_controls(0, p["T"], p["u_lo"], p["u_hi"], 5)).cuda()
    gVp, gS = rs.random_cotangents(p["T"], 2, p["K"], 11)
    gVp, gS = torch.from_numpy(gVp).cuda(), torch.from_numpy(gS).cuda()
    stream = torch.cuda.current_stream()
    ctl.tune(x0, V)  # the forward's launch shape (the adjoint reads the same checkpoints for any shape)
    f50, f99 = ev_time(torch, lambda: ctl.step(x0, V), steps, stream)
    ctl.step(x0, V)
    b50, b99 = ev_time(torch, lambda: ctl.backward(gVp, gS), steps, stream)
    kb, ke = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctl.set_timing_events(kb, ke)
    kms = []
    torch.cuda.nvtx.range_push("adjoint_backward")  # lets a profiler select these launches
    for _ in range(steps):
        ctl.backward(gVp, gS)
        torch.cuda.synchronize()
        kms.append(kb.elapsed_time(ke))
    torch.cuda.nvtx.range_pop()
    ctl.set_timing_events(None)
    ctl_launch = ctl.get_launch()
    ctl.close()
    units = p["K"] * p["M"] * p["T"]
    n_sms = torch.cuda.get_device_properties(0).multi_processor_count
    roof = adjoint_roofline(p, float(np.median(kms)) / 1e3, rates, n_sms, 2070.0)
    return {"forward_p50_ms": f50, "forward_p99_ms": f99, "forward_launch": list(ctl_launch),
            "backward_p50_ms": b50, "backward_p99_ms": b99,
            "backward_rollout_steps_per_s": units / b50 * 1e3, "roofline": roof}


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
    `--steps` updates per point (tuned launch) and the rollout kernel's
    per-pipe roofline."""
    import torch

    torch.cuda.set_device(0)
    rates = measure_pipe_rates(torch)["rates_used"]
    base = rs.preset("c5_stress")
    obs = rs.scene_obstacles(base)
    x0 = rs.scene_initial_state(base)
    V = rs.random_controls(base["model"], base["T"], base["u_lo"], base["u_hi"], 3)
    points = []
    for M in (32, 64, 128, 256):
        for alpha in (0.8, 0.95):
            p = rs.preset("c5_stress", M=M, alpha=alpha)
            m = measure_update(torch, p, obs, x0, V, args.steps, args.warmup, args.preroll, rates,
                               ClockSampler(0))
            m["ctl"].close()
            st = m["step_ms"]
            points.append({"M": M, "alpha": alpha, "p50_ms": float(np.percentile(st, 50)),
                           "p99_ms": float(np.percentile(st, 99)),
                           "rollout_steps_per_s": m["units"] / (float(np.median(st)) / 1e3),
                           "launch": m["launch"], "clocks": m["clocks"], "roofline": roofline_summary(m)})
    top = [pt for pt in points if pt["M"] == 256 and pt["alpha"] == 0.95][0]
    line = {"metric": "rollout-steps/s (K*M*T)", "value": top["rollout_steps_per_s"], "unit": "rollout-steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": top["p50_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c5 stress: dynamic single-track, K=65536, T=50, 200 obstacles, sweep of M and alpha",
                       "l2": "inputs resident; per-update working set below L2 (compute bound)"},
            "rates_per_sm_per_clock": rates, "sweep": points}
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
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c5")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-probes", action="store_true",
                    help="skip the pipe-throughput probes (the roofline then uses nominal rates)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-studies", action="store_true",
                    help="skip the other workloads' sections of the line")
    ap.add_argument("--sections", default="",
                    help=f"comma-separated subset of the line's sections ({', '.join(SECTIONS)}); default all")
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
