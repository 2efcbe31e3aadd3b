"""FP64 CPU oracle of one RA-MPPI control update (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does, and
this package never imports the product.

The arithmetic lives in ``ra_mppi_oracle.c`` (plain C, float64, loops in
the order of the paper's Algorithm 1).  This module only builds that file
with gcc and marshals numpy arrays through ctypes.  Inputs are taken as the
float32 values the CUDA path receives, promoted to float64.
"""

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ra_mppi_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile the oracle with gcc (no FMA contraction, OpenMP over samples)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Problem(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int32), ("K", ctypes.c_int32), ("M", ctypes.c_int32),
        ("T", ctypes.c_int32), ("substeps", ctypes.c_int32),
        ("noise_type", ctypes.c_int32), ("obs_mode", ctypes.c_int32),
        ("cvar_mode", ctypes.c_int32), ("risk_mask", ctypes.c_uint32),
        ("n_threads", ctypes.c_int32),
        ("dt", ctypes.c_double),
        ("model_params", ctypes.c_double * 8),
        ("sigma_u", ctypes.c_double * 2), ("u_lo", ctypes.c_double * 2),
        ("u_hi", ctypes.c_double * 2),
        ("w_scale", ctypes.c_double * 4),
        ("mix_p", ctypes.c_double), ("mix_scale", ctypes.c_double),
        ("w_dev", ctypes.c_double), ("w_speed", ctypes.c_double),
        ("v_target", ctypes.c_double), ("gamma", ctypes.c_double),
        ("w_obs", ctypes.c_double), ("w_bdry", ctypes.c_double),
        ("c4", ctypes.c_double), ("c5", ctypes.c_double), ("c_lin", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("track_straight", ctypes.c_double), ("track_radius", ctypes.c_double),
        ("track_half_width", ctypes.c_double),
        ("lam", ctypes.c_double), ("alpha", ctypes.c_double), ("A", ctypes.c_double),
        ("B", ctypes.c_double), ("C_u", ctypes.c_double), ("eta", ctypes.c_double),
        ("band_delta", ctypes.c_double), ("risk_param", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("iteration", ctypes.c_uint64),
        ("instance_id", ctypes.c_uint32), ("pad_", ctypes.c_uint32),
        ("is_scale", ctypes.c_double), ("is_frac", ctypes.c_double),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_I32 = ctypes.POINTER(ctypes.c_int32)
_P = ctypes.POINTER(Problem)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.orc_philox.argtypes = [_U32, _U32, _U32]
        L.orc_uniform.argtypes = [ctypes.c_uint32]
        L.orc_uniform.restype = ctypes.c_double
        L.orc_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _D]
        L.orc_mix_value.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double]
        L.orc_mix_value.restype = ctypes.c_double
        L.orc_control_noise.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _D]
        L.orc_process_noise.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _D]
        L.orc_dynamics.argtypes = [_P, _D, _D, _D]
        L.orc_track.argtypes = [_P, ctypes.c_double, ctypes.c_double, _D]
        L.orc_cvar.argtypes = [_D, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32]
        L.orc_cvar.restype = ctypes.c_double
        L.orc_risk.argtypes = [_D, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                               ctypes.c_double]
        L.orc_risk.restype = ctypes.c_double
        L.orc_risk_w.argtypes = [_D, _D, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                 ctypes.c_double]
        L.orc_risk_w.restype = ctypes.c_double
        L.orc_is_weights.argtypes = [_P, ctypes.c_int32, _D]
        L.orc_is_weights.restype = ctypes.c_int32
        L.orc_samples.argtypes = [_P, _D, _D, _D, ctypes.c_int32, _I32, ctypes.c_int32] + [_D] * 11
        L.orc_samples.restype = ctypes.c_int32
        L.orc_update.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                 _D, _D, _D, _D]
        L.orc_update.restype = ctypes.c_int32
        L.orc_plant_step.argtypes = [_P, ctypes.c_uint64, _D, _D, _D, ctypes.c_int32, _D]
        L.orc_plant_step.restype = ctypes.c_int32
        L.orc_state_cost.argtypes = [_P, _D, _D, ctypes.c_int32, ctypes.c_uint32]
        L.orc_state_cost.restype = ctypes.c_double
        L.orc_terminal_cost.argtypes = [_P, _D]
        L.orc_terminal_cost.restype = ctypes.c_double
        L.orc_sizeof_problem.restype = ctypes.c_int32
        L.orc_n_warm.argtypes = [_P]
        L.orc_n_warm.restype = ctypes.c_int32
        L.orc_backward.argtypes = [_P, _D, _D, _D, ctypes.c_int32, _D, _D, _D, _D]
        L.orc_backward.restype = ctypes.c_int32
        assert L.orc_sizeof_problem() == ctypes.sizeof(Problem)
        _lib = L
    return _lib


def _f32(v):
    return float(np.float32(v))


def _arr(a, dtype=np.float64):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _ptr(a, typ=_D):
    if a is None:
        return ctypes.cast(None, typ)
    return a.ctypes.data_as(typ)


def make_problem(p, iteration=0, band_delta=1e-4, n_threads=1, exact=False):
    """Oracle problem from a preset dict; reals are rounded to float32 first
    (exact=True keeps them as given, for finite differences)."""
    _f32 = (lambda v: float(v)) if exact else globals()["_f32"]
    pr = Problem()
    for name in ("model", "K", "M", "T", "substeps", "noise_type", "obs_mode", "cvar_mode"):
        setattr(pr, name, int(p[name]))
    pr.risk_mask = int(p["risk_mask"])
    pr.n_threads = int(n_threads)
    pr.dt = _f32(p["dt"])
    for i in range(8):
        pr.model_params[i] = _f32(p["model_params"][i])
    for i in range(2):
        pr.sigma_u[i] = _f32(p["sigma_u"][i])
        pr.u_lo[i] = _f32(p["u_lo"][i])
        pr.u_hi[i] = _f32(p["u_hi"][i])
    for i in range(4):
        pr.w_scale[i] = _f32(p["w_scale"][i])
    for name in ("mix_p", "mix_scale", "w_dev", "w_speed", "v_target", "gamma", "w_obs",
                 "w_bdry", "c4", "c5", "c_lin", "kappa", "track_straight", "track_radius",
                 "track_half_width", "lam", "alpha", "A", "B", "C_u", "eta", "risk_param"):
        setattr(pr, name, _f32(p[name]))
    pr.band_delta = float(band_delta)
    pr.seed = int(p["seed"]) & 0xFFFFFFFFFFFFFFFF
    pr.iteration = int(iteration)
    pr.instance_id = int(p["instance_id"]) & 0xFFFFFFFF
    pr.is_scale = _f32(p.get("is_scale", 1.0))
    pr.is_frac = _f32(p.get("is_frac", 0.0))
    return pr


def nx_nu(p):
    m = int(p["model"])
    return (4, 2) if m == 0 else (6, 2) if m == 1 else (1, 1)


# ---------------------------------------------------------------- primitives

def philox(ctr, key):
    c = _arr(ctr, np.uint32)
    k = _arr(key, np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_ptr(c, _U32), _ptr(k, _U32), _ptr(out, _U32))
    return out


def uniform(x):
    return lib().orc_uniform(int(x))


def box_muller(a, b):
    out = np.zeros(2)
    lib().orc_box_muller(int(a), int(b), _ptr(out))
    return out


def mix_value(sel, word, b, p, mix_scale):
    return lib().orc_mix_value(int(sel), int(word), float(b), float(p), float(mix_scale))


def control_noise(prob, k, t):
    out = np.zeros(2)
    lib().orc_control_noise(ctypes.byref(prob), int(k), int(t), _ptr(out))
    return out


def process_noise(prob, k, m, t):
    out = np.zeros(4)
    lib().orc_process_noise(ctypes.byref(prob), int(k), int(m), int(t), _ptr(out))
    return out


def dynamics(prob, x, u):
    x = _arr(x)
    u = _arr(u)
    xn = np.zeros(6)
    lib().orc_dynamics(ctypes.byref(prob), _ptr(x), _ptr(u), _ptr(xn))
    return xn[: len(x)]


def track(prob, px, py):
    out = np.zeros(3)
    lib().orc_track(ctypes.byref(prob), float(px), float(py), _ptr(out))
    return out  # e, s, d


def state_cost(prob, x, obs, mask):
    x = _arr(x)
    o = _arr(np.asarray(obs, dtype=np.float32).reshape(-1, 3) if len(obs) else np.zeros((0, 3)))
    return lib().orc_state_cost(ctypes.byref(prob), _ptr(x), _ptr(o), int(len(o)), int(mask))


def terminal_cost(prob, x):
    x = _arr(x)
    return lib().orc_terminal_cost(ctypes.byref(prob), _ptr(x))


def cvar(L, alpha, B=1.0, mode=0):
    L = _arr(L)
    return lib().orc_cvar(_ptr(L), int(L.size), float(alpha), float(B), int(mode))


def risk(L, alpha, B=1.0, mode=0, threshold=0.0):
    """Risk measure of a set of risk costs (CVaR forms, VaR, chance, mean)."""
    L = _arr(L)
    return lib().orc_risk(_ptr(L), int(L.size), float(alpha), float(B), int(mode), float(threshold))


def risk_w(L, w, alpha, B=1.0, mode=0, threshold=0.0):
    """Risk measure of the weighted empirical distribution of the risk costs
    L with weights w (None: all equal)."""
    L = _arr(L)
    w = None if w is None else _arr(w)
    return lib().orc_risk_w(_ptr(L), _ptr(w), int(L.size), float(alpha), float(B), int(mode), float(threshold))


def is_weights(p, k, iteration=0):
    """Importance weights of the M disturbed rollouts of sample k (all 1 when
    importance sampling is off)."""
    prob = make_problem(p, iteration)
    w = np.zeros(int(p["M"]))
    rc = lib().orc_is_weights(ctypes.byref(prob), int(k), _ptr(w))
    if rc != 0:
        raise RuntimeError(f"orc_is_weights failed: {rc}")
    return w


def n_warm(prob):
    return lib().orc_n_warm(ctypes.byref(prob))


# ---------------------------------------------------------------- pipeline

def samples(p, x0, V, obs, ks=None, iteration=0, band_delta=1e-4, n_threads=1, want_L=False, exact=False):
    """Per-sample stage of one update for the sample indices ks (default all)."""
    prob = make_problem(p, iteration, band_delta, n_threads, exact=exact)
    nx, nu = nx_nu(p)
    K, M, T = int(p["K"]), int(p["M"]), int(p["T"])
    ks = np.arange(K, dtype=np.int32) if ks is None else _arr(ks, np.int32)
    nk = int(ks.size)
    cast = np.float64 if exact else np.float32
    x0 = _arr(np.asarray(x0, dtype=cast))
    V = _arr(np.asarray(V, dtype=cast).reshape(T, nu))
    o = _arr(np.asarray(obs, dtype=np.float32).reshape(-1, 3)) if len(obs) else np.zeros((0, 3))
    out = {name: np.zeros(nk) for name in ("S", "cvar", "S_tilde", "S_lo", "S_hi", "cvar_lo",
                                          "cvar_hi", "St_lo", "St_hi")}
    out["U"] = np.zeros((nk, T, nu))
    Lbuf = np.zeros((nk, M)) if want_L else None
    rc = lib().orc_samples(ctypes.byref(prob), _ptr(x0), _ptr(V), _ptr(o), int(len(o)),
                           _ptr(ks, _I32), nk, _ptr(out["U"]), _ptr(out["S"]), _ptr(Lbuf),
                           _ptr(out["cvar"]), _ptr(out["S_tilde"]), _ptr(out["S_lo"]),
                           _ptr(out["S_hi"]), _ptr(out["cvar_lo"]), _ptr(out["cvar_hi"]),
                           _ptr(out["St_lo"]), _ptr(out["St_hi"]))
    if rc != 0:
        raise RuntimeError(f"orc_samples failed: {rc}")
    if want_L:
        out["L"] = Lbuf
    out["ks"] = ks
    return out


def update(S_tilde, U, lam):
    """Softmin weights and V+ (Eqs. 4, 5, 17) on given costs and controls."""
    S_tilde = _arr(S_tilde)
    U = _arr(U)
    K, T, nu = U.shape
    Vp = np.zeros((T, nu))
    w = np.zeros(K)
    rc = lib().orc_update(K, T, nu, float(lam), _ptr(S_tilde), _ptr(U), _ptr(Vp), _ptr(w))
    if rc != 0:
        raise RuntimeError(f"orc_update failed: {rc}")
    return Vp, w


def step(p, x0, V, obs, iteration=0, band_delta=1e-4, n_threads=1, want_L=False, exact=False):
    """One full RA-MPPI update: per-sample stage for all k, then the update."""
    out = samples(p, x0, V, obs, None, iteration, band_delta, n_threads, want_L, exact=exact)
    Vp, w = update(out["S_tilde"], out["U"], float(p["lam"]) if exact else _f32(p["lam"]))
    out["V_plus"] = Vp
    out["weights"] = w
    return out


def plant_step(p, x, u, iteration, obs):
    prob = make_problem(p, iteration)
    x = _arr(x)
    u = _arr(u)
    o = _arr(np.asarray(obs, dtype=np.float32).reshape(-1, 3)) if len(obs) else np.zeros((0, 3))
    xo = np.zeros(6)
    hit = lib().orc_plant_step(ctypes.byref(prob), int(iteration), _ptr(x), _ptr(u), _ptr(o),
                               int(len(o)), _ptr(xo))
    return xo[: len(x)], np.array([hit & 1, (hit >> 1) & 1])


def closed_loop(p, x0, V0, obs, n_updates, shift=True, iteration0=0, n_threads=1):
    """Receding-horizon loop of Alg. 1 on a simulated plant (small cases).

    Each iteration: update from the current plant state, apply v0+ to the
    plant (its own noise stream), then warm-start V from V+ (shifted left by
    one step with the last control repeated when `shift`).  Returns the
    states, the V+ sequence and the counts (steps inside an obstacle, steps
    off the track).
    """
    x = np.asarray(x0, dtype=np.float64).copy()
    V = np.asarray(V0, dtype=np.float64).copy()
    xs, Vs, hits = [x.copy()], [], np.zeros(2, dtype=np.int64)
    for n in range(n_updates):
        it = iteration0 + n
        out = step(p, x.astype(np.float32), V.astype(np.float32), obs, it, n_threads=n_threads)
        Vp = out["V_plus"]
        Vs.append(Vp.copy())
        x, hit = plant_step(p, x, Vp[0], it, obs)
        hits += hit
        xs.append(x.copy())
        V = np.concatenate([Vp[1:], Vp[-1:]], 0) if shift else Vp
    return np.array(xs), np.array(Vs), hits


THETA_NAMES = ("w_dev", "w_speed", "gamma", "w_obs")


def backward(p, x0, V, obs, gV_plus, gS_tilde=None, iteration=0, exact=False):
    """Analytic vector-Jacobian product of one update: gradients of
    <gV_plus, V+> + <gS_tilde, S~> w.r.t. V [T, nu] and theta =
    (w_dev, w_speed, gamma, w_obs)."""
    prob = make_problem(p, iteration, exact=exact)
    nx, nu = nx_nu(p)
    T, K = int(p["T"]), int(p["K"])
    cast = np.float64 if exact else np.float32
    x0 = _arr(np.asarray(x0, dtype=cast))
    V = _arr(np.asarray(V, dtype=cast).reshape(T, nu))
    o = _arr(np.asarray(obs, dtype=np.float32).reshape(-1, 3)) if len(obs) else np.zeros((0, 3))
    gVp = _arr(np.asarray(gV_plus, dtype=np.float64).reshape(T, nu))
    gS = None if gS_tilde is None else _arr(np.asarray(gS_tilde, dtype=np.float64).reshape(K))
    gV = np.zeros((T, nu))
    gth = np.zeros(4)
    rc = lib().orc_backward(ctypes.byref(prob), _ptr(x0), _ptr(V), _ptr(o), int(len(o)), _ptr(gVp),
                            _ptr(gS), _ptr(gV), _ptr(gth))
    if rc != 0:
        raise RuntimeError(f"orc_backward failed: {rc}")
    return gV, gth


def objective(p, x0, V, obs, gV_plus, gS_tilde=None, iteration=0, theta=None):
    """<gV_plus, V+> + <gS_tilde, S~> of one update in float64 (for finite
    differences); theta overrides (w_dev, w_speed, gamma, w_obs)."""
    q = dict(p)
    if theta is not None:
        for name, v in zip(THETA_NAMES, theta):
            q[name] = float(v)
    out = step(q, x0, V, obs, iteration=iteration, exact=True)
    val = float(np.sum(np.asarray(gV_plus) * out["V_plus"]))
    if gS_tilde is not None:
        val += float(np.sum(np.asarray(gS_tilde) * out["S_tilde"]))
    return val
