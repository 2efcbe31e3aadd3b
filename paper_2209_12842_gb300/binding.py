"""ctypes binding of libramppi.so (include/ra_mppi.h), argument marshalling only.

Every step of the RA-MPPI update runs in the library's CUDA kernels; this
module fills the problem struct, passes device pointers (torch tensors'
data_ptr()) and the CUDA stream, and turns status codes into exceptions.
There is no fallback: if the library is missing or fails to load, every
entry point raises.
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libramppi.so")

RA_MPPI_OK = 0
RA_MPPI_EINVAL = -1
RA_MPPI_ENOMEM = -2
RA_MPPI_ECUDA = -3
RA_MPPI_ETIMEOUT = -4
RA_MPPI_ENONFINITE = -5
RA_MPPI_EUNSUPPORTED = -6
STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT",
                -5: "ENONFINITE", -6: "EUNSUPPORTED"}

RA_MPPI_KEEP_RISK_COSTS = 1
RA_MPPI_DIFFERENTIABLE = 2


class RaMppiError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)} {detail}".strip())


class ra_mppi_problem(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int32), ("K", ctypes.c_int32), ("M", ctypes.c_int32),
        ("T", ctypes.c_int32), ("substeps", ctypes.c_int32), ("noise_type", ctypes.c_int32),
        ("obs_mode", ctypes.c_int32), ("cvar_mode", ctypes.c_int32),
        ("risk_mask", ctypes.c_uint32), ("flags", ctypes.c_int32),
        ("dt", ctypes.c_float), ("model_params", ctypes.c_float * 8),
        ("sigma_u", ctypes.c_float * 2), ("u_lo", ctypes.c_float * 2), ("u_hi", ctypes.c_float * 2),
        ("w_scale", ctypes.c_float * 4), ("mix_p", ctypes.c_float), ("mix_scale", ctypes.c_float),
        ("w_dev", ctypes.c_float), ("w_speed", ctypes.c_float), ("v_target", ctypes.c_float),
        ("gamma", ctypes.c_float), ("w_obs", ctypes.c_float), ("w_bdry", ctypes.c_float),
        ("c4", ctypes.c_float), ("c5", ctypes.c_float), ("c_lin", ctypes.c_float),
        ("kappa", ctypes.c_float), ("track_straight", ctypes.c_float),
        ("track_radius", ctypes.c_float), ("track_half_width", ctypes.c_float),
        ("lambda_", ctypes.c_float), ("alpha", ctypes.c_float), ("A", ctypes.c_float),
        ("B", ctypes.c_float), ("C_u", ctypes.c_float), ("eta", ctypes.c_float),
        ("risk_param", ctypes.c_float),
        ("max_obstacles", ctypes.c_int32), ("instance_id", ctypes.c_uint32),
        ("seed", ctypes.c_uint64),
        ("is_scale", ctypes.c_float), ("is_frac", ctypes.c_float),
    ]


class ra_mppi_instance(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("M", ctypes.c_int32), ("T", ctypes.c_int32),
                ("max_obstacles", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("instance_id", ctypes.c_uint32), ("reserved", ctypes.c_int32)]


_VP = ctypes.c_void_p
_FP = ctypes.c_void_p  # float* passed as integer address
_lib = None
_load_error = None


def _declare(L):
    L.ra_mppi_problem_size.restype = ctypes.c_int32
    L.ra_mppi_create.argtypes = [ctypes.POINTER(ra_mppi_problem), ctypes.c_int32, ctypes.POINTER(_VP)]
    L.ra_mppi_destroy.argtypes = [_VP]
    L.ra_mppi_destroy.restype = None
    L.ra_mppi_set_obstacles.argtypes = [_VP, _FP, ctypes.c_int32, _VP]
    L.ra_mppi_step.argtypes = [_VP, _FP, _FP, _FP, _FP, _FP, _VP]
    L.ra_mppi_step_host.argtypes = [_VP, _FP, _FP, _FP, _FP, _VP]
    L.ra_mppi_workspace.argtypes = [_VP] + [ctypes.POINTER(_VP)] * 4
    L.ra_mppi_copy_workspace.argtypes = [_VP, _FP, _FP, _FP, _FP, _VP]
    L.ra_mppi_copy_weights.argtypes = [_VP, _FP, _VP]
    L.ra_mppi_get_state.argtypes = [_VP, ctypes.POINTER(ctypes.c_uint64)]
    L.ra_mppi_set_state.argtypes = [_VP, ctypes.c_uint64]
    L.ra_mppi_get_status.argtypes = [_VP]
    L.ra_mppi_last_error.argtypes = [_VP]
    L.ra_mppi_last_error.restype = ctypes.c_char_p
    L.ra_mppi_set_launch.argtypes = [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    L.ra_mppi_set_timing_events.argtypes = [_VP, _VP, _VP]
    L.ra_mppi_set_tail_split.argtypes = [_VP, ctypes.c_int32]
    L.ra_mppi_set_tail_split.restype = ctypes.c_int
    L.ra_mppi_get_launch_plan.argtypes = [_VP] + [ctypes.POINTER(ctypes.c_int32)] * 4
    L.ra_mppi_get_launch_plan.restype = ctypes.c_int
    L.ra_mppi_set_diagnostics.argtypes = [_VP, _VP]
    L.ra_mppi_set_diagnostics.restype = ctypes.c_int
    L.ra_mppi_tune.argtypes = [_VP, _FP, _FP, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]
    L.ra_mppi_tune.restype = ctypes.c_int
    L.ra_mppi_get_launch.argtypes = [_VP] + [ctypes.POINTER(ctypes.c_int32)] * 3
    L.ra_mppi_get_launch.restype = ctypes.c_int
    L.ra_mppi_set_cost_weights.argtypes = [_VP, ctypes.POINTER(ctypes.c_float)]
    L.ra_mppi_set_cost_weights.restype = ctypes.c_int
    L.ra_mppi_backward.argtypes = [_VP, _FP, _FP, _FP, _FP, _VP]
    L.ra_mppi_backward.restype = ctypes.c_int
    L.ra_mppi_closed_loop_step.argtypes = [_VP, _FP, _FP, _FP, _FP, ctypes.c_int32, _VP]
    L.ra_mppi_closed_loop_step.restype = ctypes.c_int
    L.ra_mppi_softmin_update_noalloc.argtypes = [_FP, _FP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_float, _FP, _VP]
    L.ra_mppi_softmin_update_noalloc.restype = ctypes.c_int
    L.ra_mppi_pipe_probe.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_float),
                                     ctypes.POINTER(ctypes.c_double)]
    L.ra_mppi_pipe_probe.restype = ctypes.c_int
    _I64P = ctypes.POINTER(ctypes.c_int64)
    _I32P = ctypes.POINTER(ctypes.c_int32)
    L.ra_mppi_batch_create.argtypes = [ctypes.POINTER(ra_mppi_problem), ctypes.POINTER(ra_mppi_instance),
                                       ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_VP)]
    L.ra_mppi_batch_io.argtypes = [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I64P]
    L.ra_mppi_batch_destroy.argtypes = [_VP]
    L.ra_mppi_batch_destroy.restype = None
    L.ra_mppi_batch_layout.argtypes = [_VP, _I64P]
    L.ra_mppi_batch_buffers.argtypes = [_VP] + [ctypes.POINTER(_VP)] * 4
    L.ra_mppi_batch_set_obstacles.argtypes = [_VP, ctypes.c_int32, _FP, ctypes.c_int32, _VP]
    L.ra_mppi_batch_write_inputs.argtypes = [_VP, _FP, _FP, _VP]
    L.ra_mppi_batch_read_outputs.argtypes = [_VP, _FP, _FP, _VP]
    L.ra_mppi_step_batched.argtypes = [_VP, _VP]
    L.ra_mppi_step_batched_eager.argtypes = [_VP, _VP]
    L.ra_mppi_batch_copy_workspace.argtypes = [_VP, _FP, _FP, _FP, _VP]
    L.ra_mppi_batch_set_iteration.argtypes = [_VP, ctypes.c_uint64]
    L.ra_mppi_batch_get_status.argtypes = [_VP]
    L.ra_mppi_batch_set_launch.argtypes = [_VP, ctypes.c_int32, ctypes.c_int32]
    L.ra_mppi_batch_set_timing_events.argtypes = [_VP, _VP, _VP]
    L.ra_mppi_batch_set_diagnostics.argtypes = [_VP, _VP]
    L.ra_mppi_batch_get_launch.argtypes = [_VP, _I32P, _I32P, _I32P]
    L.ra_mppi_batch_tune.argtypes = [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]
    L.ra_mppi_batch_last_error.argtypes = [_VP]
    L.ra_mppi_batch_last_error.restype = ctypes.c_char_p
    for name in ("ra_mppi_batch_create", "ra_mppi_batch_io", "ra_mppi_batch_layout", "ra_mppi_batch_buffers",
                 "ra_mppi_batch_set_obstacles", "ra_mppi_step_batched", "ra_mppi_step_batched_eager",
                 "ra_mppi_batch_write_inputs", "ra_mppi_batch_read_outputs",
                 "ra_mppi_batch_copy_workspace", "ra_mppi_batch_set_iteration", "ra_mppi_batch_get_status",
                 "ra_mppi_batch_set_launch", "ra_mppi_batch_get_launch", "ra_mppi_batch_tune",
                 "ra_mppi_batch_set_timing_events", "ra_mppi_batch_set_diagnostics"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("ra_mppi_create", "ra_mppi_set_obstacles", "ra_mppi_step", "ra_mppi_step_host",
                 "ra_mppi_workspace", "ra_mppi_copy_workspace", "ra_mppi_copy_weights", "ra_mppi_get_state",
                 "ra_mppi_set_state", "ra_mppi_get_status", "ra_mppi_set_launch", "ra_mppi_set_timing_events"):
        getattr(L, name).restype = ctypes.c_int


def lib():
    """The loaded library; raises if it has not been built or cannot load."""
    global _lib, _load_error
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it with `python -m paper_2209_12842_gb300.build` "
            "(there is no CPU fallback)")
    try:
        L = ctypes.CDLL(LIB_PATH)
    except OSError as e:  # pragma: no cover - depends on the host
        _load_error = e
        raise RuntimeError(f"cannot load {LIB_PATH}: {e}") from e
    _declare(L)
    if L.ra_mppi_problem_size() != ctypes.sizeof(ra_mppi_problem):
        raise RuntimeError("ra_mppi_problem layout mismatch between binding and library")
    _lib = L
    return _lib


def _f(v):
    return float(v)


def ra_mppi_problem_from(p, flags=0, max_obstacles=None):
    """Fill the C problem struct from a preset dict (see ra_scenes.presets)."""
    pr = ra_mppi_problem()
    for name in ("model", "K", "M", "T", "substeps", "noise_type", "obs_mode", "cvar_mode"):
        setattr(pr, name, int(p[name]))
    pr.risk_mask = int(p["risk_mask"])
    pr.flags = int(flags)
    pr.dt = _f(p["dt"])
    for i in range(8):
        pr.model_params[i] = _f(p["model_params"][i])
    for i in range(2):
        pr.sigma_u[i] = _f(p["sigma_u"][i])
        pr.u_lo[i] = _f(p["u_lo"][i])
        pr.u_hi[i] = _f(p["u_hi"][i])
    for i in range(4):
        pr.w_scale[i] = _f(p["w_scale"][i])
    for name in ("mix_p", "mix_scale", "w_dev", "w_speed", "v_target", "gamma", "w_obs", "w_bdry",
                 "c4", "c5", "c_lin", "kappa", "track_straight", "track_radius", "track_half_width",
                 "alpha", "A", "B", "C_u", "eta", "risk_param"):
        setattr(pr, name, _f(p[name]))
    pr.lambda_ = _f(p["lam"])
    n_obs = int(p.get("n_obs", 0))
    pr.max_obstacles = int(max_obstacles if max_obstacles is not None else max(n_obs, 1))
    pr.instance_id = int(p["instance_id"]) & 0xFFFFFFFF
    pr.seed = int(p["seed"]) & 0xFFFFFFFFFFFFFFFF
    pr.is_scale = _f(p.get("is_scale", 1.0))
    pr.is_frac = _f(p.get("is_frac", 0.0))
    return pr


def _check(rc, where, handle=None):
    if rc != RA_MPPI_OK:
        detail = ""
        if handle:
            msg = lib().ra_mppi_last_error(handle)
            detail = msg.decode() if msg else ""
        raise RaMppiError(rc, where, detail)


# ------------------------------------------------------------------ C names

def ra_mppi_create(problem, device=-1):
    h = _VP()
    _check(lib().ra_mppi_create(ctypes.byref(problem), int(device), ctypes.byref(h)), "ra_mppi_create")
    return h


def ra_mppi_destroy(h):
    lib().ra_mppi_destroy(h)


def ra_mppi_set_obstacles(h, xyr_ptr, n_obs, stream=0):
    _check(lib().ra_mppi_set_obstacles(h, xyr_ptr, int(n_obs), stream), "ra_mppi_set_obstacles", h)


def ra_mppi_step(h, x0_ptr, V_in_ptr, V_out_ptr, S_tilde_ptr=None, cvar_ptr=None, stream=0):
    _check(lib().ra_mppi_step(h, x0_ptr, V_in_ptr, V_out_ptr, S_tilde_ptr, cvar_ptr, stream),
           "ra_mppi_step", h)


def ra_mppi_step_host(h, x0_ptr, V_in_ptr, V_out_ptr, S_tilde_ptr=None, stream=0):
    _check(lib().ra_mppi_step_host(h, x0_ptr, V_in_ptr, V_out_ptr, S_tilde_ptr, stream),
           "ra_mppi_step_host", h)


def ra_mppi_closed_loop_step(h, x_ptr, V_ptr, S_tilde_ptr=None, collisions_ptr=None, shift=1, stream=0):
    _check(lib().ra_mppi_closed_loop_step(h, x_ptr, V_ptr, S_tilde_ptr, collisions_ptr, int(shift), stream),
           "ra_mppi_closed_loop_step", h)


def ra_mppi_set_diagnostics(h, counter_ptr=None):
    _check(lib().ra_mppi_set_diagnostics(h, counter_ptr), "ra_mppi_set_diagnostics", h)


def ra_mppi_tune(h, x0_ptr, V_ptr, replays=3):
    ms = ctypes.c_float()
    _check(lib().ra_mppi_tune(h, x0_ptr, V_ptr, int(replays), ctypes.byref(ms)), "ra_mppi_tune", h)
    return ms.value


def ra_mppi_get_launch(h):
    w, i, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().ra_mppi_get_launch(h, ctypes.byref(w), ctypes.byref(i), ctypes.byref(g)), "ra_mppi_get_launch", h)
    return w.value, i.value, g.value


def ra_mppi_set_cost_weights(h, theta):
    arr = (ctypes.c_float * 4)(*[float(v) for v in theta])
    _check(lib().ra_mppi_set_cost_weights(h, arr), "ra_mppi_set_cost_weights", h)


def ra_mppi_backward(h, gV_plus_ptr, gS_tilde_ptr, gV_ptr, gtheta_ptr, stream=0):
    _check(lib().ra_mppi_backward(h, gV_plus_ptr, gS_tilde_ptr, gV_ptr, gtheta_ptr, stream), "ra_mppi_backward", h)


def ra_mppi_workspace(h):
    ptrs = [_VP() for _ in range(4)]
    _check(lib().ra_mppi_workspace(h, *[ctypes.byref(p) for p in ptrs]), "ra_mppi_workspace", h)
    return [p.value for p in ptrs]


def ra_mppi_copy_weights(h, W_ptr, stream=0):
    _check(lib().ra_mppi_copy_weights(h, W_ptr, stream), "ra_mppi_copy_weights", h)


def ra_mppi_copy_workspace(h, U_ptr=None, S_ptr=None, cvar_ptr=None, L_ptr=None, stream=0):
    _check(lib().ra_mppi_copy_workspace(h, U_ptr, S_ptr, cvar_ptr, L_ptr, stream),
           "ra_mppi_copy_workspace", h)


def ra_mppi_get_state(h):
    it = ctypes.c_uint64()
    _check(lib().ra_mppi_get_state(h, ctypes.byref(it)), "ra_mppi_get_state", h)
    return it.value


def ra_mppi_set_state(h, iteration):
    _check(lib().ra_mppi_set_state(h, int(iteration)), "ra_mppi_set_state", h)


def ra_mppi_get_status(h):
    return lib().ra_mppi_get_status(h)


def ra_mppi_last_error(h):
    msg = lib().ra_mppi_last_error(h)
    return msg.decode() if msg else ""


def ra_mppi_set_launch(h, warps_per_block=0, ilp=0, warps_per_sample=0):
    _check(lib().ra_mppi_set_launch(h, int(warps_per_block), int(ilp), int(warps_per_sample)),
           "ra_mppi_set_launch", h)


def ra_mppi_set_tail_split(h, enable):
    _check(lib().ra_mppi_set_tail_split(h, 1 if enable else 0), "ra_mppi_set_tail_split", h)


def ra_mppi_get_launch_plan(h):
    """(grid, first tail block or -1, tail warps per sample, blocks per SM)."""
    v = [ctypes.c_int32() for _ in range(4)]
    _check(lib().ra_mppi_get_launch_plan(h, *[ctypes.byref(x) for x in v]), "ra_mppi_get_launch_plan", h)
    return tuple(x.value for x in v)


def ra_mppi_set_timing_events(h, begin_event_handle=None, end_event_handle=None):
    _check(lib().ra_mppi_set_timing_events(h, begin_event_handle, end_event_handle),
           "ra_mppi_set_timing_events", h)


def ra_mppi_softmin_update_noalloc(S_tilde_ptr, U_ptr, K, T, nu, lam, V_out_ptr, stream=0):
    """Softmin-weighted update from caller buffers, without any allocation."""
    return lib().ra_mppi_softmin_update_noalloc(S_tilde_ptr, U_ptr, int(K), int(T), int(nu), float(lam),
                                                V_out_ptr, stream)


def ra_mppi_pipe_probe(kind, iters, device=-1):
    """(ms, lane_ops) of one pipe-throughput probe launch (see the header)."""
    ms, ops = ctypes.c_float(), ctypes.c_double()
    _check(lib().ra_mppi_pipe_probe(int(kind), int(iters), int(device), ctypes.byref(ms), ctypes.byref(ops)),
           "ra_mppi_pipe_probe")
    return ms.value, ops.value


# ------------------------------------------------------------------ batched path

def _bcheck(rc, where, b=None):
    if rc != RA_MPPI_OK:
        detail = ""
        if b:
            msg = lib().ra_mppi_batch_last_error(b)
            detail = msg.decode() if msg else ""
        raise RaMppiError(rc, where, detail)


def ra_mppi_batch_create(problem, instances, device=-1):
    arr = (ra_mppi_instance * len(instances))(*instances)
    b = _VP()
    _bcheck(lib().ra_mppi_batch_create(ctypes.byref(problem), arr, len(instances), int(device), ctypes.byref(b)),
            "ra_mppi_batch_create")
    return b


def ra_mppi_batch_io(b, n):
    """(x0_packed, V_packed, offsets): the library-owned input buffers and the
    per-problem offsets (as ra_mppi_batch_layout)."""
    x0, V = _VP(), _VP()
    off = (ctypes.c_int64 * (4 * n))()
    _bcheck(lib().ra_mppi_batch_io(b, ctypes.byref(x0), ctypes.byref(V), off), "ra_mppi_batch_io", b)
    return x0.value, V.value, [tuple(off[4 * i:4 * i + 4]) for i in range(n)]


def ra_mppi_batch_destroy(b):
    lib().ra_mppi_batch_destroy(b)


def ra_mppi_batch_layout(b, n):
    off = (ctypes.c_int64 * (4 * n))()
    _bcheck(lib().ra_mppi_batch_layout(b, off), "ra_mppi_batch_layout", b)
    return [tuple(off[4 * i:4 * i + 4]) for i in range(n)]


def ra_mppi_batch_buffers(b):
    ptrs = [_VP() for _ in range(4)]
    _bcheck(lib().ra_mppi_batch_buffers(b, *[ctypes.byref(p) for p in ptrs]), "ra_mppi_batch_buffers", b)
    return [p.value for p in ptrs]


def ra_mppi_batch_set_obstacles(b, i, xyr_ptr, n_obs, stream=0):
    _bcheck(lib().ra_mppi_batch_set_obstacles(b, int(i), xyr_ptr, int(n_obs), stream),
            "ra_mppi_batch_set_obstacles", b)


def ra_mppi_batch_write_inputs(b, x0_ptr=None, V_ptr=None, stream=0):
    _bcheck(lib().ra_mppi_batch_write_inputs(b, x0_ptr, V_ptr, stream), "ra_mppi_batch_write_inputs", b)


def ra_mppi_batch_read_outputs(b, V_out_ptr=None, S_tilde_ptr=None, stream=0):
    _bcheck(lib().ra_mppi_batch_read_outputs(b, V_out_ptr, S_tilde_ptr, stream), "ra_mppi_batch_read_outputs", b)


def ra_mppi_step_batched(b, stream=0):
    _bcheck(lib().ra_mppi_step_batched(b, stream), "ra_mppi_step_batched", b)


def ra_mppi_step_batched_eager(b, stream=0):
    _bcheck(lib().ra_mppi_step_batched_eager(b, stream), "ra_mppi_step_batched_eager", b)


def ra_mppi_batch_copy_workspace(b, U_ptr=None, S_ptr=None, cvar_ptr=None, stream=0):
    _bcheck(lib().ra_mppi_batch_copy_workspace(b, U_ptr, S_ptr, cvar_ptr, stream),
            "ra_mppi_batch_copy_workspace", b)


def ra_mppi_batch_set_iteration(b, iteration):
    _bcheck(lib().ra_mppi_batch_set_iteration(b, int(iteration)), "ra_mppi_batch_set_iteration", b)


def ra_mppi_batch_get_status(b):
    return lib().ra_mppi_batch_get_status(b)


def ra_mppi_batch_set_launch(b, warps_per_block, ilp):
    _bcheck(lib().ra_mppi_batch_set_launch(b, int(warps_per_block), int(ilp)), "ra_mppi_batch_set_launch", b)


def ra_mppi_batch_get_launch(b):
    w, i, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _bcheck(lib().ra_mppi_batch_get_launch(b, ctypes.byref(w), ctypes.byref(i), ctypes.byref(g)),
            "ra_mppi_batch_get_launch", b)
    return w.value, i.value, g.value


def ra_mppi_batch_set_timing_events(b, begin_event_handle=None, end_event_handle=None):
    _bcheck(lib().ra_mppi_batch_set_timing_events(b, begin_event_handle, end_event_handle),
            "ra_mppi_batch_set_timing_events", b)


def ra_mppi_batch_set_diagnostics(b, counter_ptr=None):
    _bcheck(lib().ra_mppi_batch_set_diagnostics(b, counter_ptr), "ra_mppi_batch_set_diagnostics", b)


def ra_mppi_batch_tune(b, replays=3):
    ms = ctypes.c_float()
    _bcheck(lib().ra_mppi_batch_tune(b, int(replays), ctypes.byref(ms)), "ra_mppi_batch_tune", b)
    return ms.value
