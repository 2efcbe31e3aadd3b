"""Seeded scene and state generators (inputs only, float32-exact).

Obstacles are placed "uniform on the track" by rejection sampling: a point is
drawn uniformly in the stadium's bounding box and kept when it lies within
the track band, so the accepted points are uniform by area.  A keep-out disc
around the start position keeps the first state collision free.
"""

import math

import numpy as np

from .presets import (
    MODEL_DYN_SINGLE_TRACK,
    MODEL_KIN_BICYCLE,
    MODEL_LINEAR_TEST,
    model_dims,
)

BASE_SEED = 12842
_KEEP_OUT = 0.8  # metres around the start position free of obstacle centres


def _in_band(px, py, straight, radius, half_width):
    half = 0.5 * straight
    if abs(px) <= half:
        dist = abs(abs(py) - radius)
    else:
        dist = abs(math.hypot(abs(px) - half, py) - radius)
    return dist <= half_width


def make_obstacles(seed, n, r_lo, r_hi, straight=10.0, radius=4.0,
                   half_width=1.0, start=(0.0, -4.0)):
    """(n, 3) float32 array of obstacle circles (x, y, r), seeded."""
    rng = np.random.default_rng(seed)
    out = np.zeros((n, 3), dtype=np.float32)
    half = 0.5 * straight
    xmax = half + radius + half_width
    ymax = radius + half_width
    i = 0
    while i < n:
        px = rng.uniform(-xmax, xmax)
        py = rng.uniform(-ymax, ymax)
        if not _in_band(px, py, straight, radius, half_width):
            continue
        if math.hypot(px - start[0], py - start[1]) < _KEEP_OUT:
            continue
        r = rng.uniform(r_lo, r_hi) if r_hi > r_lo else r_lo
        out[i] = (px, py, r)
        i += 1
    return out


def obstacles_ahead(seed, n, r_lo, r_hi, x_from=0.3, x_to=2.5, y_center=-4.0,
                    lateral=0.6):
    """(n, 3) float32 obstacles scattered on the straight just ahead of the
    start, so that short horizons from rest still meet them (dense-hit
    parity scenes)."""
    rng = np.random.default_rng(seed)
    out = np.zeros((n, 3), dtype=np.float32)
    for i in range(n):
        out[i, 0] = rng.uniform(x_from, x_to)
        out[i, 1] = y_center + rng.uniform(-lateral, lateral)
        out[i, 2] = rng.uniform(r_lo, r_hi) if r_hi > r_lo else r_lo
    return out


def scene_obstacles(p, seed=None):
    """The preset's obstacle field on its own track (seeded by the preset)."""
    R = float(p["track_radius"])
    return make_obstacles(p["seed"] if seed is None else seed, int(p["n_obs"]), *p["obs_r"],
                          straight=float(p["track_straight"]), radius=R,
                          half_width=float(p["track_half_width"]), start=(0.0, -R))


def scene_initial_state(p):
    """Start at the preset's track origin (0, -R) heading along +x."""
    return initial_state(int(p["model"]), radius=float(p["track_radius"]))


def initial_state(model, radius=4.0):
    """Start at the track origin (0, -R) heading along +x."""
    if model == MODEL_KIN_BICYCLE:
        x = [0.0, -radius, 0.0, 0.0]
    elif model == MODEL_DYN_SINGLE_TRACK:
        x = [0.0, -radius, 0.0, 1.0, 0.0, 0.0]
    elif model == MODEL_LINEAR_TEST:
        x = [0.0]
    else:
        raise ValueError(model)
    return np.asarray(x, dtype=np.float32)


def zero_controls(model, T):
    nx, nu, _ = model_dims(model)
    return np.zeros((T, nu), dtype=np.float32)


def random_controls(model, T, u_lo, u_hi, seed):
    """Warm-start controls drawn uniformly inside the control box."""
    nx, nu, _ = model_dims(model)
    rng = np.random.default_rng(seed)
    lo = np.asarray(u_lo[:nu], dtype=np.float64)
    hi = np.asarray(u_hi[:nu], dtype=np.float64)
    lo = np.maximum(lo, -10.0)
    hi = np.minimum(hi, 10.0)
    return rng.uniform(lo, hi, size=(T, nu)).astype(np.float32)


def batched_instances(B, seed=BASE_SEED):
    """Per-instance sizes of the uneven batched workload.

    K log-uniform in [512, 8192], M from {16, 32, 64, 128, 256}, T uniform in
    [20, 60], obstacle count uniform in [5, 60]; instance i has seed
    BASE_SEED + i.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(B):
        K = int(round(math.exp(rng.uniform(math.log(512), math.log(8192)))))
        M = int(rng.choice([16, 32, 64, 128, 256]))
        T = int(rng.integers(20, 61))
        n_obs = int(rng.integers(5, 61))
        out.append(dict(K=K, M=M, T=T, n_obs=n_obs, seed=BASE_SEED + i,
                        instance_id=i))
    return out


def random_cotangents(T, nu, K, seed):
    """Seeded cotangents for V+ (T x nu) and for the sample costs (K)."""
    rng = np.random.default_rng(seed)
    gV = rng.standard_normal((T, nu)).astype(np.float32)
    gS = (rng.standard_normal(K) * 1e-3).astype(np.float32)
    return gV, gS
