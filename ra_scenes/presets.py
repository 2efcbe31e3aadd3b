"""Problem presets for the five RA-MPPI workloads and the small parity cases.

Values are the workload definitions (vehicle, sampling, noise, scene, risk
parameters).  Where a workload leaves a quantity open, the value here is the
reading recorded in the design notes (weights of the cost terms, tyre
geometry, integrator sub-steps, noise layout).

Letters: K control samples, M disturbed (process-noise) rollouts per sample,
T horizon steps.  The paper itself writes M, N, K for these three (Sec. III,
Algorithm 1); this code uses K, M, T throughout.
"""

import copy

MODEL_KIN_BICYCLE = 0
MODEL_DYN_SINGLE_TRACK = 1
MODEL_LINEAR_TEST = 2

NOISE_GAUSS = 0
NOISE_LAPLACE_MIX = 1
NOISE_UNIFORM = 2
NOISE_IMPULSE = 3

OBS_INDICATOR = 0
OBS_SOFTPLUS = 1

CVAR_RU = 0
CVAR_TCE = 1
RISK_VAR = 2
RISK_CHANCE = 3
RISK_MEAN = 4
RISK_MEANVAR = 5

# bits of risk_mask: which running-cost terms make up the risk cost l(x)
RISK_DEV = 1
RISK_SPEED = 2
RISK_OBS = 4
RISK_BDRY = 8
RISK_LIN = 16


def model_dims(model):
    """(nx, nu, number of process-noise slots) of a model id."""
    if model == MODEL_KIN_BICYCLE:
        return 4, 2, 4
    if model == MODEL_DYN_SINGLE_TRACK:
        return 6, 2, 3
    if model == MODEL_LINEAR_TEST:
        return 1, 1, 1
    raise ValueError(f"unknown model {model}")


_COMMON = dict(
    substeps=1,
    sigma_u=(0.3, 1.0),
    u_lo=(-0.4, -3.0),
    u_hi=(0.4, 3.0),
    mix_p=0.0,
    mix_scale=1.0,
    # running cost q: deviation, speed tracking, obstacles, boundary, linear
    w_dev=1.0,
    w_speed=1.0,
    v_target=4.0,
    gamma=1.0,          # control-cost weight, gamma in [0, lambda] (Eq. 4)
    w_obs=1000.0,
    w_bdry=0.0,
    c4=0.0,
    c5=0.0,
    c_lin=0.0,
    obs_mode=OBS_INDICATOR,
    kappa=20.0,
    risk_mask=RISK_OBS,
    track_straight=10.0,
    track_radius=4.0,
    track_half_width=1.0,
    lam=1.0,
    alpha=0.9,
    A=1.0,
    B=1.0,
    C_u=0.0,
    eta=0.0,
    cvar_mode=CVAR_RU,
    risk_param=0.0,
    # importance-sampled rollouts: the last floor(is_frac M) rollouts draw
    # their process noise at is_scale times its size (off: 1.0 / 0.0)
    is_scale=1.0,
    is_frac=0.0,
    seed=12842,
    instance_id=0,
    n_obs=10,
    obs_r=(0.3, 0.3),
)

_KIN = dict(model=MODEL_KIN_BICYCLE, dt=0.05,
            # [0] wheelbase (m)
            model_params=(0.33, 0, 0, 0, 0, 0, 0, 0),
            noise_type=NOISE_GAUSS,
            # process-noise std of (x, y, psi, v)
            w_scale=(0.05, 0.05, 0.02, 0.1))

_DYN = dict(model=MODEL_DYN_SINGLE_TRACK, dt=0.02, substeps=6,
            # m, Iz, lf, lr, Pacejka B, C, D, v_x floor of the slip angles
            model_params=(2.5, 0.02, 0.165, 0.165, 10.0, 1.5, 1.0, 1.0),
            noise_type=NOISE_LAPLACE_MIX,
            # Laplace scale on (vx, vy, r); mixed with a Gaussian of std
            # mix_scale * scale with probability mix_p
            w_scale=(0.02, 0.02, 0.02, 0.0),
            mix_p=0.1, mix_scale=5.0)

PRESETS = {
    # plain single update, kinematic bicycle
    "c1_plain": dict(_COMMON, **_KIN, K=256, M=32, T=20),
    # paper-scale closed loop, dynamic single-track, heavy-tailed noise
    "c2_closed_loop": dict(_COMMON, **_DYN, K=4096, M=128, T=40, n_obs=50,
                           obs_r=(0.2, 0.5)),
    # one instance of the batched workload (the batch varies K, M, T, scene)
    "c3_instance": dict(_COMMON, **_KIN, K=1024, M=64, T=40, n_obs=30),
    # differentiation workload: softplus obstacle barrier
    "c4_gradient": dict(_COMMON, **_KIN, K=1024, M=64, T=30,
                        obs_mode=OBS_SOFTPLUS, kappa=20.0),
    # stress / roofline: dynamic single-track, 200 obstacles
    "c5_stress": dict(_COMMON, **_DYN, K=65536, M=256, T=50, n_obs=200,
                      obs_r=(0.2, 0.5), alpha=0.95),
    # small parity cases (several tiles and a ragged tail)
    "small_kin": dict(_COMMON, **_KIN, K=77, M=32, T=13, n_obs=10),
    "small_dyn": dict(_COMMON, **_DYN, K=45, M=64, T=11, n_obs=20,
                      obs_r=(0.2, 0.5)),
    # the paper's simulation setting (Sec. V-A): K = 1024 samples, M = 300
    # disturbed rollouts, T = 30, lambda = 0.35, eta = 0.2, A = 10, running
    # cost 2 boundary + 1 obstacle + 0.1 deviation^2, terminal progress
    # cost 0.6 - 2 s, risk cost l = q; alpha = 0.7, C_u = 0.6 (the loosened
    # setting of Sec. V-B); a stadium of the paper's width (0.6 m),
    # corner radius (0.3 m) and centreline length (10.9 m); 10 obstacles of
    # radius 0.1 m; Gaussian disturbance 0.2 on the velocity states
    "paper_sim": dict(_COMMON, **dict(_DYN, noise_type=NOISE_GAUSS, w_scale=(0.2, 0.2, 0.2, 0.0), mix_p=0.0),
                      K=1024, M=300, T=30, w_dev=0.1, w_speed=0.0, w_obs=1.0, w_bdry=2.0, c4=0.6, c5=2.0,
                      gamma=0.35, lam=0.35, eta=0.2, A=10.0, alpha=0.7, C_u=0.6,
                      risk_mask=RISK_DEV | RISK_OBS | RISK_BDRY,
                      track_straight=4.5075, track_radius=0.3, track_half_width=0.3, n_obs=10,
                      obs_r=(0.1, 0.1)),
    # linear-Gaussian test system x+ = x + dt*u + w with cost c_lin * x
    "linear_test": dict(_COMMON, model=MODEL_LINEAR_TEST, dt=1.0,
                        model_params=(0,) * 8, noise_type=NOISE_GAUSS,
                        w_scale=(0.5, 0, 0, 0), sigma_u=(0.0, 0.0),
                        u_lo=(-1e30, -1e30), u_hi=(1e30, 1e30),
                        w_dev=0.0, w_speed=0.0, w_obs=0.0, gamma=0.0,
                        c_lin=1.0, risk_mask=RISK_LIN, C_u=-1e30,
                        K=16, M=256, T=10, n_obs=0),
}


def preset(name, **overrides):
    """A deep copy of a preset with keyword overrides applied."""
    if name not in PRESETS:
        raise KeyError(f"unknown preset {name!r}; have {sorted(PRESETS)}")
    p = copy.deepcopy(PRESETS[name])
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(f"unknown problem field {k!r}")
        p[k] = v
    return p
