"""Seeded synthetic inputs for RA-MPPI updates.

This module is the only code that the FP64 oracle (``oracle/``) and the CUDA
path (``paper_2209_12842_gb300``) share.  It produces *inputs* only: problem
parameter presets, obstacle fields, initial states, warm-start controls and
cotangents.  It performs none of the method's arithmetic (no dynamics, no
costs, no risk measure, no weighting).

Every real number handed out here is rounded to float32 first, so both sides
see bit-identical inputs: the CUDA path computes on those float32 values and
the oracle promotes the very same values to float64.
"""

from .presets import (  # noqa: F401
    PRESETS,
    preset,
    model_dims,
    MODEL_KIN_BICYCLE,
    MODEL_DYN_SINGLE_TRACK,
    MODEL_LINEAR_TEST,
    NOISE_GAUSS,
    NOISE_LAPLACE_MIX,
    NOISE_UNIFORM,
    NOISE_IMPULSE,
    OBS_INDICATOR,
    OBS_SOFTPLUS,
    CVAR_RU,
    CVAR_TCE,
    RISK_VAR,
    RISK_CHANCE,
    RISK_MEAN,
    RISK_MEANVAR,
    RISK_DEV,
    RISK_SPEED,
    RISK_OBS,
    RISK_BDRY,
    RISK_LIN,
)
from .scene import (  # noqa: F401
    make_obstacles,
    obstacles_ahead,
    scene_obstacles,
    scene_initial_state,
    initial_state,
    zero_controls,
    random_controls,
    batched_instances,
    random_cotangents,
    BASE_SEED,
)
