"""GB300 (sm_103a) implementation of the Risk-Aware MPPI control update.

The update (sampling, nominal and disturbed rollouts, CVaR, violation cost,
softmin update) runs in hand-written CUDA kernels behind the C ABI of
``include/ra_mppi.h`` (``libramppi.so``).  ``binding`` exposes those C
functions under their own names; ``RaMppi`` wraps one handle with torch
device buffers and streams.
"""

from . import binding  # noqa: F401
from .binding import RaMppiError, lib  # noqa: F401


def __getattr__(name):
    # the controller imports torch; keep `import paper_2209_12842_gb300` light
    if name in ("RaMppi", "RaMppiBatch", "RaMppiUpdate"):
        from . import controller

        return getattr(controller, name)
    raise AttributeError(name)
