"""Shared helpers of the GPU parity tests (comparison rules, not arithmetic).

Tolerances (stage-wise protocol):
  controls U            rel 2e-6, abs 2e-6 (one float32 rounding of the
                        Box-Muller transform; clipping is exact)
  S_k, CVaR_k, S~_k     rel 1e-4 with an absolute floor 1e-4 max(1, median|S~|);
                        a sample whose FP64 band [value at r - delta,
                        value at r + delta] is not a point passes when the GPU
                        value lies in the band (plus the same tolerance): an
                        obstacle indicator may flip under float32 position drift
  CVaR on identical L   rel 1e-5 (float32 tail sums of at most 256 terms)
  V+ from the GPU's S~, U   abs 1e-5
"""

import numpy as np

RTOL = 1e-4


def abs_floor(ref):
    return 1e-4 * max(1.0, float(np.median(np.abs(ref))))


def check_banded(name, gpu, ref, lo, hi, rtol=RTOL, floor=None):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    atol = abs_floor(ref) if floor is None else floor
    tol = rtol * np.abs(ref) + atol
    close = np.abs(gpu - ref) <= tol
    banded = lo < hi
    in_band = (gpu >= lo - tol) & (gpu <= hi + tol)
    ok = close | (banded & in_band)
    bad = np.nonzero(~ok)[0]
    assert bad.size == 0, (
        f"{name}: {bad.size} of {gpu.size} outside tolerance, first {bad[:5]}: "
        f"gpu={gpu[bad[:5]]} ref={ref[bad[:5]]} band=({lo[bad[:5]]}, {hi[bad[:5]]})")
    return int(np.sum(banded & ~close))
