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

import oracle

RTOL = 1e-4


def importance_on(p):
    """Whether a preset draws importance-sampled rollouts (at least one)."""
    s = float(np.float32(p.get("is_scale", 1.0)))
    f = float(np.float32(p.get("is_frac", 0.0)))
    return s != 1.0 and f > 0.0 and int(np.floor(f * int(p["M"]))) > 0


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


def compare(p, g, ref, check_update=True):
    ks = ref["ks"]
    # 1. sampled controls
    np.testing.assert_allclose(g["U"][ks], ref["U"], rtol=2e-6, atol=2e-6)
    # 2. per-sample stage
    nS = check_banded("S", g["S"][ks], ref["S"], ref["S_lo"], ref["S_hi"])
    nC = check_banded("CVaR", g["cvar"][ks], ref["cvar"], ref["cvar_lo"], ref["cvar_hi"],
                      floor=1e-4 * max(1.0, float(np.median(np.abs(ref["S_tilde"])))))
    nT = check_banded("S_tilde", g["S_tilde"][ks], ref["S_tilde"], ref["St_lo"], ref["St_hi"])
    # 3. CVaR on the GPU's own risk costs (and its own importance weights,
    # which must match the oracle's within the float32 error of their log
    # density ratio: about 1e-6 per draw from the Box-Muller transcendentals,
    # bounded here by 4e-6 per draw)
    if g["L"] is not None:
        alpha = float(np.float32(p["alpha"]))
        Bs = float(np.float32(p["B"]))
        weighted = importance_on(p)
        for i, k in enumerate(ks):
            w = None
            if weighted:
                w = g["W"][k].astype(np.float64)
                w_ref = oracle.is_weights(p, k)
                n_draws = int(p["T"]) * int(np.count_nonzero(np.asarray(p["w_scale"], np.float32)))
                np.testing.assert_allclose(np.log(w), np.log(w_ref), rtol=0, atol=4e-6 * n_draws,
                                           err_msg=f"importance weights of sample {k}")
            want = oracle.risk_w(g["L"][k].astype(np.float64), w, alpha, Bs, p["cvar_mode"],
                                 float(np.float32(p.get("risk_param", 0.0))))
            assert abs(g["cvar"][k] - want) <= 1e-5 * max(1.0, abs(want)), (k, g["cvar"][k], want)
    # 4. update stage on the GPU's S~ and U
    if check_update:
        Vo, _ = oracle.update(g["S_tilde"].astype(np.float64), g["U"].astype(np.float64),
                              float(np.float32(p["lam"])))
        np.testing.assert_allclose(g["V_plus"], Vo, atol=1e-5, rtol=0)
    return nS, nC, nT
