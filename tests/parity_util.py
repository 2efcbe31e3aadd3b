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
  end-to-end V+ (the GPU's V+ against the oracle's own V+, when the oracle
                        ran every sample): reported with the softmin's
                        amplification bound and checked against it.  With
                        D = max_k |S~_gpu - S~_oracle| every weight ratio
                        w'_k / w_k lies in [exp(-2D/lambda), exp(2D/lambda)]
                        (Eqs. 5, 17), so |dV+| <= (exp(2D/lambda) - 1)
                        max_k ||U_k - V+||_inf + max |dU| + 1e-5 (rounding of
                        the update); to first order 2 D / lambda max_k ||U_k -
                        V+||_inf, the form the scope gives.
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


def vplus_bound(p, g, ref):
    """(deviation, bound, first-order bound, D) of the GPU's end-to-end V+
    against the oracle's own V+, from the oracle's per-sample results over
    every sample (ref["ks"] must be 0..K-1)."""
    K = int(p["K"])
    assert len(ref["ks"]) == K and np.array_equal(ref["ks"], np.arange(K))
    lam = float(np.float32(p["lam"]))
    Vo, _ = oracle.update(ref["S_tilde"], ref["U"], lam)
    dev = float(np.max(np.abs(g["V_plus"].astype(np.float64) - Vo)))
    sg = g["S_tilde"].astype(np.float64)
    so = np.asarray(ref["S_tilde"], np.float64)
    both = np.isfinite(sg) & np.isfinite(so)
    assert np.array_equal(np.isfinite(sg), np.isfinite(so)), "finite S~ differ between GPU and oracle"
    D = float(np.max(np.abs(sg[both] - so[both]))) if both.any() else 0.0
    spread = float(np.max(np.abs(np.asarray(ref["U"], np.float64) - Vo[None]))) if K else 0.0
    dU = float(np.max(np.abs(g["U"].astype(np.float64) - ref["U"])))
    with np.errstate(over="ignore"):
        bound = float(np.expm1(2.0 * D / lam)) * spread + dU + 1e-5
    first = 2.0 * D / lam * spread
    return dev, bound, first, D


def check_vplus_bound(name, p, g, ref):
    dev, bound, first, D = vplus_bound(p, g, ref)
    print(f"{name}: end-to-end |V+_gpu - V+_oracle| = {dev:.3e}, bound {bound:.3e} "
          f"(first order 2 D/lambda max||U - V+|| = {first:.3e}, D = max|dS~| = {D:.3e}, "
          f"ratio {dev / bound if bound > 0 else 0.0:.3f})")
    assert dev <= bound, (name, dev, bound)
    return dev, bound


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
        # 5. end to end, when the oracle ran every sample
        if len(ks) == int(p["K"]) and np.array_equal(ks, np.arange(int(p["K"]))):
            check_vplus_bound(f"K={p['K']} M={p['M']} T={p['T']}", p, g, ref)
    return nS, nC, nT
