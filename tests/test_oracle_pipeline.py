"""Pins of the oracle's whole update (CPU only).

P3   zero process noise: every disturbed rollout equals the nominal one, so
     CVaR_k = L_k(nominal) for any alpha and either CVaR form; with l = q,
     gamma = 0 and phi = 0 that is S_k itself
P4   softmin weights: sum to 1, shift invariance, lambda -> 0 selects the
     argmin (ties split), lambda -> inf averages
P5   K = 1 gives V+ = U_0; V+ stays in the control box; equal costs average
P12  hand-worked K = M = T = 2 update (tests/golden/tiny_linear.json)
     plus zero-mean samples (Alg. 1), clipping, band bounds and the
     receding-horizon loop on a small case
"""

import json
import os

import numpy as np
import pytest

import ra_scenes as rs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _scene(p, seed=1):
    return rs.obstacles_ahead(seed, 8, 0.15, 0.3)


def test_p3_zero_process_noise(orc):
    for name in ("small_kin", "small_dyn"):
        p = rs.preset(name, w_scale=(0, 0, 0, 0), gamma=0.0,
                      risk_mask=rs.RISK_DEV | rs.RISK_SPEED | rs.RISK_OBS | rs.RISK_BDRY)
        x0 = rs.initial_state(p["model"])
        V = rs.random_controls(p["model"], p["T"], p["u_lo"], p["u_hi"], 3)
        for alpha in (0.5, 0.9, 0.99):
            for mode in (rs.CVAR_RU, rs.CVAR_TCE):
                p2 = dict(p, alpha=alpha, cvar_mode=mode)
                out = orc.samples(p2, x0, V, _scene(p), want_L=True)
                L = out["L"]
                assert np.all(L == L[:, :1])
                np.testing.assert_allclose(out["cvar"], L[:, 0], rtol=1e-12)
                np.testing.assert_allclose(out["S"], L[:, 0], rtol=1e-12)


def test_p4_weights(orc):
    rng = np.random.default_rng(0)
    K, T, nu = 50, 7, 2
    S = rng.normal(size=K) * 5
    U = rng.uniform(-1, 1, size=(K, T, nu))
    Vp, w = orc.update(S, U, 0.7)
    assert abs(w.sum() - 1) < 1e-15
    np.testing.assert_allclose(Vp, np.einsum("k,ktj->tj", w, U), atol=1e-15)
    Vp2, _ = orc.update(S + 1234.5, U, 0.7)
    np.testing.assert_allclose(Vp2, Vp, atol=1e-13)
    # lambda -> 0 selects the argmin; ties split the weight equally
    S2 = S.copy()
    S2[7] = S.min() - 10
    Vp3, w3 = orc.update(S2, U, 1e-6)
    np.testing.assert_allclose(Vp3, U[7], atol=1e-15)
    S2[9] = S2[7]
    Vp4, w4 = orc.update(S2, U, 1e-6)
    np.testing.assert_allclose(Vp4, 0.5 * (U[7] + U[9]), atol=1e-15)
    # lambda -> inf averages
    Vp5, _ = orc.update(S, U, 1e12)
    np.testing.assert_allclose(Vp5, U.mean(0), atol=1e-9)
    # non-finite costs get zero weight
    S3 = S.copy()
    S3[3] = np.inf
    S3[4] = np.nan
    _, w5 = orc.update(S3, U, 0.7)
    assert w5[3] == 0 and w5[4] == 0 and abs(w5.sum() - 1) < 1e-15


def test_p5_update_edges(orc):
    p = rs.preset("small_kin", K=1)
    x0 = rs.initial_state(p["model"])
    V = rs.random_controls(p["model"], p["T"], p["u_lo"], p["u_hi"], 4)
    out = orc.step(p, x0, V, _scene(p))
    np.testing.assert_allclose(out["V_plus"], out["U"][0], atol=1e-15)
    p = rs.preset("small_kin", sigma_u=(3.0, 10.0))
    out = orc.step(p, x0, V, _scene(p))
    lo = np.float32(p["u_lo"]).astype(np.float64)
    hi = np.float32(p["u_hi"]).astype(np.float64)
    assert np.all(out["U"] >= lo) and np.all(out["U"] <= hi)
    assert np.any(out["U"] == lo) and np.any(out["U"] == hi)
    assert np.all(out["V_plus"] >= lo - 1e-15) and np.all(out["V_plus"] <= hi + 1e-15)
    Vp, _ = orc.update(np.full(out["U"].shape[0], 3.0), out["U"], 1.0)
    np.testing.assert_allclose(Vp, out["U"].mean(0), atol=1e-14)


def test_p12_hand_worked(orc):
    g = json.load(open(os.path.join(GOLDEN, "tiny_linear.json")))
    s = g["setup"]
    p = rs.preset("linear_test", K=2, M=2, T=2, w_scale=(0, 0, 0, 0), eta=s["eta"],
                  alpha=s["alpha"], A=s["A"], C_u=s["C_u"], lam=s["lambda"], c_lin=s["c_lin"])
    out = orc.step(p, np.array([s["x0"]], np.float32), np.array(s["V"], np.float32),
                   np.zeros((0, 3), np.float32))
    e = g["expect"]
    np.testing.assert_allclose(out["U"], e["U"], rtol=1e-15)
    np.testing.assert_allclose(out["S"], e["S"], rtol=1e-15)
    np.testing.assert_allclose(out["cvar"], e["cvar"], rtol=1e-15)
    np.testing.assert_allclose(out["S_tilde"], e["S_tilde"], rtol=1e-15)
    np.testing.assert_allclose(out["weights"], e["weights"], rtol=1e-13)
    np.testing.assert_allclose(out["V_plus"], e["V_plus"], rtol=1e-13)


def test_zero_mean_samples(orc):
    p = rs.preset("small_kin", eta=0.25)
    prob = orc.make_problem(p)
    nw = orc.n_warm(prob)
    assert nw == int(np.ceil(0.75 * p["K"]))
    V = rs.random_controls(p["model"], p["T"], p["u_lo"], p["u_hi"], 5)
    out = orc.samples(p, rs.initial_state(0), V, _scene(p))
    for k in (0, nw - 1, nw, p["K"] - 1):
        eps = np.array([orc.control_noise(prob, k, t) for t in range(p["T"])])
        base = V.astype(np.float64) if k < nw else 0.0
        want = np.clip(base + eps, np.float32(p["u_lo"]), np.float32(p["u_hi"]))
        np.testing.assert_allclose(out["U"][k], want, rtol=1e-15)


def test_band_bounds_bracket(orc):
    p = rs.preset("c1_plain")
    out = orc.samples(p, rs.initial_state(0), rs.zero_controls(0, p["T"]), _scene(p), band_delta=1e-3)
    assert np.all(out["cvar_lo"] <= out["cvar"]) and np.all(out["cvar"] <= out["cvar_hi"])
    assert np.all(out["S_lo"] <= out["S"]) and np.all(out["S"] <= out["S_hi"])
    assert np.all(out["St_lo"] <= out["S_tilde"]) and np.all(out["S_tilde"] <= out["St_hi"])
    assert np.any(out["cvar_lo"] < out["cvar_hi"])


def test_cvar_threshold_and_gain(orc):
    p = rs.preset("c1_plain", K=32)
    base = orc.samples(p, rs.initial_state(0), rs.zero_controls(0, p["T"]), _scene(p))
    hi = orc.samples(dict(p, A=3.0, C_u=500.0), rs.initial_state(0), rs.zero_controls(0, p["T"]), _scene(p))
    cv = base["cvar"]
    want = base["S"] + np.where(cv > float(np.float32(500.0)), 3.0 * cv, 0.0)
    np.testing.assert_allclose(hi["S_tilde"], want, rtol=1e-15)
    assert np.any(cv > 500) and np.any(cv <= 500)


def test_closed_loop_small(orc):
    p = rs.preset("small_kin", K=64, M=16, T=10)
    obs = rs.make_obstacles(p["seed"], p["n_obs"], *p["obs_r"])
    xs, Vs, hits = orc.closed_loop(p, rs.initial_state(0), rs.zero_controls(0, p["T"]), obs, 12)
    assert xs.shape == (13, 4) and Vs.shape == (12, p["T"], 2)
    # the speed-tracking cost (target 4 m/s) accelerates the plant from rest
    assert xs[-1, 3] > 1.0 and xs[-1, 0] > 0.05
    # replaying update 3 from its recorded state reproduces the recorded V+
    V3 = np.concatenate([Vs[2][1:], Vs[2][-1:]], 0)
    out = orc.step(p, xs[3].astype(np.float32), V3.astype(np.float32), obs, iteration=3)
    np.testing.assert_allclose(out["V_plus"], Vs[3], rtol=1e-6, atol=1e-7)
