"""Pins of the oracle's analytic adjoint (CPU only).

P11: the vector-Jacobian product of one update, for the kinematic, the
dynamic single-track and the linear models (gradients of
<gV+, V+> + <gS~, S~> w.r.t. the mean controls V and the cost weights
theta = (w_dev, w_speed, gamma, w_obs)) against central finite differences
of the oracle's own forward pass in float64.  A component is compared only
where its two one-sided differences agree (a kink of the clip or of the
CVaR order lies between them otherwise).
"""

import numpy as np
import pytest

import ra_scenes as rs


def _fd_check(orc, p, x0, V, obs, gVp, gS, h=1e-6, rtol=1e-5):
    gV, gth = orc.backward(p, x0, V, obs, gVp, gS, exact=True)
    f0 = orc.objective(p, x0, V, obs, gVp, gS)
    fd = np.full(V.shape, np.nan)
    for t in range(V.shape[0]):
        for j in range(V.shape[1]):
            Vp = V.copy(); Vp[t, j] += h
            Vm = V.copy(); Vm[t, j] -= h
            fp, fm = orc.objective(p, x0, Vp, obs, gVp, gS), orc.objective(p, x0, Vm, obs, gVp, gS)
            right, left = (fp - f0) / h, (f0 - fm) / h
            if abs(right - left) <= 1e-3 * max(1.0, abs(right)):
                fd[t, j] = (fp - fm) / (2 * h)
    ok = ~np.isnan(fd)
    assert ok.mean() > 0.8
    scale = max(1.0, np.abs(fd[ok]).max())
    np.testing.assert_allclose(gV[ok], fd[ok], rtol=rtol, atol=rtol * scale)
    th = np.array([p[n] for n in orc.THETA_NAMES], dtype=np.float64)
    for i in range(4):
        d = h * max(1.0, abs(th[i]))
        tp, tm = th.copy(), th.copy()
        tp[i] += d
        tm[i] -= d
        fdt = (orc.objective(p, x0, V, obs, gVp, gS, theta=tp) - orc.objective(p, x0, V, obs, gVp, gS, theta=tm)) / (2 * d)
        assert abs(gth[i] - fdt) <= rtol * max(1.0, abs(fdt)), (i, gth[i], fdt)
    return gV, gth


@pytest.mark.parametrize("mode,B", [(0, 1.0), (1, 1.0), (0, 2.0), (rs.RISK_VAR, 1.0), (rs.RISK_MEAN, 1.5),
                                    (rs.RISK_MEANVAR, 1.0), (rs.RISK_MEANVAR, 2.0)])
def test_p11_kinematic_softplus(orc, mode, B):
    p = rs.preset("c4_gradient", K=12, M=8, T=6, cvar_mode=mode, B=B, risk_param=0.05,
                  risk_mask=rs.RISK_OBS | rs.RISK_DEV)
    obs = rs.obstacles_ahead(1, 6, 0.15, 0.3, x_from=0.05, x_to=0.6, lateral=0.3)
    x0 = np.array([0.0, -4.0, 0.0, 1.0])
    V = rs.random_controls(0, p["T"], p["u_lo"], p["u_hi"], 3).astype(np.float64)
    gVp, gS = rs.random_cotangents(p["T"], 2, p["K"], 7)
    gV, gth = _fd_check(orc, p, x0, V, obs, gVp, gS)
    assert np.all(np.isfinite(gV)) and np.any(gth != 0)


@pytest.mark.parametrize("noise,C", [(rs.NOISE_LAPLACE_MIX, 1.5), (rs.NOISE_GAUSS, 1.3)])
def test_p11_dynamic_single_track(orc, noise, C):
    # the dynamic model's Heun sub-steps (slip angles, Pacejka forces,
    # heading), softplus obstacles, deviation and speed in the risk cost
    mp = list(rs.preset("small_dyn")["model_params"])
    mp[5] = C
    p = rs.preset("small_dyn", K=10, M=6, T=5, substeps=3, obs_mode=rs.OBS_SOFTPLUS, kappa=20.0, w_obs=5.0,
                  noise_type=noise, model_params=tuple(mp), risk_mask=rs.RISK_OBS | rs.RISK_DEV | rs.RISK_SPEED)
    obs = rs.obstacles_ahead(2, 6, 0.15, 0.3, x_from=0.05, x_to=0.6, lateral=0.3)
    x0 = np.array([0.0, -4.0, 0.05, 2.0, 0.1, 0.3])
    V = rs.random_controls(1, p["T"], p["u_lo"], p["u_hi"], 4).astype(np.float64)
    gVp, gS = rs.random_cotangents(p["T"], 2, p["K"], 9)
    gV, gth = _fd_check(orc, p, x0, V, obs, gVp, gS)
    assert np.all(np.isfinite(gV)) and np.any(gV != 0)


@pytest.mark.parametrize("name,mode", [("c4_gradient", 0), ("c4_gradient", rs.RISK_MEANVAR), ("small_dyn", 0),
                                       ("small_dyn", rs.CVAR_TCE)])
def test_p11_importance_sampled(orc, name, mode):
    # importance weights depend on the noise only, so the risk measure of the
    # weighted costs differentiates like the plain one with weights in it
    if name == "small_dyn":
        p = rs.preset(name, K=8, M=12, T=4, substeps=2, obs_mode=rs.OBS_SOFTPLUS, kappa=20.0, w_obs=5.0,
                      risk_mask=rs.RISK_OBS | rs.RISK_DEV | rs.RISK_SPEED, mix_p=0.3)
        x0 = np.array([0.0, -4.0, 0.05, 2.0, 0.1, 0.3])
    else:
        p = rs.preset(name, K=10, M=12, T=5, risk_mask=rs.RISK_OBS | rs.RISK_DEV)
        x0 = np.array([0.0, -4.0, 0.0, 1.0])
    p = dict(p, cvar_mode=mode, B=1.5, risk_param=0.05, alpha=0.8, is_scale=1.4, is_frac=0.5)
    obs = rs.obstacles_ahead(3, 6, 0.15, 0.3, x_from=0.05, x_to=0.6, lateral=0.3)
    V = rs.random_controls(p["model"], p["T"], p["u_lo"], p["u_hi"], 6).astype(np.float64)
    gVp, gS = rs.random_cotangents(p["T"], 2, p["K"], 12)
    gV, gth = _fd_check(orc, p, x0, V, obs, gVp, gS)
    assert np.all(np.isfinite(gV)) and np.any(gV != 0)
    # and it differs from the unweighted gradient
    gV0, _ = orc.backward(dict(p, is_frac=0.0), x0, V, obs, gVp, gS, exact=True)
    assert np.max(np.abs(gV - gV0)) > 1e-6 * max(1.0, np.max(np.abs(gV0)))


def test_p11_all_terms_and_zero_mean_samples(orc):
    p = rs.preset("c4_gradient", K=10, M=6, T=5, eta=0.3, w_bdry=2.0, c4=0.6, c5=2.0, A=2.0, C_u=10.0,
                  risk_mask=rs.RISK_OBS | rs.RISK_DEV | rs.RISK_SPEED | rs.RISK_BDRY)
    obs = rs.obstacles_ahead(2, 5, 0.15, 0.3, x_from=0.05, x_to=0.6, lateral=0.3)
    x0 = np.array([0.0, -4.6, 0.1, 1.5])
    V = rs.random_controls(0, p["T"], p["u_lo"], p["u_hi"], 4).astype(np.float64)
    gVp, gS = rs.random_cotangents(p["T"], 2, p["K"], 8)
    _fd_check(orc, p, x0, V, obs, gVp, gS)


def test_p11_linear_closed_form(orc):
    """Linear system with sigma_u = 0 and no noise: every sample equals V, so
    V+ = V and the update's VJP w.r.t. V is the identity on gV+ plus the
    cost sensitivity through the (equal) weights, which cancels."""
    p = rs.preset("linear_test", K=4, M=4, T=5, w_scale=(0, 0, 0, 0))
    V = np.linspace(-0.3, 0.4, 5).reshape(5, 1)
    gVp = np.arange(1, 6, dtype=np.float64).reshape(5, 1)
    gV, gth = orc.backward(p, np.array([0.2]), V, np.zeros((0, 3)), gVp, None, exact=True)
    np.testing.assert_allclose(gV, gVp, rtol=1e-12)


def test_too_many_substeps_is_reported(orc):
    # the reverse sweep keeps at most 64 sub-step states per control step
    p = rs.preset("small_dyn", K=2, M=2, T=2, substeps=65)
    with pytest.raises(RuntimeError):
        orc.backward(p, rs.initial_state(1), rs.zero_controls(1, 2), np.zeros((0, 3)), np.ones((2, 2)))
