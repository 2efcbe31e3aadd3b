"""GPU adjoint (ra_mppi_backward, RaMppiUpdate) against the oracle's analytic
adjoint, which the CPU tests pin to central finite differences.

Tolerance: relative 1e-3 in the 2-norm of each block (gV, gtheta), and per
component with a floor of 1e-3 of the block's largest component.
"""

import numpy as np
import pytest

import oracle
import ra_scenes as rs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_12842_gb300 import build as b

    b.build()


def _close(name, got, want, rtol=1e-3):
    got, want = np.asarray(got, np.float64).ravel(), np.asarray(want, np.float64).ravel()
    nrm = np.linalg.norm(want)
    assert np.linalg.norm(got - want) <= rtol * max(nrm, 1e-12), (name, got, want)
    floor = rtol * np.abs(want).max()
    bad = np.abs(got - want) > rtol * np.abs(want) + floor
    assert not bad.any(), (name, np.nonzero(bad), got[bad], want[bad])


def _run(p, obs, x0, V, gVp, gS, iteration=0):
    from paper_2209_12842_gb300 import RaMppi

    ctl = RaMppi(p, obs, differentiable=True)
    ctl.iteration = iteration
    ctl.step(torch.from_numpy(x0).cuda(), torch.from_numpy(V).cuda())
    gV, gth = ctl.backward(torch.from_numpy(gVp).cuda(), torch.from_numpy(gS).cuda() if gS is not None else None)
    torch.cuda.synchronize()
    out = gV.cpu().numpy(), gth.cpu().numpy()
    assert ctl.status() == 0
    ctl.close()
    return out


@pytest.mark.parametrize("case", ["plain", "tce", "scaled_eta", "all_terms"])
def test_adjoint_matches_oracle_small(case):
    ov = dict(K=96, M=32, T=12)
    if case == "tce":
        ov.update(cvar_mode=rs.CVAR_TCE)
    elif case == "scaled_eta":
        ov.update(B=2.0, eta=0.25, A=3.0, C_u=5.0)
    elif case == "all_terms":
        ov.update(risk_mask=rs.RISK_OBS | rs.RISK_DEV | rs.RISK_SPEED | rs.RISK_BDRY, w_bdry=2.0, c4=0.6, c5=2.0)
    p = rs.preset("c4_gradient", **ov)
    obs = rs.obstacles_ahead(1, 8, 0.15, 0.3, x_from=0.05, x_to=0.9, lateral=0.4)
    x0 = np.array([0.0, -4.0, 0.0, 1.0], np.float32)
    V = rs.random_controls(0, p["T"], p["u_lo"], p["u_hi"], 3)
    gVp, gS = rs.random_cotangents(p["T"], 2, p["K"], 7)
    gV, gth = _run(p, obs, x0, V, gVp, gS)
    rV, rth = oracle.backward(p, x0, V, obs, gVp, gS)
    _close("gV", gV, rV)
    _close("gtheta", gth, rth)


@pytest.mark.parametrize("M,alpha", [(64, 0.8), (128, 0.9), (32, 0.5)])
def test_adjoint_tail_lane_groups(M, alpha):
    """The disturbed reverse sweep gives each rollout of a short CVaR tail a
    group of lanes: four lanes for at most 8 rollouts with a nonzero
    cotangent, two for 9 to 16, one above.  Without ties at VaR, M = 64 at
    alpha = 0.8 and M = 128 at alpha = 0.9 leave 13 tail rollouts (two lanes
    each) and M = 32 at alpha = 0.5 leaves 16 or 17; each against the
    oracle's adjoint, and two passes of the backward give the same bits."""
    from paper_2209_12842_gb300 import RaMppi

    p = rs.preset("c4_gradient", K=96, M=M, T=12, alpha=alpha)
    obs = rs.obstacles_ahead(1, 8, 0.15, 0.3, x_from=0.05, x_to=0.9, lateral=0.4)
    x0 = np.array([0.0, -4.0, 0.0, 1.0], np.float32)
    V = rs.random_controls(0, p["T"], p["u_lo"], p["u_hi"], 3)
    gVp, gS = rs.random_cotangents(p["T"], 2, p["K"], 7)
    ctl = RaMppi(p, obs, differentiable=True)
    ctl.iteration = 0
    ctl.step(torch.from_numpy(x0).cuda(), torch.from_numpy(V).cuda())
    gVp_t, gS_t = torch.from_numpy(gVp).cuda(), torch.from_numpy(gS).cuda()
    gV1, gth1 = ctl.backward(gVp_t, gS_t)
    gV2, gth2 = ctl.backward(gVp_t, gS_t)
    torch.cuda.synchronize()
    assert ctl.status() == 0
    ctl.close()
    assert torch.equal(gV1, gV2) and torch.equal(gth1, gth2)
    rV, rth = oracle.backward(p, x0, V, obs, gVp, gS)
    _close("gV", gV1.cpu().numpy(), rV)
    _close("gtheta", gth1.cpu().numpy(), rth)


@pytest.mark.parametrize("n_obs", [0, 1, 3, 4, 5, 7, 13])
def test_adjoint_obstacle_counts(n_obs):
    # the softplus gradient's obstacle loop is unrolled four times: counts
    # below, at and between multiples of four, and none; the obstacles lie on
    # and beside the path, so states inside (z > 0) and outside both occur
    p = rs.preset("c4_gradient", K=64, M=32, T=12)
    obs = (rs.obstacles_ahead(3, n_obs, 0.15, 0.3, x_from=0.05, x_to=0.9, lateral=0.4) if n_obs
           else np.zeros((0, 3), np.float32))
    p["n_obs"] = max(n_obs, 1)
    x0 = np.array([0.0, -4.0, 0.0, 1.0], np.float32)
    V = rs.random_controls(0, p["T"], p["u_lo"], p["u_hi"], 3)
    gVp, gS = rs.random_cotangents(p["T"], 2, p["K"], 7)
    gV, gth = _run(p, obs, x0, V, gVp, gS)
    rV, rth = oracle.backward(p, x0, V, obs, gVp, gS)
    _close("gV", gV, rV)
    _close("gtheta", gth, rth)


def test_adjoint_config4_full_size():
    p = rs.preset("c4_gradient")
    obs = rs.make_obstacles(p["seed"], p["n_obs"], *p["obs_r"])
    obs = np.concatenate([obs, rs.obstacles_ahead(2, 4, 0.2, 0.3, x_from=0.2, x_to=1.5)])
    p["n_obs"] = len(obs)
    x0 = np.array([0.0, -4.0, 0.0, 1.5], np.float32)
    V = rs.random_controls(0, p["T"], p["u_lo"], p["u_hi"], 5)
    gVp, gS = rs.random_cotangents(p["T"], 2, p["K"], 11)
    gV, gth = _run(p, obs, x0, V, gVp, gS)
    rV, rth = oracle.backward(p, x0, V, obs, gVp, gS)
    _close("gV", gV, rV)
    _close("gtheta", gth, rth)


def test_autograd_function_matches_backward():
    from paper_2209_12842_gb300 import RaMppi, RaMppiUpdate

    p = rs.preset("c4_gradient", K=128, M=32, T=10)
    obs = rs.obstacles_ahead(1, 8, 0.15, 0.3, x_from=0.05, x_to=0.9, lateral=0.4)
    x0 = torch.tensor([0.0, -4.0, 0.0, 1.0], device="cuda")
    V = torch.from_numpy(rs.random_controls(0, p["T"], p["u_lo"], p["u_hi"], 3)).cuda().requires_grad_(True)
    theta = torch.tensor([p["w_dev"], p["w_speed"], p["gamma"], p["w_obs"]], device="cuda", requires_grad=True)
    ctl = RaMppi(p, obs, differentiable=True)
    gVp, gS = rs.random_cotangents(p["T"], 2, p["K"], 7)
    gVp_t, gS_t = torch.from_numpy(gVp).cuda(), torch.from_numpy(gS).cuda()
    V_plus, S_tilde = RaMppiUpdate.apply(V, theta, ctl, x0)
    loss = (V_plus * gVp_t).sum() + (S_tilde * gS_t).sum()
    dV, dth = torch.autograd.grad(loss, (V, theta))
    rV, rth = oracle.backward(p, x0.cpu().numpy(), V.detach().cpu().numpy(), obs, gVp, gS)
    _close("gV", dV.cpu().numpy(), rV)
    _close("gtheta", dth.cpu().numpy(), rth)
    # gradient refinement of the warm start moves the objective downhill
    ctl.close()


@pytest.mark.parametrize("case", ["mixture_C15", "gauss_C13", "all_terms"])
def test_adjoint_dynamic_model(case):
    # reverse sweeps through the Heun sub-steps of the dynamic single-track model
    mp = list(rs.preset("small_dyn")["model_params"])
    ov = dict(K=96, M=32, T=10, obs_mode=rs.OBS_SOFTPLUS, kappa=20.0, w_obs=5.0,
              risk_mask=rs.RISK_OBS | rs.RISK_DEV | rs.RISK_SPEED)
    if case == "gauss_C13":
        mp[5] = 1.3
        ov.update(noise_type=rs.NOISE_GAUSS, w_scale=(0.05, 0.05, 0.05, 0.0))
    elif case == "all_terms":
        ov.update(risk_mask=rs.RISK_OBS | rs.RISK_DEV | rs.RISK_SPEED | rs.RISK_BDRY, w_bdry=2.0, c4=0.6, c5=2.0,
                  B=1.5, eta=0.2)
    p = rs.preset("small_dyn", model_params=tuple(mp), **ov)
    obs = rs.obstacles_ahead(1, 8, 0.15, 0.3, x_from=0.1, x_to=1.2, lateral=0.4)
    x0 = np.array([0.0, -4.0, 0.05, 2.0, 0.1, 0.3], np.float32)
    V = rs.random_controls(1, p["T"], p["u_lo"], p["u_hi"], 3)
    gVp, gS = rs.random_cotangents(p["T"], 2, p["K"], 7)
    gV, gth = _run(p, obs, x0, V, gVp, gS)
    rV, rth = oracle.backward(p, x0, V, obs, gVp, gS)
    _close("gV", gV, rV)
    _close("gtheta", gth, rth)


@pytest.mark.parametrize("case", ["kin_ru", "kin_meanvar", "dyn_ru", "dyn_tce"])
def test_adjoint_importance_sampled(case):
    # importance weights depend on the noise only: the adjoint of the weighted
    # risk measure, through the scaled noise of the proposal rollouts
    if case.startswith("kin"):
        p = rs.preset("c4_gradient", K=96, M=40, T=12, is_scale=1.4, is_frac=0.5, alpha=0.8, B=1.5,
                      cvar_mode=rs.CVAR_RU if case == "kin_ru" else rs.RISK_MEANVAR, risk_param=0.05)
        x0 = np.array([0.0, -4.0, 0.0, 1.0], np.float32)
        obs = rs.obstacles_ahead(1, 8, 0.15, 0.3, x_from=0.05, x_to=0.9, lateral=0.4)
    else:
        p = rs.preset("small_dyn", K=64, M=40, T=8, obs_mode=rs.OBS_SOFTPLUS, kappa=20.0, w_obs=5.0,
                      risk_mask=rs.RISK_OBS | rs.RISK_DEV | rs.RISK_SPEED, is_scale=1.3, is_frac=0.5, alpha=0.8,
                      cvar_mode=rs.CVAR_RU if case == "dyn_ru" else rs.CVAR_TCE, mix_p=0.3)
        x0 = np.array([0.0, -4.0, 0.05, 2.0, 0.1, 0.3], np.float32)
        obs = rs.obstacles_ahead(1, 8, 0.15, 0.3, x_from=0.1, x_to=1.2, lateral=0.4)
    V = rs.random_controls(p["model"], p["T"], p["u_lo"], p["u_hi"], 3)
    gVp, gS = rs.random_cotangents(p["T"], 2, p["K"], 7)
    gV, gth = _run(p, obs, x0, V, gVp, gS)
    rV, rth = oracle.backward(p, x0, V, obs, gVp, gS)
    _close("gV", gV, rV)
    _close("gtheta", gth, rth)


@pytest.mark.parametrize("K", [1, 33, 1024, 9000])
def test_adjoint_is_deterministic(K):
    # the prep and column reductions sum in an order fixed by K: repeated
    # backward passes give the same bits (one sample, ragged and many slices)
    p = rs.preset("c4_gradient", K=K, M=32, T=12)
    obs = rs.obstacles_ahead(1, 8, 0.15, 0.3, x_from=0.05, x_to=0.9, lateral=0.4)
    from paper_2209_12842_gb300 import RaMppi

    ctl = RaMppi(p, obs, differentiable=True)
    ctl.step(torch.tensor([0.0, -4.0, 0.0, 1.0], device="cuda"),
             torch.from_numpy(rs.random_controls(0, p["T"], p["u_lo"], p["u_hi"], 3)).cuda())
    gVp, gS = rs.random_cotangents(p["T"], 2, p["K"], 7)
    gVp, gS = torch.from_numpy(gVp).cuda(), torch.from_numpy(gS).cuda()
    runs = [tuple(t.cpu().numpy() for t in ctl.backward(gVp, gS)) for _ in range(3)]
    assert ctl.status() == 0
    ctl.close()
    for gV, gth in runs[1:]:
        np.testing.assert_array_equal(gV, runs[0][0])
        np.testing.assert_array_equal(gth, runs[0][1])
    assert np.all(np.isfinite(runs[0][0])) and np.all(np.isfinite(runs[0][1]))


@pytest.mark.parametrize("model", [0, 1])
def test_adjoint_does_not_depend_on_the_forward_launch(model):
    """The forward stores the same state checkpoints for any launch shape, so
    the backward gives the same bits whichever shape the forward ran (the
    benchmark tunes config 4's forward)."""
    from paper_2209_12842_gb300 import RaMppi

    if model == 0:
        p = rs.preset("c4_gradient", K=200, M=64, T=17)
        obs = rs.obstacles_ahead(1, 8, 0.15, 0.3, x_from=0.05, x_to=0.9, lateral=0.4)
        x0 = torch.tensor([0.0, -4.0, 0.0, 1.0], device="cuda")
    else:
        p = rs.preset("small_dyn", K=70, M=64, T=11)
        obs = rs.obstacles_ahead(1, 8, 0.15, 0.3, x_from=0.3, x_to=2.5)
        x0 = torch.from_numpy(rs.initial_state(1)).cuda()
    V = torch.from_numpy(rs.random_controls(model, p["T"], p["u_lo"], p["u_hi"], 3)).cuda()
    gVp, gS = rs.random_cotangents(p["T"], 2, p["K"], 7)
    gVp, gS = torch.from_numpy(gVp).cuda(), torch.from_numpy(gS).cuda()
    outs = []
    for launch in [(4, 1, 1), (2, 2, 1), (8, 1, 2), (2, 1, 2)]:
        ctl = RaMppi(p, obs, differentiable=True)
        ctl.set_launch(*launch)
        ctl.iteration = 0
        Vp = ctl.step(x0, V)
        gV, gth = ctl.backward(gVp, gS)
        outs.append((Vp.cpu().numpy(), gV.cpu().numpy(), gth.cpu().numpy()))
        assert ctl.status() == 0
        ctl.close()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            np.testing.assert_array_equal(a, b)


def test_adjoint_rejects_missing_flag():
    from paper_2209_12842_gb300 import RaMppi, RaMppiError

    q = rs.preset("small_kin")
    ctl = RaMppi(q, rs.obstacles_ahead(1, 4, 0.2, 0.3))
    ctl.step(torch.from_numpy(rs.initial_state(0)).cuda(), torch.zeros(q["T"], 2, device="cuda"))
    with pytest.raises(RaMppiError):
        ctl.backward(torch.ones(q["T"], 2, device="cuda"))
    ctl.close()
