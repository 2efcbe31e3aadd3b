"""GPU parity of the other disturbance families, risk measures, large M,
warps-per-sample launch shapes and the paper's simulation preset (needs a
GB300), against the oracle with the stage-wise protocol of the parity tests.
"""

import numpy as np
import pytest

import oracle
import ra_scenes as rs
from parity_util import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_12842_gb300 import build as b

    b.build()


def _gpu(p, obs, x0, V, launch=None, iteration=0, keep_L=True):
    from paper_2209_12842_gb300 import RaMppi

    ctl = RaMppi(p, obs, keep_risk_costs=keep_L)
    if launch is not None:
        ctl.set_launch(*launch)
    ctl.iteration = iteration
    Vp = ctl.step(torch.from_numpy(np.asarray(x0, np.float32)).cuda(), torch.from_numpy(np.asarray(V, np.float32)).cuda())
    ws = ctl.workspace()
    torch.cuda.synchronize()
    g = dict(V_plus=Vp.cpu().numpy(), S_tilde=ctl.S_tilde.cpu().numpy(), cvar=ctl.cvar.cpu().numpy(),
             U=ws["U"].cpu().numpy(), S=ws["S"].cpu().numpy(), L=ws["L"].cpu().numpy() if keep_L else None,
             status=ctl.status())
    ctl.close()
    return g


def _scene(p, dense=True):
    model = p["model"]
    if dense:
        return rs.obstacles_ahead(4, max(int(p["n_obs"]), 1), *p["obs_r"], x_from=0.1 if model == 1 else 0.3,
                                  x_to=1.2 if model == 1 else 2.5)
    return rs.scene_obstacles(p)


@pytest.mark.parametrize("name", ["small_kin", "small_dyn"])
@pytest.mark.parametrize("noise", ["uniform", "impulse"])
def test_disturbance_families(name, noise):
    if noise == "uniform":
        ov = dict(noise_type=rs.NOISE_UNIFORM)
    else:
        ov = dict(noise_type=rs.NOISE_IMPULSE, mix_p=0.05,
                  w_scale=(0.45, 0.45, 0.0, 0.0) if name == "small_kin" else (0.5, 0.5, 0.5, 0.0))
    p = rs.preset(name, **ov)
    obs = _scene(p)
    x0 = rs.initial_state(p["model"])
    V = rs.random_controls(p["model"], p["T"], p["u_lo"], p["u_hi"], 3)
    g = _gpu(p, obs, x0, V)
    assert g["status"] == 0
    compare(p, g, oracle.samples(p, x0, V, obs, n_threads=8))


@pytest.mark.parametrize("mode", ["var", "chance", "mean", "meanvar"])
def test_risk_measures(mode):
    m = {"var": rs.RISK_VAR, "chance": rs.RISK_CHANCE, "mean": rs.RISK_MEAN, "meanvar": rs.RISK_MEANVAR}[mode]
    param = 1e-3 if mode == "meanvar" else 500.0
    for B in (1.0, 2.0):
        p = rs.preset("small_kin", cvar_mode=m, B=B, risk_param=param, K=96)
        obs = _scene(p)
        x0 = rs.initial_state(0)
        V = rs.random_controls(0, p["T"], p["u_lo"], p["u_hi"], 5)
        g = _gpu(p, obs, x0, V)
        ref = oracle.samples(p, x0, V, obs, n_threads=8)
        if B == 1.0:
            compare(p, g, ref)
        # the measure of the GPU's own risk costs
        a = float(np.float32(p["alpha"]))
        for k in range(p["K"]):
            Lk = g["L"][k].astype(np.float64)
            if m == rs.RISK_CHANCE and B != 1.0:
                # the scaled cost is formed in float32 on the GPU: a cost within
                # rounding of the threshold may fall on either side
                lo = oracle.risk(Lk, a, B, m, param + 1e-3)
                hi = oracle.risk(Lk, a, B, m, param - 1e-3)
                assert lo - 1e-7 <= g["cvar"][k] <= hi + 1e-7, (mode, B, k, g["cvar"][k], lo, hi)
                continue
            want = oracle.risk(Lk, a, B, m, float(np.float32(param)))
            assert abs(g["cvar"][k] - want) <= 1e-5 * max(1.0, abs(want)), (mode, B, k, g["cvar"][k], want)


@pytest.mark.parametrize("M,launch", [(300, (4, 1, 4)), (300, (8, 2, 2)), (512, (8, 1, 8)), (512, (4, 4, 1)),
                                      (100, (2, 1, 2)), (300, (5, 2, 5)), (300, (6, 2, 3)), (512, (3, 2, 3)),
                                      (100, (6, 4, 1))])
def test_large_M_and_warps_per_sample(M, launch):
    p = rs.preset("small_dyn", M=M, K=37)
    obs = _scene(p)
    x0 = rs.initial_state(1)
    V = rs.random_controls(1, p["T"], p["u_lo"], p["u_hi"], 7)
    base = _gpu(p, obs, x0, V, launch=(4, 1, 1))
    g = _gpu(p, obs, x0, V, launch=launch)
    for key in ("U", "S", "cvar", "S_tilde", "L"):
        np.testing.assert_array_equal(g[key], base[key], err_msg=f"{launch} {key}")
    compare(p, g, oracle.samples(p, x0, V, obs, n_threads=8))


@pytest.mark.parametrize("M", [32, 17, 5])
@pytest.mark.parametrize("launch", [(4, 2, 1), (1, 2, 1), (7, 2, 1)])
def test_two_samples_per_warp(M, launch):
    """At most 32 rollouts per sample, dynamic model, interleave 2: each warp
    steps two samples at once; an odd K leaves the last warp's second sample
    empty. Same bits as one sample per warp, and the oracle's results."""
    p = rs.preset("small_dyn", M=M, K=37)
    obs = _scene(p)
    x0 = rs.initial_state(1)
    V = rs.random_controls(1, p["T"], p["u_lo"], p["u_hi"], 9)
    base = _gpu(p, obs, x0, V, launch=(4, 1, 1))
    g = _gpu(p, obs, x0, V, launch=launch)
    for key in ("U", "S", "cvar", "S_tilde", "L", "V_plus"):
        np.testing.assert_array_equal(g[key], base[key], err_msg=f"{launch} {key}")
    compare(p, g, oracle.samples(p, x0, V, obs, n_threads=8))


def test_two_samples_per_warp_is_the_default():
    from paper_2209_12842_gb300 import RaMppi

    p = rs.preset("small_dyn", M=32, K=64)
    ctl = RaMppi(p, _scene(p))
    assert ctl.get_launch()[1] == 2
    ctl.close()


@pytest.mark.parametrize("launch", [(4, 1, 1), (4, 2, 2), (8, 2, 1), (3, 1, 3)])
def test_obstacle_x_window(launch):
    """More than 64 obstacles on the dynamic model: the cull first narrows to
    the obstacles within the largest radius of the warp's box in x (stored
    sorted by x).  Small obstacles along the path, a few large ones (the
    largest radius sets the window) and far-away ones on both sides; counts
    must equal the oracle's, with the same bits for every launch shape."""
    p = rs.preset("small_dyn", K=37, M=64, n_obs=120)
    near = rs.obstacles_ahead(11, 100, 0.02, 0.08, x_from=-0.5, x_to=1.5, lateral=0.5)
    big = np.array([[0.9, -3.2, 0.6], [-3.0, -4.0, 0.9]], np.float32)
    far = rs.obstacles_ahead(12, 18, 0.1, 0.3, x_from=-40.0, x_to=40.0, lateral=20.0)
    obs = np.concatenate([near, big, far])
    x0 = rs.initial_state(1)
    V = rs.random_controls(1, p["T"], p["u_lo"], p["u_hi"], 5)
    base = _gpu(p, obs, x0, V, launch=(4, 1, 1))
    g = _gpu(p, obs, x0, V, launch=launch)
    for key in ("U", "S", "cvar", "S_tilde", "L"):
        np.testing.assert_array_equal(g[key], base[key], err_msg=f"{launch} {key}")
    assert np.any(g["L"] > 0)
    compare(p, g, oracle.samples(p, x0, V, obs, n_threads=8))


@pytest.mark.parametrize("name,n_obs", [("small_dyn", 120), ("small_kin", 40)])
def test_obstacle_order_does_not_matter(name, n_obs):
    """The library keeps the obstacles sorted by x; with the indicator cost the
    results are the same bits for any order of the input list."""
    p = rs.preset(name, K=37, M=64, n_obs=n_obs)
    obs = rs.obstacles_ahead(13, n_obs, 0.05, 0.2, x_from=-0.5, x_to=2.0, lateral=0.5)
    x0 = rs.initial_state(p["model"])
    V = rs.random_controls(p["model"], p["T"], p["u_lo"], p["u_hi"], 6)
    a = _gpu(p, obs, x0, V)
    b = _gpu(p, obs[np.random.default_rng(0).permutation(n_obs)], x0, V)
    for key in ("U", "S", "cvar", "S_tilde", "L", "V_plus"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)


def test_paper_preset():
    p = rs.preset("paper_sim", K=96)
    obs = rs.scene_obstacles(p)
    obs = np.concatenate([obs, np.array([[0.25, -0.3, 0.1], [0.45, -0.2, 0.1]], np.float32)])
    p["n_obs"] = len(obs)
    x0 = rs.scene_initial_state(p)
    V = rs.random_controls(1, p["T"], p["u_lo"], p["u_hi"], 9)
    g = _gpu(p, obs, x0, V)
    assert g["status"] == 0
    compare(p, g, oracle.samples(p, x0, V, obs, n_threads=8))


@pytest.mark.parametrize("mode", ["var", "mean", "meanvar"])
def test_adjoint_other_measures(mode):
    from paper_2209_12842_gb300 import RaMppi

    m = {"var": rs.RISK_VAR, "mean": rs.RISK_MEAN, "meanvar": rs.RISK_MEANVAR}[mode]
    p = rs.preset("c4_gradient", K=96, M=32, T=12, cvar_mode=m, risk_param=0.05, B=1.5,
                  risk_mask=rs.RISK_OBS | rs.RISK_DEV)
    obs = rs.obstacles_ahead(1, 8, 0.15, 0.3, x_from=0.05, x_to=0.9, lateral=0.4)
    x0 = np.array([0.0, -4.0, 0.0, 1.0], np.float32)
    V = rs.random_controls(0, p["T"], p["u_lo"], p["u_hi"], 3)
    gVp, gS = rs.random_cotangents(p["T"], 2, p["K"], 7)
    ctl = RaMppi(p, obs, differentiable=True)
    ctl.step(torch.from_numpy(x0).cuda(), torch.from_numpy(V).cuda())
    gV, gth = ctl.backward(torch.from_numpy(gVp).cuda(), torch.from_numpy(gS).cuda())
    torch.cuda.synchronize()
    ctl.close()
    rV, rth = oracle.backward(p, x0, V, obs, gVp, gS)
    for got, want in ((gV.cpu().numpy(), rV), (gth.cpu().numpy(), rth)):
        got, want = np.asarray(got, np.float64).ravel(), np.asarray(want, np.float64).ravel()
        assert np.linalg.norm(got - want) <= 1e-3 * np.linalg.norm(want), (mode, got, want)


def test_obstacle_extent_is_enforced():
    from paper_2209_12842_gb300 import RaMppi, RaMppiError

    p = rs.preset("small_kin")
    ctl = RaMppi(p, np.array([[499.0, -10.0, 1.0]], np.float32))  # on the boundary: accepted
    for bad in ([[499.5, 0.0, 1.0]], [[0.0, -600.0, 0.3]], [[0.0, 0.0, 501.0]]):
        with pytest.raises(RaMppiError):
            ctl.set_obstacles(np.array(bad, np.float32))
    ctl.close()
