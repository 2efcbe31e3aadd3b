"""GPU parity of the importance-sampled rollouts (needs a GB300).

With is_scale = s and is_frac = f, the last floor(f M) rollouts of a sample
draw their process noise at s times its size, and the risk measures are those
of the weighted empirical distribution of the M risk costs under the
deterministic-mixture weights (the oracle's reading; the paper only names
importance sampling for alpha near 1, Sec. III-A).  Checked against the
oracle with the stage-wise protocol; the risk costs of the nominal-scale
rollouts keep the bits of a run without importance sampling; results do not
depend on the launch shape; the discrete measures (VaR, the literal tail
mean) are checked for validity, since a float32 weight sum may pick the
neighbouring order statistic where the FP64 sums are within rounding of
(1 - alpha) W.
"""

import numpy as np
import pytest

import oracle
import ra_scenes as rs
from parity_util import compare, importance_on

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_12842_gb300 import build as b

    b.build()


def _gpu(p, obs, x0, V, launch=None):
    from paper_2209_12842_gb300 import RaMppi

    ctl = RaMppi(p, obs, keep_risk_costs=True)
    if launch is not None:
        ctl.set_launch(*launch)
    Vp = ctl.step(torch.from_numpy(np.asarray(x0, np.float32)).cuda(), torch.from_numpy(np.asarray(V, np.float32)).cuda())
    ws = ctl.workspace()
    torch.cuda.synchronize()
    g = dict(V_plus=Vp.cpu().numpy(), S_tilde=ctl.S_tilde.cpu().numpy(), cvar=ctl.cvar.cpu().numpy(),
             U=ws["U"].cpu().numpy(), S=ws["S"].cpu().numpy(), L=ws["L"].cpu().numpy(), status=ctl.status())
    if importance_on(p):
        g["W"] = ctl.importance_weights().cpu().numpy()
    ctl.close()
    return g


def _case(name, **ov):
    p = rs.preset(name, is_scale=1.5, is_frac=0.5, **ov)
    model = p["model"]
    obs = rs.obstacles_ahead(4, max(int(p["n_obs"]), 1), *p["obs_r"], x_from=0.1 if model == 1 else 0.3,
                             x_to=1.2 if model == 1 else 2.5)
    x0 = rs.initial_state(model)
    V = rs.random_controls(model, p["T"], p["u_lo"], p["u_hi"], 4)
    return p, obs, x0, V


@pytest.mark.parametrize("name", ["small_kin", "small_dyn"])
@pytest.mark.parametrize("mode", [rs.CVAR_RU, rs.RISK_MEAN, rs.RISK_CHANCE, rs.RISK_MEANVAR])
def test_importance_parity(name, mode):
    p, obs, x0, V = _case(name, cvar_mode=mode, alpha=0.95, risk_param=500.0 if mode == rs.RISK_CHANCE else 1e-3)
    g = _gpu(p, obs, x0, V)
    assert g["status"] == 0
    compare(p, g, oracle.samples(p, x0, V, obs, n_threads=8))


@pytest.mark.parametrize("name", ["small_kin", "small_dyn"])
def test_nominal_scale_rollouts_keep_their_bits(name):
    p, obs, x0, V = _case(name)
    g = _gpu(p, obs, x0, V)
    plain = _gpu(dict(p, is_frac=0.0), obs, x0, V)
    m0 = int(p["M"]) - int(np.floor(float(np.float32(0.5)) * int(p["M"])))
    np.testing.assert_array_equal(g["L"][:, :m0], plain["L"][:, :m0])
    np.testing.assert_array_equal(g["S"], plain["S"])
    np.testing.assert_array_equal(g["U"], plain["U"])
    # switched off by the scale: the plain kernel, same bits everywhere
    off = _gpu(dict(p, is_scale=1.0), obs, x0, V)
    for key in ("L", "cvar", "S_tilde", "V_plus"):
        np.testing.assert_array_equal(off[key], plain[key], err_msg=key)


@pytest.mark.parametrize("launch", [(4, 2, 1), (8, 2, 2), (2, 1, 2), (3, 1, 1)])
def test_importance_launch_shapes(launch):
    p, obs, x0, V = _case("small_dyn", M=100, K=37)
    base = _gpu(p, obs, x0, V, launch=(4, 1, 1))
    g = _gpu(p, obs, x0, V, launch=launch)
    for key in ("L", "cvar", "S_tilde", "V_plus"):
        np.testing.assert_array_equal(g[key], base[key], err_msg=f"{launch} {key}")
    compare(p, g, oracle.samples(p, x0, V, obs, n_threads=8))


@pytest.mark.parametrize("M,launch", [(512, (8, 2, 8)), (512, (4, 1, 4)), (33, (2, 1, 1)), (300, (6, 2, 3)),
                                      (2, (4, 2, 1))])
def test_importance_sizes(M, launch):
    # large, ragged and tiny M (M = 2 with f = 1/2: one proposal rollout)
    p, obs, x0, V = _case("small_kin", M=M, K=21)
    base = _gpu(p, obs, x0, V, launch=(4, 1, 1))
    g = _gpu(p, obs, x0, V, launch=launch)
    for key in ("L", "W", "cvar", "S_tilde", "V_plus"):
        np.testing.assert_array_equal(g[key], base[key], err_msg=f"{M} {launch} {key}")
    compare(p, g, oracle.samples(p, x0, V, obs, n_threads=8))


def test_importance_config2_full_size_sampled():
    # config 2 at full size (K = 4096, M = 128, T = 40, mixture noise) with
    # importance sampling, on sampled k, in the tuned launch
    from paper_2209_12842_gb300 import RaMppi

    p = rs.preset("c2_closed_loop", is_scale=1.1, is_frac=0.5, alpha=0.99)
    obs = rs.obstacles_ahead(5, int(p["n_obs"]), *p["obs_r"], x_from=0.1, x_to=1.2)
    x0 = rs.initial_state(1)
    V = rs.random_controls(1, p["T"], p["u_lo"], p["u_hi"], 4)
    ctl = RaMppi(p, obs)
    ctl.tune(torch.from_numpy(x0).cuda(), torch.from_numpy(V).cuda(), 2)
    launch = ctl.get_launch()
    ctl.close()
    g = _gpu(p, obs, x0, V, launch=launch)
    K = int(p["K"])
    ks = np.unique(np.concatenate([[0, K // 2, K - 1], np.random.default_rng(3).integers(0, K, 13)])).astype(np.int32)
    compare(p, g, oracle.samples(p, x0, V, obs, ks=ks, n_threads=8))


def test_importance_single_rollout_is_plain():
    # M = 1: floor(f M) = 0 proposal rollouts, so importance sampling is off
    p, obs, x0, V = _case("small_dyn", M=1)
    g = _gpu(p, obs, x0, V)
    plain = _gpu(dict(p, is_frac=0.0), obs, x0, V)
    for key in ("L", "cvar", "S_tilde", "V_plus"):
        np.testing.assert_array_equal(g[key], plain[key], err_msg=key)
    assert "W" not in g


@pytest.mark.parametrize("mode", [rs.RISK_VAR, rs.CVAR_TCE])
def test_importance_var_and_tail_mean_are_valid(mode):
    """VaR must be a risk cost v with W(L > v) <= tau <= W(L >= v) up to
    float32 rounding of the weight sums; the literal tail mean must be the
    weighted mean over {L >= v} for such a v."""
    p, obs, x0, V = _case("small_kin", cvar_mode=mode, alpha=0.9, M=64)
    g = _gpu(p, obs, x0, V)
    alpha = float(np.float32(0.9))
    for k in range(int(p["K"])):
        L = g["L"][k].astype(np.float64)
        w = g["W"][k].astype(np.float64)  # the kernel's own weights (checked against the oracle's elsewhere)
        W = w.sum()
        tau = (1 - alpha) * W
        slack = 1e-5 * W
        v = g["cvar"][k] if mode == rs.RISK_VAR else None
        if mode == rs.RISK_VAR:
            assert v in L, (k, v)
            cands = [v]
        else:
            cands = [c for c in np.unique(L) if w[L > c].sum() <= tau + slack and w[L >= c].sum() >= tau - slack]
        ok = False
        for c in cands:
            valid = w[L > c].sum() <= tau + slack and w[L >= c].sum() >= tau - slack
            if mode == rs.RISK_VAR:
                ok |= valid
            else:
                tce = np.sum(w[L >= c] * L[L >= c]) / w[L >= c].sum()
                ok |= valid and abs(g["cvar"][k] - tce) <= 1e-5 * max(1.0, abs(tce))
        assert ok, (k, g["cvar"][k])


def test_importance_is_refused_where_unsupported():
    from paper_2209_12842_gb300 import RaMppi
    from paper_2209_12842_gb300.binding import RaMppiError

    p, obs, x0, V = _case("small_kin")
    ctl = RaMppi(p, obs)
    with pytest.raises(RaMppiError):
        ctl.set_launch(4, 4, 1)  # importance-sampled rollouts interleave 1 or 2
    ctl.close()
    plain = RaMppi(dict(p, is_frac=0.0), obs, keep_risk_costs=True)
    plain.step(torch.from_numpy(x0).cuda(), torch.from_numpy(V).cuda())
    with pytest.raises(RaMppiError):
        plain.importance_weights()  # no weights without importance sampling
    plain.close()
