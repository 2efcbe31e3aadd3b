"""Pins of the oracle's other disturbance families and risk measures (CPU).

Disturbances (the paper's noise study, Sec. V-B): uniform U[-a, a] (KS test
against scipy), impulse (jump rate p, jump size exactly a in a uniformly
random planar direction).  Risk measures in place of CVaR (the swappable
risk block, Sec. III-A): VaR = L_(ceil(alpha M)) (order statistic, and its
scaling identity), the chance measure P(L > c) against the Gaussian tail
probability of the linear test system, the mean against mu, mean-variance
against mu + kappa s^2 (M - 1) / M and hand values; with zero process noise
every measure equals the deterministic risk cost.
"""

import numpy as np
import pytest
from scipy import stats

import ra_scenes as rs


def test_uniform_disturbance(orc):
    p = rs.preset("c1_plain", noise_type=rs.NOISE_UNIFORM, w_scale=(0.2, 0.1, 0.05, 0.0))
    prob = orc.make_problem(p)
    w = np.array([orc.process_noise(prob, k, m, t) for k in range(3) for m in range(40) for t in range(40)])
    for s, a in enumerate((0.2, 0.1, 0.05)):
        a32 = float(np.float32(a))
        assert stats.kstest(w[:, s], stats.uniform(loc=-a32, scale=2 * a32).cdf).pvalue > 1e-3
        assert np.all(np.abs(w[:, s]) <= a32)
    assert np.all(w[:, 3] == 0)
    c = np.corrcoef(w[:, :3].T)
    assert np.max(np.abs(c - np.eye(3))) < 4 / np.sqrt(len(w))


def test_impulse_disturbance(orc):
    p = rs.preset("c1_plain", noise_type=rs.NOISE_IMPULSE, w_scale=(0.45, 0.45, 0.0, 0.0), mix_p=0.02)
    prob = orc.make_problem(p)
    w = np.array([orc.process_noise(prob, k, m, t) for k in range(10) for m in range(50) for t in range(50)])
    jump = np.any(w != 0, axis=1)
    n = len(w)
    assert abs(jump.mean() - 0.02) < 4 * np.sqrt(0.02 * 0.98 / n)
    mag = np.hypot(w[jump, 0], w[jump, 1])
    np.testing.assert_allclose(mag, float(np.float32(0.45)), rtol=1e-12)
    ang = np.arctan2(w[jump, 1], w[jump, 0])
    assert stats.kstest(ang, stats.uniform(loc=-np.pi, scale=2 * np.pi).cdf).pvalue > 1e-3
    assert np.all(w[:, 2:] == 0)


@pytest.mark.parametrize("B", [1.0, 0.5, 2.0])
def test_var_is_the_order_statistic(orc, B):
    rng = np.random.default_rng(3)
    for M in (1, 7, 32, 100):
        L = rng.gamma(2.0, size=M)
        for alpha in (0.5, 0.9, float(np.float32(0.95))):
            j = int(np.ceil(alpha * M))
            want = B * np.sort(L)[j - 1] + (1 - B) * L.mean()
            assert orc.risk(L, alpha, B, rs.RISK_VAR) == pytest.approx(want, rel=1e-12)


def test_chance_and_mean_linear_gaussian(orc):
    T, M = 10, 200_000
    sw = float(np.float32(0.5))
    c = float(np.float32(2.0))
    V = (np.arange(T) * 0.1 - 0.3).astype(np.float32).reshape(T, 1)
    x0 = np.array([0.25], np.float32)
    xs = 0.25 + np.concatenate([[0.0], np.cumsum(V[:, 0].astype(np.float64))])[:T]
    mu = xs.sum()
    s = sw * np.sqrt((T - 1) * T * (2 * T - 1) / 6.0)
    p = rs.preset("linear_test", K=1, M=M, T=T, w_scale=(sw, 0, 0, 0), cvar_mode=rs.RISK_CHANCE, risk_param=c)
    out = orc.samples(p, x0, V, np.zeros((0, 3), np.float32), ks=[0])
    want = stats.norm.sf((c - mu) / s)
    assert abs(out["cvar"][0] - want) < 4 * np.sqrt(want * (1 - want) / M), (out["cvar"][0], want)
    p = dict(p, cvar_mode=rs.RISK_MEAN)
    out = orc.samples(p, x0, V, np.zeros((0, 3), np.float32), ks=[0])
    assert abs(out["cvar"][0] - mu) < 4 * s / np.sqrt(M)


def test_zero_noise_every_measure_is_the_cost(orc):
    p = rs.preset("small_kin", w_scale=(0, 0, 0, 0), gamma=0.0, risk_mask=rs.RISK_OBS | rs.RISK_DEV | rs.RISK_SPEED)
    obs = rs.obstacles_ahead(1, 8, 0.15, 0.3)
    x0 = rs.initial_state(0)
    V = rs.random_controls(0, p["T"], p["u_lo"], p["u_hi"], 2)
    for mode in (rs.RISK_VAR, rs.RISK_MEAN, rs.RISK_MEANVAR):
        out = orc.samples(dict(p, cvar_mode=mode, risk_param=3.0), x0, V, obs, want_L=True)
        np.testing.assert_allclose(out["cvar"], out["L"][:, 0], rtol=1e-12)
    out = orc.samples(dict(p, cvar_mode=rs.RISK_CHANCE, risk_param=500.0), x0, V, obs, want_L=True)
    np.testing.assert_array_equal(out["cvar"], (out["L"][:, 0] > 500.0).astype(float))


def test_mean_variance_hand_values(orc):
    mv = rs.RISK_MEANVAR
    # L = (0, 2): mean 1, population variance 1
    assert orc.risk(np.array([0.0, 2.0]), 0.9, 1.0, mv, 3.0) == 4.0
    # B = 2 doubles the deviations: variance 4
    assert orc.risk(np.array([0.0, 2.0]), 0.9, 2.0, mv, 3.0) == 13.0
    # L = (1, 1, 4): mean 2, variance (1 + 1 + 4) / 3 = 2
    assert orc.risk(np.array([1.0, 1.0, 4.0]), 0.5, 1.0, mv, 0.5) == pytest.approx(3.0, rel=1e-15)
    rng = np.random.default_rng(8)
    L = rng.gamma(2.0, size=50)
    # kappa = 0 and B = 0 give the mean; a shift moves it by the shift
    assert orc.risk(L, 0.9, 1.0, mv, 0.0) == pytest.approx(L.mean(), rel=1e-14)
    assert orc.risk(L, 0.9, 0.0, mv, 7.0) == pytest.approx(L.mean(), rel=1e-14)
    assert orc.risk(L + 10.0, 0.9, 1.0, mv, 2.0) == pytest.approx(orc.risk(L, 0.9, 1.0, mv, 2.0) + 10.0, rel=1e-13)
    assert orc.risk(np.full(9, 5.0), 0.9, 1.0, mv, 4.0) == 5.0


def test_mean_variance_linear_gaussian(orc):
    T, M = 10, 200_000
    sw = float(np.float32(0.5))
    kappa = float(np.float32(0.3))
    V = (np.arange(T) * 0.1 - 0.3).astype(np.float32).reshape(T, 1)
    x0 = np.array([0.25], np.float32)
    xs = 0.25 + np.concatenate([[0.0], np.cumsum(V[:, 0].astype(np.float64))])[:T]
    mu = xs.sum()
    s2 = sw**2 * (T - 1) * T * (2 * T - 1) / 6.0
    p = rs.preset("linear_test", K=1, M=M, T=T, w_scale=(sw, 0, 0, 0), cvar_mode=rs.RISK_MEANVAR, risk_param=kappa)
    out = orc.samples(p, x0, V, np.zeros((0, 3), np.float32), ks=[0])
    want = mu + kappa * s2 * (M - 1) / M
    # standard error of mean + kappa * variance for a normal sample
    se = np.sqrt(s2 / M + kappa**2 * 2 * s2**2 / (M - 1))
    assert abs(out["cvar"][0] - want) < 4 * se, (out["cvar"][0], want, se)
