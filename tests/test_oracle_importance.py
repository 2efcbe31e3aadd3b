"""Pins of the oracle's importance-sampled risk (CPU).

The paper leaves importance sampling out and only names it as the remedy
when alpha approaches 1 (Sec. III-A).  The oracle's reading: the last
floor(is_frac M) rollouts of a sample draw their process noise at is_scale
times its size, every rollout gets the deterministic-mixture (balance
heuristic) weight w = 1 / ((1 - b) + b q/p) of its noise path, b the
fraction drawn from the proposal, and the risk measures become those of the
weighted empirical distribution of the risk costs.

Pins:
- equal weights give the unweighted measures (whose own pins are in
  test_oracle_cvar.py and test_oracle_families.py);
- weighted RU CVaR equals the brute-force minimum of the Rockafellar-Uryasev
  objective over its breakpoints;
- integer weights equal replicating each cost that many times, for every
  measure (this fixes the weighted VaR index and the variance's divisor);
- scaling all weights changes nothing;
- the weights equal 1 / ((1 - b) + b exp(G)) with G summed from scipy's
  normal and Laplace log densities over the path's values (branch read from
  the selector word), and E_p[w] = 1 (unbiasedness) within sampling error;
- with importance sampling switched off (is_frac = 0, is_scale = 1, or
  fewer than one proposal rollout) results are bit-identical to the plain
  oracle;
- on the linear-Gaussian test system at alpha = 0.99 the importance-sampled
  CVaR is unbiased for the closed form within sampling error and has a
  smaller spread than plain Monte Carlo with the same M.
"""

import numpy as np
import pytest
from scipy import stats

import ra_scenes as rs

MODES = (rs.CVAR_RU, rs.CVAR_TCE, rs.RISK_VAR, rs.RISK_CHANCE, rs.RISK_MEAN, rs.RISK_MEANVAR)


def _ru_weighted_bruteforce(L, w, alpha):
    W = w.sum()
    tau = (1.0 - alpha) * W
    return min(c + np.sum(w * np.maximum(L - c, 0.0)) / tau for c in L)


@pytest.mark.parametrize("B", [1.0, 0.5, 2.0])
def test_equal_weights_give_the_unweighted_measures(orc, B):
    rng = np.random.default_rng(1)
    for M in (1, 5, 32, 129):
        L = np.round(rng.gamma(2.0, size=M), 1)  # ties included
        for alpha in (0.5, float(np.float32(0.9)), float(np.float32(0.99))):
            for mode in MODES:
                thr = 2.0 if mode == rs.RISK_CHANCE else 0.7
                want = orc.risk(L, alpha, B, mode, thr)
                got = orc.risk_w(L, np.full(M, 3.0), alpha, B, mode, thr)
                assert got == pytest.approx(want, rel=1e-12, abs=1e-12), (M, alpha, mode)


@pytest.mark.parametrize("alpha", [0.5, 0.9, 0.99])
def test_weighted_ru_equals_bruteforce(orc, alpha):
    rng = np.random.default_rng(2)
    for M in (1, 2, 7, 40):
        for _ in range(20):
            L = rng.normal(size=M)
            w = rng.gamma(0.5, size=M) + 1e-3
            got = orc.risk_w(L, w, alpha, 1.0, rs.CVAR_RU)
            assert got == pytest.approx(_ru_weighted_bruteforce(L, w, alpha), rel=1e-12, abs=1e-12)


def test_integer_weights_equal_replication(orc):
    rng = np.random.default_rng(3)
    for M in (1, 3, 10, 33):
        for _ in range(10):
            L = np.round(rng.normal(size=M), 1)
            n = rng.integers(1, 4, size=M)
            rep = np.repeat(L, n)
            for alpha in (0.5, 0.75, float(np.float32(0.9)), float(np.float32(0.97))):
                for B in (1.0, 0.5):
                    for mode in MODES:
                        want = orc.risk(rep, alpha, B, mode, 0.3137)
                        got = orc.risk_w(L, n.astype(float), alpha, B, mode, 0.3137)
                        assert got == pytest.approx(want, rel=1e-12, abs=1e-12), (M, alpha, B, mode)


def test_weight_scale_invariance_and_non_finite(orc):
    rng = np.random.default_rng(4)
    L = rng.normal(size=50)
    w = rng.gamma(1.0, size=50)
    for mode in MODES:
        a = orc.risk_w(L, w, 0.9, 1.0, mode, 0.1)
        assert orc.risk_w(L, 17.0 * w, 0.9, 1.0, mode, 0.1) == pytest.approx(a, rel=1e-12, abs=1e-14)
    L[7] = np.nan
    assert orc.risk_w(L, w, 0.9, 1.0, rs.CVAR_RU) == np.inf


def _key(p, iteration):
    seed = int(p["seed"])
    return np.array([seed & 0xFFFFFFFF, ((seed >> 32) ^ iteration) & 0xFFFFFFFF], np.uint32)


def _log_ratio_path(orc, p, prob, k, m, g, s):
    """ln q - ln p over rollout m's path, from scipy's densities."""
    G = 0.0
    key = _key(p, 0)
    thresh = np.floor(min(np.float64(np.float32(p["mix_p"])) * 2.0**32, 2.0**32 - 1))
    for t in range(int(p["T"])):
        w = g * orc.process_noise(prob, k, m, t)  # the nominal values, scaled
        sel = orc.philox([t, m, k, int(p["instance_id"])], key)
        for slot in range(3 if p["model"] == rs.MODEL_DYN_SINGLE_TRACK else 4 if p["model"] == 0 else 1):
            b = float(np.float32(p["w_scale"][slot]))
            if b == 0.0:
                continue
            if p["noise_type"] == rs.NOISE_GAUSS:
                dist_p, dist_q = stats.norm(scale=b), stats.norm(scale=s * b)
            elif sel[slot] < thresh:
                sd = float(np.float32(p["mix_scale"])) * b
                dist_p, dist_q = stats.norm(scale=sd), stats.norm(scale=s * sd)
            else:
                dist_p, dist_q = stats.laplace(scale=b), stats.laplace(scale=s * b)
            G += dist_q.logpdf(w[slot]) - dist_p.logpdf(w[slot])
    return G


@pytest.mark.parametrize("name", ["small_kin", "small_dyn"])
def test_weights_from_library_densities(orc, name):
    s, frac = 1.5, 0.25
    p = rs.preset(name, M=16, T=6, is_scale=s, is_frac=frac, mix_p=0.3 if name == "small_dyn" else 0.0)
    prob = orc.make_problem(p)
    s32 = float(np.float32(s))
    M_s = int(np.floor(float(np.float32(frac)) * 16))
    b = M_s / 16
    for k in (0, 5):
        w = orc.is_weights(p, k)
        for m in range(16):
            g = s32 if m >= 16 - M_s else 1.0
            G = _log_ratio_path(orc, p, prob, k, m, g, s32)
            assert w[m] == pytest.approx(1.0 / ((1.0 - b) + b * np.exp(G)), rel=1e-11), (k, m)
        assert np.all(w <= 1.0 / (1.0 - b) + 1e-15)


@pytest.mark.parametrize("name,noise", [("linear_test", rs.NOISE_GAUSS), ("small_dyn", rs.NOISE_LAPLACE_MIX)])
def test_weights_are_unbiased(orc, name, noise):
    """E_p[w] = 1 for the balance-heuristic weights: the mean over the
    nominal and proposal rollouts together estimates it without bias."""
    p = rs.preset(name, M=200, T=8, noise_type=noise, is_scale=1.3, is_frac=0.5,
                  mix_p=0.1 if noise == rs.NOISE_LAPLACE_MIX else 0.0)
    w = np.concatenate([orc.is_weights(p, k) for k in range(20)])
    assert abs(w.mean() - 1.0) < 4 * w.std() / np.sqrt(w.size), (w.mean(), w.std())


@pytest.mark.parametrize("off", [dict(is_frac=0.0, is_scale=2.0), dict(is_frac=0.5, is_scale=1.0),
                                 dict(is_frac=0.01, is_scale=2.0)])
def test_switched_off_is_bit_identical(orc, off):
    p = rs.preset("small_kin", M=64)
    obs = rs.obstacles_ahead(1, 8, 0.15, 0.3)
    x0 = rs.initial_state(0)
    V = rs.random_controls(0, p["T"], p["u_lo"], p["u_hi"], 2)
    a = orc.samples(p, x0, V, obs, want_L=True)
    b = orc.samples(dict(p, **off), x0, V, obs, want_L=True)
    for key in ("S", "cvar", "S_tilde", "L", "cvar_lo", "cvar_hi"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)
    assert np.all(orc.is_weights(dict(p, **off), 3) == 1.0)


def test_unsupported_noise_types_are_refused(orc):
    for noise in (rs.NOISE_UNIFORM, rs.NOISE_IMPULSE):
        p = rs.preset("small_kin", noise_type=noise, is_scale=1.5, is_frac=0.5, mix_p=0.02)
        with pytest.raises(RuntimeError):
            orc.is_weights(p, 0)
        with pytest.raises(RuntimeError):
            orc.samples(p, rs.initial_state(0), np.zeros((p["T"], 2), np.float32), np.zeros((0, 3), np.float32))


def test_proposal_rollouts_are_scaled(orc):
    """The last floor(is_frac M) rollouts carry exactly is_scale times the
    nominal noise: with one step the risk cost c x_1 is linear in it."""
    p = rs.preset("linear_test", K=2, M=8, T=2, w_scale=(0.5, 0, 0, 0), is_scale=2.0, is_frac=0.25)
    V = np.zeros((2, 1), np.float32)
    x0 = np.array([0.0], np.float32)
    on = orc.samples(p, x0, V, np.zeros((0, 3), np.float32), want_L=True)["L"]
    off = orc.samples(dict(p, is_frac=0.0), x0, V, np.zeros((0, 3), np.float32), want_L=True)["L"]
    np.testing.assert_array_equal(on[:, :6], off[:, :6])
    np.testing.assert_allclose(on[:, 6:], 2.0 * off[:, 6:], rtol=1e-15)


@pytest.mark.slow
def test_linear_gaussian_alpha_099(orc):
    """Closed-form CVaR of the linear-Gaussian system (see the P2 pin): the
    importance-sampled estimate is unbiased within sampling error, with a
    smaller spread across independent samples than plain Monte Carlo."""
    T, M, K = 10, 1000, 300
    sw = float(np.float32(0.5))
    alpha = float(np.float32(0.99))
    V = (np.arange(T) * 0.1 - 0.3).astype(np.float32).reshape(T, 1)
    x0 = np.array([0.25], np.float32)
    xs = 0.25 + np.concatenate([[0.0], np.cumsum(V[:, 0].astype(np.float64))])[:T]
    mu = xs.sum()
    s = sw * np.sqrt((T - 1) * T * (2 * T - 1) / 6.0)
    want = mu + s * stats.norm.pdf(stats.norm.ppf(alpha)) / (1 - alpha)
    base = rs.preset("linear_test", K=K, M=M, T=T, w_scale=(sw, 0, 0, 0), alpha=alpha)
    plain = orc.samples(base, x0, V, np.zeros((0, 3), np.float32), n_threads=8)["cvar"]
    imp = orc.samples(dict(base, is_scale=1.5, is_frac=0.5), x0, V, np.zeros((0, 3), np.float32),
                      n_threads=8)["cvar"]
    for cv in (plain, imp):
        # the O(1/M) bias of the empirical CVaR plus 4 standard errors of the mean
        assert abs(cv.mean() - want) < 0.02 * s + 4 * cv.std() / np.sqrt(K), (cv.mean(), want)
    assert imp.std() < 0.85 * plain.std(), (imp.std(), plain.std())
