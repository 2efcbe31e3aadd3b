"""Pins of the oracle's risk measure (CPU only).

P1  fractional sorted-tail CVaR equals the Rockafellar-Uryasev minimum
    min_c c + sum (L - c)_+ / ((1 - alpha) M), found by brute force
P2  CVaR of a Gaussian risk cost (linear test system) matches
    mu + s phi(Phi^-1(alpha)) / (1 - alpha) within 4 standard errors
P6  risk sensitivity scaling (Eqs. 18, 19): CVaR(L_a) = B CVaR(L) + (1 - B) mean
P7  literal tail mean (Eqs. 12, 13) <= fractional tail <= max; both equal
    their order-statistic forms when alpha M is an integer
"""

import numpy as np
import pytest
from scipy import stats

import ra_scenes as rs

ALPHAS = [float(np.float32(a)) for a in (0.5, 0.75, 0.8, 0.9, 0.95, 0.99, 0.3)]


def _ru_bruteforce(L, alpha):
    L = np.asarray(L, dtype=np.float64)
    M = L.size
    # the objective is convex piecewise linear with kinks at the samples
    return min(c + np.maximum(L - c, 0).sum() / ((1 - alpha) * M) for c in L)


@pytest.mark.parametrize("alpha", ALPHAS)
def test_p1_ru_equals_bruteforce(orc, alpha):
    rng = np.random.default_rng(int(alpha * 1000))
    for M in (1, 2, 3, 5, 8, 10, 16):
        for trial in range(6):
            if trial % 3 == 0:
                L = rng.normal(size=M)
            elif trial % 3 == 1:
                L = rng.integers(0, 3, size=M) * 1000.0  # heavy ties (indicator costs)
            else:
                L = rng.exponential(size=M)
            got = orc.cvar(L, alpha, 1.0, rs.CVAR_RU)
            want = _ru_bruteforce(L, alpha)
            assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (M, L, got, want)


def test_p1_single_and_constant(orc):
    assert orc.cvar([3.5], 0.9) == 3.5
    assert orc.cvar([2.0] * 7, 0.9) == pytest.approx(2.0, abs=1e-14)
    assert orc.cvar([2.0] * 7, 0.9, mode=rs.CVAR_TCE) == 2.0


@pytest.mark.parametrize("B", [0.0, 0.5, 1.0, 2.0, 3.7])
def test_p6_scaling_closed_form(orc, B):
    rng = np.random.default_rng(5)
    for M in (4, 10, 33, 128):
        L = rng.gamma(2.0, size=M) * 10
        for alpha in ALPHAS:
            got = orc.cvar(L, alpha, B, rs.CVAR_RU)
            want = B * orc.cvar(L, alpha, 1.0, rs.CVAR_RU) + (1 - B) * L.mean()
            assert abs(got - want) <= 1e-10 * max(1.0, abs(want))
    if B == 0.0:
        L = rng.normal(size=17)
        assert orc.cvar(L, 0.9, 0.0) == pytest.approx(L.mean(), abs=1e-12)


def test_p7_tail_mean_ordering(orc):
    rng = np.random.default_rng(9)
    for trial in range(300):
        M = int(rng.integers(1, 60))
        L = rng.integers(0, 4, size=M) * 1000.0 if trial % 2 else rng.normal(size=M)
        alpha = ALPHAS[trial % len(ALPHAS)]
        tce = orc.cvar(L, alpha, 1.0, rs.CVAR_TCE)
        ru = orc.cvar(L, alpha, 1.0, rs.CVAR_RU)
        assert tce <= ru + 1e-9 * max(1, abs(ru))
        assert ru <= L.max() + 1e-9 * max(1, abs(ru))
    # alpha M integer, no ties: the fractional tail is the mean of the top
    # (1 - alpha) M order statistics; the literal tail mean over {L >= VaR}
    # also counts VaR = L_(j) itself, i.e. the top M - j + 1 values
    L = rng.normal(size=40)
    a = 0.75
    s = np.sort(L)
    assert orc.cvar(L, a, 1.0, rs.CVAR_RU) == pytest.approx(s[30:].mean(), rel=1e-13)
    assert orc.cvar(L, a, 1.0, rs.CVAR_TCE) == pytest.approx(s[29:].mean(), rel=1e-13)


def test_tce_is_the_literal_tail_mean_with_ties(orc):
    # indicator-style costs: VaR falls on 0, the literal mean includes all zeros
    # (2 hits of 32, alpha M = 28.8, j = 29, VaR = L_(29) = 0)
    L = np.array([0.0] * 30 + [1000.0] * 2)
    alpha = float(np.float32(0.9))
    assert orc.cvar(L, alpha, 1.0, rs.CVAR_TCE) == pytest.approx(2000.0 / 32)
    # the fractional tail takes the (1 - alpha) M = 3.2 worst values
    aM = alpha * 32
    assert orc.cvar(L, alpha, 1.0, rs.CVAR_RU) == pytest.approx(2000.0 / (32 - aM), rel=1e-14)
    # 4 hits: VaR lands on 1000 and both forms give 1000
    L = np.array([0.0] * 28 + [1000.0] * 4)
    assert orc.cvar(L, alpha, 1.0, rs.CVAR_TCE) == 1000.0
    assert orc.cvar(L, alpha, 1.0, rs.CVAR_RU) == pytest.approx(1000.0, rel=1e-14)


def test_non_finite_ranks_worst(orc):
    for bad in (np.nan, np.inf):
        L = np.array([1.0, 2.0, bad, 3.0])
        assert orc.cvar(L, 0.75, 1.0, rs.CVAR_RU) == np.inf
        assert orc.cvar(L, 0.75, 1.0, rs.CVAR_TCE) == np.inf


@pytest.mark.slow
def test_p2_gaussian_closed_form(orc):
    """Linear system x+ = x + u + w, w ~ N(0, s_w^2), risk cost c x on x_0..x_{T-1}:
    L ~ N(mu, s^2), s^2 = c^2 s_w^2 (T-1) T (2T-1) / 6."""
    T, M = 10, 1_000_000
    sw = float(np.float32(0.5))
    alpha = float(np.float32(0.9))
    V = (np.arange(T) * 0.1 - 0.3).astype(np.float32).reshape(T, 1)
    p = rs.preset("linear_test", K=1, M=M, T=T, w_scale=(sw, 0, 0, 0), alpha=alpha)
    x0 = np.array([0.25], dtype=np.float32)
    out = orc.samples(p, x0, V, np.zeros((0, 3), np.float32), ks=[0], n_threads=1)
    c = 1.0
    xs = float(x0[0]) + np.concatenate([[0.0], np.cumsum(V[:, 0].astype(np.float64))])[:T]
    mu = c * xs.sum()
    s = abs(c) * sw * np.sqrt((T - 1) * T * (2 * T - 1) / 6.0)
    z = stats.norm.ppf(alpha)
    want = mu + s * stats.norm.pdf(z) / (1 - alpha)
    # asymptotic standard error of the empirical CVaR: sd((L - VaR)_+) / ((1 - alpha) sqrt(M))
    q = mu + s * z
    zz = (q - mu) / s
    e1 = s * (stats.norm.pdf(zz) - zz * stats.norm.sf(zz))
    e2 = s**2 * ((1 + zz**2) * stats.norm.sf(zz) - zz * stats.norm.pdf(zz))
    se = np.sqrt(e2 - e1**2) / ((1 - alpha) * np.sqrt(M))
    assert abs(out["cvar"][0] - want) < 4 * se, (out["cvar"][0], want, se)
    # the nominal cost is the mean of L (zero-mean noise, linear cost)
    assert abs(out["S"][0] - mu) < 1e-12 * max(1, abs(mu))


@pytest.mark.slow
def test_p2_wrong_index_convention_is_detectable(orc):
    """Charging the risk cost on x_1..x_T instead of x_0..x_{T-1} would change
    the variance to s_w^2 T (T+1)(2T+1)/6; the test above resolves that."""
    T, M = 10, 1_000_000
    sw, alpha = float(np.float32(0.5)), float(np.float32(0.9))
    s_right = sw * np.sqrt((T - 1) * T * (2 * T - 1) / 6.0)
    s_wrong = sw * np.sqrt(T * (T + 1) * (2 * T + 1) / 6.0)
    k = stats.norm.pdf(stats.norm.ppf(alpha)) / (1 - alpha)
    se_bound = 3 * s_right / ((1 - alpha) * np.sqrt(M))
    assert (s_wrong - s_right) * k > 8 * se_bound
