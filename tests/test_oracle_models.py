"""Pins of the oracle's vehicle models, track geometry and costs (CPU only).

P8  kinematic bicycle: straight-line Euler sums; constant steer traces a
    regular polygon (all states equidistant from one centre)
P8' dynamic single-track: straight-line motion is exact for Heun (constant
    acceleration), left/right mirror symmetry, neutral-steer steady yaw rate
P9  stadium track: lateral deviation, arc length and boundary distance at
    hand-computed points
"""

import math

import numpy as np
import pytest

import ra_scenes as rs


def _prob(orc, name, **kw):
    return orc.make_problem(rs.preset(name, **kw))


def test_p8_kinematic_straight(orc):
    pr = _prob(orc, "c1_plain")
    dt = float(np.float32(0.05))
    a = 1.5
    x = np.array([1.0, -4.0, 0.0, 0.5])
    xs = [x]
    for t in range(12):
        x = orc.dynamics(pr, x, [0.0, a])
        xs.append(x)
    xs = np.array(xs)
    v = 0.5 + a * dt * np.arange(13)
    np.testing.assert_allclose(xs[:, 3], v, rtol=1e-14)
    np.testing.assert_allclose(xs[:, 0], 1.0 + dt * np.concatenate([[0], np.cumsum(v[:-1])]), rtol=1e-14)
    np.testing.assert_allclose(xs[:, 1], -4.0, atol=0)
    np.testing.assert_allclose(xs[:, 2], 0.0, atol=0)


def test_p8_kinematic_polygon(orc):
    pr = _prob(orc, "c1_plain")
    dt = float(np.float32(0.05))
    Lw = float(np.float32(0.33))
    delta, v = 0.3, 2.0
    x = np.array([0.0, 0.0, 0.0, v])
    pts = [x[:2]]
    for t in range(40):
        x = orc.dynamics(pr, x, [delta, 0.0])
        pts.append(x[:2])
    pts = np.array(pts)
    dpsi = v * dt * math.tan(delta) / Lw
    assert x[2] == pytest.approx(40 * dpsi, rel=1e-13)
    # vertices of a regular polygon with edge v dt and turn dpsi lie on a circle
    R = (v * dt / 2) / math.sin(dpsi / 2)
    # centre: perpendicular bisector of the first edge, rotated by dpsi/2
    c = np.array([v * dt / 2, (v * dt / 2) / math.tan(dpsi / 2)])
    np.testing.assert_allclose(np.hypot(*(pts - c).T), R, rtol=1e-11)


def test_p8_dynamic_straight_is_exact(orc):
    pr = _prob(orc, "c2_closed_loop")
    dt = float(np.float32(0.02))
    a = 2.0
    x = np.array([0.0, -4.0, 0.0, 1.2, 0.0, 0.0])
    for t in range(25):
        x = orc.dynamics(pr, x, [0.0, a])
    T = 25 * dt
    assert x[3] == pytest.approx(1.2 + a * T, rel=1e-13)
    assert x[0] == pytest.approx(1.2 * T + 0.5 * a * T * T, rel=1e-12)
    assert x[1] == -4.0 and x[2] == 0.0 and x[4] == 0.0 and x[5] == 0.0


def test_p8_dynamic_mirror_symmetry(orc):
    pr = _prob(orc, "c2_closed_loop")
    xa = np.array([0.0, 0.0, 0.0, 2.0, 0.0, 0.0])
    xb = xa.copy()
    for t in range(30):
        d = 0.25 * math.sin(0.3 * t)
        xa = orc.dynamics(pr, xa, [d, 0.5])
        xb = orc.dynamics(pr, xb, [-d, 0.5])
    flip = np.array([1, -1, -1, 1, -1, -1])
    np.testing.assert_allclose(xa, flip * xb, atol=1e-12)


def test_p8_dynamic_neutral_steer_yaw_rate(orc):
    """Equal axle loads and tyres (lf = lr): neutral steer, so at small slip
    the steady yaw rate is vx delta / (lf + lr)."""
    pr = _prob(orc, "c2_closed_loop")
    delta = 0.02
    x = np.array([0.0, 0.0, 0.0, 2.0, 0.0, 0.0])
    for t in range(150):
        x = orc.dynamics(pr, x, [delta, 0.0])
    vx = x[3]
    r_ss = vx * delta / 0.33
    assert x[5] == pytest.approx(r_ss, rel=0.03)


@pytest.mark.parametrize("px,py,e,s,d", [
    (0.0, -4.0, 0.0, 0.0, 1.0),                      # start of the lap
    (2.0, -4.5, 0.5, 2.0, 0.5),                      # bottom straight, outside
    (-2.0, -3.7, -0.3, 2 * 10 + 2 * math.pi * 4 - 2.0, 0.7),  # bottom straight, left half
    (0.0, 4.2, 0.2, 5 + 4 * math.pi + 5, 0.8),       # top straight midpoint
    (9.0, 0.0, 0.0, 5 + 2 * math.pi, 1.0),           # right arc apex
    (5.0 + 3.0 / math.sqrt(2), 3.0 / math.sqrt(2), -1.0, 5 + 4 * 3 * math.pi / 4, 0.0),
    (-9.5, 0.0, 0.5, 5 + 4 * math.pi + 10 + 2 * math.pi, 0.5),  # left arc apex
    (5.0, 4.0, 0.0, 5 + 4 * math.pi, 1.0),           # right-arc / top junction
])
def test_p9_track_geometry(orc, px, py, e, s, d):
    pr = _prob(orc, "c1_plain")
    got = orc.track(pr, px, py)
    np.testing.assert_allclose(got, [e, s, d], atol=1e-12)


def test_costs_at_hand_points(orc):
    p = rs.preset("c1_plain", w_bdry=2.0, c4=0.6, c5=2.0)
    pr = orc.make_problem(p)
    obs = np.array([[1.0, -4.0, 0.3], [1.2, -4.0, 0.3]], dtype=np.float32)
    x = np.array([1.1, -4.5, 0.0, 3.0])
    # deviation 0.5^2, speed (3-4)^2, both obstacles at distance
    # hypot(0.1, 0.5) = 0.51 > 0.3: no hit; boundary: d = 0.5
    want = 0.25 + 1.0 + 0.0 + 2.0 * (math.atan(-50.0) / math.pi + 0.5)
    assert orc.state_cost(pr, x, obs, 0xFF) == pytest.approx(want, rel=1e-12)
    x2 = np.array([1.1, -4.1, 0.0, 3.0])  # inside both circles
    want2 = 0.01 + 1.0 + 2000.0 + 2.0 * (math.atan(-90.0) / math.pi + 0.5)
    assert orc.state_cost(pr, x2, obs, 0xFF) == pytest.approx(want2, rel=1e-12)
    assert orc.state_cost(pr, x2, obs, rs.RISK_OBS) == 2000.0
    assert orc.terminal_cost(pr, x) == pytest.approx(float(np.float32(0.6)) - 2.0 * 1.1, rel=1e-12)


def test_softplus_barrier(orc):
    p = rs.preset("c4_gradient")
    pr = orc.make_problem(p)
    obs = np.array([[0.0, 0.0, 0.3]], dtype=np.float32)
    r = float(np.float32(0.3))
    for dist in (0.0, 0.2, 0.3, 0.5, 2.0):
        x = np.array([dist, 0.0, 0.0, 0.0])
        z = 20.0 * (r - dist)
        want = 1000.0 * math.log1p(math.exp(z)) / 20.0
        assert orc.state_cost(pr, x, obs, rs.RISK_OBS) == pytest.approx(want, rel=1e-12)
