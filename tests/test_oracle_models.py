"""Pins of the oracle's vehicle models, track geometry and costs (CPU only).

P8  kinematic bicycle: straight-line Euler sums; constant steer traces a
    regular polygon (all states equidistant from one centre)
P8' dynamic single-track: straight-line motion is exact for Heun (constant
    acceleration), left/right mirror symmetry, neutral-steer steady yaw rate
P8'' dynamic single-track tyre law, axle loads, mass and yaw inertia from
    the derivative read off the one-period map (peak force, cornering
    stiffness, shape at B alpha = 1, single-axle yaw ratios, vx floor, Heun
    composition, understeer gradient with lf != lr)
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


# ---------------------------------------------------------------------------
# P8'' the dynamic model's tyre-force law, axle loads, mass and yaw inertia.
#
# The derivative f(x, u) of the single-track model is read off the oracle's
# public one-period map by Richardson extrapolation of two tiny Heun steps,
# so nothing below calls or retypes the oracle's derivative.  It is then
# checked against textbook properties of the single-track model with static
# axle loads Fz_f = m g lr / L, Fz_r = m g lf / L and the Magic-Formula
# lateral force D Fz sin(C atan(B alpha)):
#   - the peak force is D Fz, reached at slip tan(pi / (2 C)) / B;
#   - the cornering stiffness (slope at zero slip) is B C D Fz;
#   - at B alpha = 1 the force is D Fz sin(C pi / 4);
#   - pure sideslip of a vehicle with static loads and equal tyres gives no
#     yaw moment, whatever lf and lr (lf Fz_f = lr Fz_r);
#   - a force on one axle only turns the body with r' / a_y = l m / Iz;
#   - the front force acts along the steered wheel: it slows vx by
#     a_y tan(delta);
#   - with equal tyres on both axles the static loads make the vehicle
#     neutral steer, so the linear bicycle's understeer gradient
#     K = m (lr / C_f - lf / C_r) / L is zero for any lf != lr and the steady
#     yaw rate is vx delta / (L + K vx^2) = vx delta / L.
# Body parameters lf = 0.12 m, lr = 0.21 m (unequal on purpose), m = 2.5 kg,
# Iz = 0.02 kg m^2, B = 10, C = 1.5, D = 1, vx floor 0.5 m/s.
# ---------------------------------------------------------------------------
G = 9.81
MP_UNEQUAL = (2.5, 0.02, 0.12, 0.21, 10.0, 1.5, 1.0, 0.5)


def _dyn_problem(orc, mp, dt, substeps=1):
    p = rs.preset("c2_closed_loop", model_params=mp, dt=dt, substeps=substeps)
    return orc.make_problem(p, exact=True)


def _deriv(orc, x, u, mp=MP_UNEQUAL, h=1e-6):
    """f(x, u) from two Heun steps of h and h/2: D(h) = (Phi_h(x) - x) / h =
    f + h/2 J f + O(h^2), so 2 D(h/2) - D(h) = f + O(h^2)."""
    x = np.asarray(x, np.float64)
    d1 = (orc.dynamics(_dyn_problem(orc, mp, h), x, u) - x) / h
    d2 = (orc.dynamics(_dyn_problem(orc, mp, h / 2), x, u) - x) / (h / 2)
    return 2.0 * d2 - d1


def _peak_slip(mp):
    return math.tan(math.pi / (2.0 * mp[5])) / mp[4]


def test_dyn_kinematics_rotate_body_velocity(orc):
    """(x', y') is the body velocity (vx, vy) rotated by the heading; psi' = r."""
    x = np.array([1.0, 2.0, 0.7, 2.0, 0.3, 0.5])
    f = _deriv(orc, x, [0.1, 0.5])
    assert math.hypot(f[0], f[1]) == pytest.approx(math.hypot(2.0, 0.3), rel=1e-7)
    assert math.atan2(f[1], f[0]) == pytest.approx(0.7 + math.atan2(0.3, 2.0), rel=1e-7)
    assert f[2] == pytest.approx(0.5, rel=1e-7)


def test_dyn_pure_sideslip_peak_and_no_yaw(orc):
    """Pure sideslip (delta = 0, r = 0): both axles see alpha = -atan(vy / vx);
    total lateral acceleration D g sin(C atan(B alpha)) peaks at D g exactly at
    alpha* = tan(pi / 2C) / B, and the yaw moment vanishes for lf != lr."""
    mp = MP_UNEQUAL
    vx = 2.0
    a_star = _peak_slip(mp)
    x = np.array([0.0, 0.0, 0.0, vx, vx * math.tan(a_star), 0.0])
    f = _deriv(orc, x, [0.0, 0.0])
    assert f[4] == pytest.approx(-mp[6] * G, rel=1e-6)  # peak lateral force D (Fz_f + Fz_r) / m
    assert abs(f[5]) < 1e-6 * (mp[2] * mp[0] * G / mp[1])  # no yaw moment
    assert abs(f[3]) < 1e-6  # vx' = r vy = 0
    for s in (0.9, 1.1):  # it is a maximum
        xs = x.copy()
        xs[4] = vx * math.tan(s * a_star)
        assert abs(_deriv(orc, xs, [0.0, 0.0])[4]) < mp[6] * G * (1 - 1e-4)


def test_dyn_cornering_stiffness_and_shape(orc):
    """Slope at zero slip B C D g (per unit load); D g sin(C pi/4) at B alpha = 1."""
    mp = MP_UNEQUAL
    vx = 2.0
    alpha = 1e-5
    x = np.array([0.0, 0.0, 0.0, vx, -vx * math.tan(alpha), 0.0])
    f = _deriv(orc, x, [0.0, 0.0])
    assert f[4] / alpha == pytest.approx(mp[4] * mp[5] * mp[6] * G, rel=1e-6)
    alpha = 1.0 / mp[4]
    x[4] = -vx * math.tan(alpha)
    f = _deriv(orc, x, [0.0, 0.0])
    assert f[4] == pytest.approx(mp[6] * G * math.sin(mp[5] * math.pi / 4), rel=1e-6)


def test_dyn_front_axle_force_load_and_inertia(orc):
    """Steer only (vy = r = 0): the rear tyre has no slip, so the front force
    alone accelerates the body.  At alpha_f = delta = alpha* it is the front
    axle's peak D m g lr / L; r' / vy' = lf m / Iz; vx' = a - vy' tan(delta)."""
    mp = MP_UNEQUAL
    m, Iz, lf, lr = mp[:4]
    delta = _peak_slip(mp)
    a = 0.7
    f = _deriv(orc, [0.0, 0.0, 0.0, 2.0, 0.0, 0.0], [delta, a])
    assert f[4] == pytest.approx(mp[6] * G * lr / (lf + lr) * math.cos(delta), rel=1e-6)
    assert f[5] / f[4] == pytest.approx(lf * m / Iz, rel=1e-6)
    assert f[3] == pytest.approx(a - f[4] * math.tan(delta), rel=1e-6)


def test_dyn_rear_axle_force_load_and_inertia(orc):
    """vy = -lf r, delta = 0: the front tyre has no slip; the rear slip is
    atan(L r / vx).  At alpha_r = alpha* the rear force is the rear axle's
    peak D m g lf / L; r' / (vy' + r vx) = -lr m / Iz; vx' = r vy."""
    mp = MP_UNEQUAL
    m, Iz, lf, lr = mp[:4]
    vx = 2.0
    r = vx * math.tan(_peak_slip(mp)) / (lf + lr)
    x = np.array([0.0, 0.0, 0.0, vx, -lf * r, r])
    f = _deriv(orc, x, [0.0, 0.0])
    ay = f[4] + r * vx  # lateral force over mass
    assert ay == pytest.approx(mp[6] * G * lf / (lf + lr), rel=1e-6)
    assert f[5] / ay == pytest.approx(-lr * m / Iz, rel=1e-6)
    assert f[3] == pytest.approx(r * (-lf * r), rel=1e-6)


def test_dyn_slip_uses_vx_floor(orc):
    """Below the floor the slip angles use the floor speed: the lateral
    acceleration of a slow pure sideslip does not depend on vx there."""
    ys = [_deriv(orc, [0.0, 0.0, 0.0, vx, 0.05, 0.0], [0.0, 0.0])[4] for vx in (0.1, 0.3, 0.5)]
    np.testing.assert_allclose(ys, ys[0], rtol=1e-7)
    above = _deriv(orc, [0.0, 0.0, 0.0, 0.8, 0.05, 0.0], [0.0, 0.0])[4]
    assert abs(above) < abs(ys[0]) * 0.9  # a smaller slip above the floor


def test_dyn_heun_composition(orc):
    """One control period with one sub-step is Heun's explicit trapezoid
    x + h/2 (f(x) + f(x + h f(x))) of the model's derivative (read off the
    oracle itself by tiny steps)."""
    x = np.array([0.5, -3.0, 0.4, 2.5, 0.2, -0.8])
    u = [0.15, 1.0]
    h = 0.004
    f1 = _deriv(orc, x, u)
    f2 = _deriv(orc, x + h * f1, u)
    want = x + 0.5 * h * (f1 + f2)
    got = orc.dynamics(_dyn_problem(orc, MP_UNEQUAL, h), x, u)
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-9)


def test_dyn_understeer_steady_state_unequal_axles(orc):
    """Linear bicycle with lf != lr, equal tyres and static loads: cornering
    stiffnesses C_f,r = B C D Fz_f,r give the understeer gradient
    K = m (lr / C_f - lf / C_r) / L = 0, so the steady yaw rate at small steer
    is vx delta / (L + K vx^2) = vx delta / L."""
    mp = MP_UNEQUAL
    m, Iz, lf, lr, Bt, Ct, Dt = mp[:7]
    L = lf + lr
    Cf = Bt * Ct * Dt * m * G * lr / L
    Cr = Bt * Ct * Dt * m * G * lf / L
    K = m * (lr / Cf - lf / Cr) / L
    pr = _dyn_problem(orc, mp, 0.02, substeps=6)
    delta = 0.02
    x = np.array([0.0, 0.0, 0.0, 2.5, 0.0, 0.0])
    for _ in range(150):
        x = orc.dynamics(pr, x, [delta, 0.0])
    vx = x[3]
    assert x[5] == pytest.approx(vx * delta / (L + K * vx * vx), rel=0.01)
