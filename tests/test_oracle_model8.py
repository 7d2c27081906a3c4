"""Pins of the oracle's single-track model with wheel speeds and combined slip (model 2, 8 states).

Each test checks the model against a fact that does not come from its own code: the free-rolling
equilibrium, mirror symmetry, the wheel-torque balance (true for any tyre law), the friction-ellipse
bound, and the reduction to the separately pinned 6-state bicycle when both wheels roll freely.
Derivatives are read from one explicit-Euler step (n_sub = 1): (x_next - x) / dt.
"""
import numpy as np
import pytest

import oracle
import workload


def _prob(kappa=0.0, **kw):
    p = workload.wheels_problem(1, 2, 1)
    p.kappa = np.full(16, kappa, np.float32)
    p.track_len = 100.0
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _f32(x):
    return float(np.float32(x))


def _deriv(o, p, x, u):
    return (o.model_step(np.asarray(x, float), np.asarray(u, float)) - np.asarray(x, float)) / _f32(p.dt)


def test_free_rolling_equilibrium():
    """Straight track, no steer, no torque, no lateral motion and wheels at v/R: no force acts, so
    the state only advances along the track, s += v dt."""
    p = _prob()
    o = oracle.Oracle(p)
    R = _f32(p.wheel_radius)
    x = np.array([6.0, 0.0, 0.0, 6.0 / R, 6.0 / R, 0.0, 0.3, 10.0])
    xn = o.model_step(x, np.array([0.0, 0.0]))
    expect = x.copy()
    expect[7] += 6.0 * _f32(p.dt)
    np.testing.assert_allclose(xn, expect, rtol=1e-14, atol=1e-12)


def test_mirror_symmetry():
    """Reflecting the road (steer, v_y, r, e_psi, e_y and the curvature change sign) reflects the motion."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        x = np.array([rng.uniform(3, 8), rng.normal(0, 0.5), rng.normal(0, 0.5), rng.uniform(20, 90),
                      rng.uniform(20, 90), rng.normal(0, 0.2), rng.normal(0, 0.5), rng.uniform(0, 50)])
        u = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-1, 1)])
        k = rng.uniform(-0.05, 0.05)
        a = oracle.Oracle(_prob(k)).model_step(x, u)
        flip = np.array([1, -1, -1, 1, 1, -1, -1, 1.0])
        b = oracle.Oracle(_prob(-k)).model_step(x * flip, u * np.array([-1, 1.0]))
        np.testing.assert_allclose(b, a * flip, rtol=1e-12, atol=1e-12)


def test_wheel_torque_balance():
    """Going straight without yaw or side slip, m v_x' = F_xf + F_xr and I_w omega' = -R F_x (+ the
    drive torque at the rear) give m R v_x' + I_w (omega_F' + omega_R') = tau_max throttle, whatever
    the tyre law and however much the wheels slip."""
    p = _prob(n_sub=1, dt=1e-3)
    o = oracle.Oracle(p)
    rng = np.random.default_rng(4)
    m, R, Iw, tau = (_f32(p.mass), _f32(p.wheel_radius), _f32(p.wheel_inertia), _f32(p.tau_max))
    for _ in range(50):
        vx = rng.uniform(0.5, 9.0)
        x = np.array([vx, 0.0, 0.0, rng.uniform(0, 120), rng.uniform(0, 120), 0.0, 0.0, 5.0])
        thr = rng.uniform(-1, 1)
        d = _deriv(o, p, x, [0.0, thr])
        lhs = m * R * d[0] + Iw * (d[3] + d[4])
        assert abs(lhs - tau * thr) < 1e-9 * max(1.0, abs(tau * thr)), (lhs, tau * thr)


def test_forces_stay_inside_the_friction_ellipse():
    """With no steer the tyre forces follow from the derivatives: F_xf = -I_w omega_F' / R,
    F_xr = (tau - I_w omega_R') / R, and (F_yf, F_yr) from m (v_y' + v_x r) = F_yf + F_yr,
    I_z r' = l_f F_yf - l_r F_yr. Every wheel's (F_x / mu_x F_z)^2 + (F_y / mu F_z)^2 stays <= 1 and
    approaches 1 once the combined slip saturates the tyre."""
    p = _prob(n_sub=1, dt=1e-4)
    o = oracle.Oracle(p)
    rng = np.random.default_rng(5)
    m, Iz, lf, lr = _f32(p.mass), _f32(p.Iz), _f32(p.lf), _f32(p.lr)
    R, Iw, tau = _f32(p.wheel_radius), _f32(p.wheel_inertia), _f32(p.tau_max)
    g, mux, muy = _f32(p.g), _f32(p.mu_x), _f32(p.mu)
    Fz = np.array([m * g * lr / (lf + lr), m * g * lf / (lf + lr)])
    worst = 0.0
    for _ in range(200):
        vx = rng.uniform(2.0, 9.0)
        x = np.array([vx, rng.normal(0, 1.0), rng.normal(0, 1.0), rng.uniform(0, 150), rng.uniform(0, 150),
                      0.0, 0.0, 5.0])
        thr = rng.uniform(-1, 1)
        d = _deriv(o, p, x, [0.0, thr])
        Fx = np.array([-Iw * d[3] / R, (tau * thr - Iw * d[4]) / R])
        A = np.array([[1.0, 1.0], [lf, -lr]])
        Fy = np.linalg.solve(A, np.array([m * (d[1] + x[0] * x[2]), Iz * d[2]]))
        e = (Fx / (mux * Fz)) ** 2 + (Fy / (muy * Fz)) ** 2
        assert np.all(e <= 1.0 + 1e-7), e
        worst = max(worst, e.max())
    assert worst > 0.95  # large slips reach the ellipse


@pytest.mark.parametrize("steer", [0.0, 0.2, -0.3])
def test_free_rolling_wheels_reduce_to_the_bicycle_model(steer):
    """With both wheels rolling freely (zero longitudinal slip) and no torque, the combined-slip tyre
    gives the bicycle model's lateral force mu F_z sin(C atan(B alpha)) and no longitudinal force: the
    derivatives of (v_x, v_y, r, e_psi, e_y, s) equal the 6-state model's with zero acceleration."""
    p8 = _prob(0.02, n_sub=1, dt=1e-3)
    p6 = workload.config0()
    for name in ("mass", "Iz", "lf", "lr", "tire_B", "tire_C", "mu", "g", "vx_floor", "dt", "n_sub"):
        setattr(p6, name, getattr(p8, name))
    p6.kappa, p6.track_len = p8.kappa, p8.track_len
    o8, o6 = oracle.Oracle(p8), oracle.Oracle(p6)
    rng = np.random.default_rng(6)
    R = _f32(p8.wheel_radius)
    lf = _f32(p8.lf)
    st = _f32(steer)
    for _ in range(20):
        vx, vy, r = rng.uniform(3, 8), rng.normal(0, 0.4), rng.normal(0, 0.4)
        ep, ey, s = rng.normal(0, 0.2), rng.normal(0, 0.5), rng.uniform(0, 50)
        wf = (vx * np.cos(st) + (vy + lf * r) * np.sin(st)) / R
        d8 = _deriv(o8, p8, [vx, vy, r, wf, vx / R, ep, ey, s], [st, 0.0])
        d6 = _deriv(o6, p6, [vx, vy, r, ep, ey, s], [st, 0.0])
        np.testing.assert_allclose(d8[[0, 1, 2, 5, 6, 7]], d6, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("steer", [0.25, -0.15])
def test_pure_longitudinal_slip_in_a_kinematic_turn(steer):
    """No side slip on either axle (v_y + l_f r = v_x tan(steer), v_y = l_r r) and a free-rolling rear
    wheel: only the front wheel's longitudinal slip kappa = (R omega_F - v_F) / v_F acts, with
    v_F = v_x / cos(steer) its forward speed, so F_xf = mu_x F_zf sin(C atan(B kappa)) (the pure-slip
    magic formula), and v_x' = F_xf cos(steer) / m + v_y r, v_y' = F_xf sin(steer) / m - v_x r,
    r' = l_f F_xf sin(steer) / I_z, omega_F' = -R F_xf / I_w, omega_R' = 0."""
    p = _prob(n_sub=1, dt=1e-5)
    o = oracle.Oracle(p)
    m, Iz, lf, lr = _f32(p.mass), _f32(p.Iz), _f32(p.lf), _f32(p.lr)
    R, Iw, g = _f32(p.wheel_radius), _f32(p.wheel_inertia), _f32(p.g)
    B, C, mux = _f32(p.tire_B), _f32(p.tire_C), _f32(p.mu_x)
    st = _f32(steer)
    Fzf = m * g * lr / (lf + lr)
    for kappa in (-0.3, -0.02, 0.01, 0.15, 0.6):
        vx = 5.0
        r = vx * np.tan(st) / (lf + lr)
        vy = lr * r
        vF = vx / np.cos(st)
        x = [vx, vy, r, vF * (1 + kappa) / R, vx / R, 0.0, 0.0, 5.0]
        d = _deriv(o, p, x, [st, 0.0])
        F = mux * Fzf * np.sin(C * np.arctan(B * kappa))
        expect = [F * np.cos(st) / m + vy * r, F * np.sin(st) / m - vx * r, lf * F * np.sin(st) / Iz,
                  -R * F / Iw, 0.0]
        np.testing.assert_allclose(d[:5], expect, rtol=1e-6, atol=1e-6 * max(1.0, abs(F)))


def test_combined_slip_follows_the_magic_formula_at_the_slip_magnitude():
    """Defining law of the combined-slip tyre: the force points along the (kappa, alpha) slip vector,
    scaled by the friction ellipse's axes, and its normalised size equals the pure-slip curve at the
    combined slip: (F_x / mu_x F_z)^2 + (F_y / mu F_z)^2 = sin^2(C atan(B sqrt(kappa^2 + alpha^2))).
    Forces are read from the derivatives (no steer, both axles slipping both ways)."""
    p = _prob(n_sub=1, dt=1e-5)
    o = oracle.Oracle(p)
    m, Iz, lf, lr = _f32(p.mass), _f32(p.Iz), _f32(p.lf), _f32(p.lr)
    R, Iw, tau, g = _f32(p.wheel_radius), _f32(p.wheel_inertia), _f32(p.tau_max), _f32(p.g)
    B, C, mux, muy = _f32(p.tire_B), _f32(p.tire_C), _f32(p.mu_x), _f32(p.mu)
    Fz = np.array([m * g * lr / (lf + lr), m * g * lf / (lf + lr)])
    rng = np.random.default_rng(7)
    for _ in range(100):
        vx, vy, r = rng.uniform(3, 8), rng.normal(0, 0.5), rng.normal(0, 0.5)
        wf, wr = vx / R * (1 + rng.normal(0, 0.1)), vx / R * (1 + rng.normal(0, 0.1))
        d = _deriv(o, p, [vx, vy, r, wf, wr, 0.0, 0.0, 5.0], [0.0, 0.0])
        Fx = np.array([-Iw * d[3] / R, -Iw * d[4] / R])
        Fy = np.linalg.solve(np.array([[1.0, 1.0], [lf, -lr]]), np.array([m * (d[1] + vx * r), Iz * d[2]]))
        kap = np.array([(R * wf - vx) / vx, (R * wr - vx) / vx])
        alp = np.array([-np.arctan((vy + lf * r) / vx), -np.arctan((vy - lr * r) / vx)])
        sl = np.hypot(kap, alp)
        np.testing.assert_allclose((Fx / (mux * Fz)) ** 2 + (Fy / (muy * Fz)) ** 2,
                                   np.sin(C * np.arctan(B * sl)) ** 2, rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(Fx / (mux * Fz) * alp, Fy / (muy * Fz) * kap, rtol=1e-6, atol=1e-9)
