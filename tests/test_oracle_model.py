"""Pins of the oracle's vehicle model, track lookup and back-off coefficient (CPU only).

The model is the dynamic single-track vehicle in the road-aligned frame (Sec. V-A uses a planar
single-track model); each check below is a closed form or a symmetry that holds independently of
the code under test.
"""
import math
import os

import numpy as np
import pytest
from scipy import special

import oracle
import workload


def _straight(prob):
    prob.kappa = np.zeros(64, np.float32)
    prob.track_len = 100.0
    return prob


def test_backoff_matches_normal_quantiles():
    path = os.path.join(os.path.dirname(__file__), "golden", "normal_quantiles.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for delta, nu in rows:
        assert oracle.backoff_gaussian(float(delta)) == pytest.approx(float(nu), rel=1e-14)
        assert oracle.backoff_gaussian(float(delta)) == pytest.approx(special.ndtri(1 - float(delta)), rel=1e-13)
    assert oracle.backoff_cantelli(0.05) == pytest.approx(math.sqrt(19.0), rel=1e-15)


def test_pure_longitudinal_motion_closed_form():
    """Straight track, zero steer, no lateral motion: v_x(t) = v0 + a t exactly and the Euler
    recurrence s_{j+1} = s_j + h v_x,j gives s = s0 + dt v0 + a h^2 n (n - 1) / 2."""
    p = _straight(workload.config0())
    o = oracle.Oracle(p)
    v0, a, s0 = 8.0, 1.5, 3.0
    x = np.array([v0, 0, 0, 0, 0, s0], float)
    xn = o.model_step(x, np.array([0.0, a]))
    dt = float(np.float32(p.dt))
    n = p.n_sub
    h = dt / n
    assert xn[0] == pytest.approx(v0 + a * dt, rel=1e-14)
    assert xn[5] == pytest.approx(s0 + dt * v0 + a * h * h * n * (n - 1) / 2, rel=1e-14)
    assert np.all(xn[1:5] == 0.0)


def test_mirror_symmetry_on_straight_track():
    """Reflecting the lateral axis (v_y, r, e_psi, e_y, steer -> negatives) reflects the step."""
    p = _straight(workload.config0())
    o = oracle.Oracle(p)
    rng = np.random.default_rng(0)
    mirror = np.array([1, -1, -1, -1, -1, 1], float)
    for _ in range(20):
        x = np.array([rng.uniform(2, 15), rng.normal(0, .5), rng.normal(0, .3), rng.normal(0, .1),
                      rng.normal(0, 1), rng.uniform(0, 50)])
        u = np.array([rng.uniform(-.4, .4), rng.uniform(-3, 3)])
        a = o.model_step(x, u)
        b = o.model_step(x * mirror, u * np.array([-1, 1]))
        np.testing.assert_allclose(b, a * mirror, rtol=1e-13, atol=1e-13)


def test_linear_tyre_regime_matches_linear_bicycle():
    """Small steer from straight driving: with one Euler substep the lateral accelerations equal
    the textbook linear single-track model with cornering stiffness C_a = mu F_z B C."""
    p = _straight(workload.config0())
    p.n_sub = 1
    o = oracle.Oracle(p)
    f = lambda x: float(np.float32(x))
    m, Iz, lf, lr, g = f(p.mass), f(p.Iz), f(p.lf), f(p.lr), f(p.g)
    Caf = f(p.mu) * m * g * lr / (lf + lr) * f(p.tire_B) * f(p.tire_C)
    dt = f(p.dt)
    vx, d = 10.0, 1e-5
    xn = o.model_step(np.array([vx, 0, 0, 0, 0, 0.0]), np.array([d, 0.0]))
    ay = (xn[1] - 0.0) / dt
    rdot = xn[2] / dt
    assert ay == pytest.approx(Caf * d / m, rel=1e-6)
    assert rdot == pytest.approx(lf * Caf * d / Iz, rel=1e-6)


def test_constant_curvature_path_following():
    """On a circle (kappa = 1/R), centred with matching yaw rate r = v_x kappa and no heading or
    lateral error, the path-frame rates are s' = v_x, e_psi' = 0 and e_y' = 0 (first substep)."""
    p = workload.config0()
    R = 50.0
    p.kappa = np.full(32, 1.0 / R, np.float32)
    p.n_sub = 1
    p.dt = 1e-3
    o = oracle.Oracle(p)
    kap = float(np.float32(1.0 / R))
    vx = 10.0
    xn = o.model_step(np.array([vx, 0.0, vx * kap, 0.0, 0.0, 0.0]), np.array([0.0, 0.0]))
    dt = float(np.float32(1e-3))
    assert xn[5] == pytest.approx(dt * vx, rel=1e-14)
    assert abs(xn[3]) < 1e-15
    assert xn[4] == 0.0


def test_track_lookup_interpolates_and_wraps():
    p = workload.config0()
    o = oracle.Oracle(p)
    kap = p.kappa.astype(float)
    n, L = kap.size, float(np.float32(p.track_len))
    for i in (0, 1, 100, n - 1):
        assert o.kappa_at(i * L / n) == pytest.approx(kap[i], abs=1e-12)
        mid = o.kappa_at((i + 0.5) * L / n)
        assert mid == pytest.approx(0.5 * (kap[i] + kap[(i + 1) % n]), abs=1e-12)
        assert o.kappa_at(i * L / n + L) == pytest.approx(kap[i], abs=1e-12)
        assert o.kappa_at(i * L / n - L) == pytest.approx(kap[i], abs=1e-12)


def test_track_generator_geometry():
    """The tabulated curvature of a closed simple curve integrates to one full turn."""
    for seed in (0, 1, 7):
        kappa, L = workload.make_track(seed)
        assert 2 * math.pi * 54 < L < 2 * math.pi * 66 + 10
        total_turn = kappa.astype(float).sum() * L / kappa.size
        assert total_turn == pytest.approx(2 * math.pi, rel=1e-4)


def test_double_integrator_step_closed_form():
    p = workload.double_integrator_problem(1, 2, 1)
    o = oracle.Oracle(p)
    dt = float(np.float32(p.dt))
    x = np.array([1.0, -2.0, 0.5, 0.25])
    u = np.array([0.3, -0.7])
    A = np.block([[np.eye(2), dt * np.eye(2)], [np.zeros((2, 2)), np.eye(2)]])
    B = np.vstack([0.5 * dt * dt * np.eye(2), dt * np.eye(2)])
    np.testing.assert_allclose(o.model_step(x, u), A @ x + B @ u, rtol=1e-15, atol=1e-15)
