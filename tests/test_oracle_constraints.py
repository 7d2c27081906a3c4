"""Pins of the oracle's general constraint set (Assumption 1, Eq. "deterministic_chance_constraint",
Eq. "DCBFchoice0", Eq. "DCBFchoice", Remark 1).

Each test checks the oracle against something other than itself: linear-Gaussian closed-form moments
with scipy's erfinv for the back-off, an exact zero-spread case with the collision indicator, the
algebraic tie to the (separately pinned) racing barrier, and Cantelli's distribution-free bound
checked on the particles themselves.
"""
import math

import numpy as np
import pytest
from scipy.special import erfinv

import oracle
import workload
from tests.test_oracle_resample import _xi
from tests.test_oracle_solve import CORRELATED_W, _di_mats


def _nu(c):
    p = float(np.float32(c["p"]))
    if c.get("backoff", "gaussian") == "gaussian":
        return math.sqrt(2.0) * float(erfinv(1.0 - 2.0 * p))
    return math.sqrt((1.0 - p) / p)


def _c_and_eta(c, x):
    """c(x) and grad c(x) written from the constraint's definition."""
    x = np.asarray(x, float)
    if c["kind"] == "halfspace":
        a = np.zeros(x.size)
        a[: len(c["a"])] = np.float32(c["a"])
        return float(a @ x - np.float32(c["b"])), a
    i, j = c["i"], c["j"]
    o = np.float32(c["center"]).astype(float)
    r = float(np.float32(c["radius"]))
    eta = np.zeros(x.size)
    eta[i], eta[j] = -2.0 * (x[i] - o[0]), -2.0 * (x[j] - o[1])
    return r * r - (x[i] - o[0]) ** 2 - (x[j] - o[1]) ** 2, eta


def _quiet_di(K, M, T, q_w):
    p = workload.double_integrator_problem(K=K, M=M, T=T, q_w=q_w)
    p.Sigma_eps = np.diag([1e-30, 1e-30])  # u = v exactly
    return p


CONS = (workload.halfspace((0, 1, 0, 0), 1.5, 0.05),
        workload.halfspace((1 / math.sqrt(2), 1 / math.sqrt(2), 0, 0), 2.0, 0.1, backoff="cantelli"),
        workload.disk(0, 1, (1.0, -0.5), 0.4, 0.02))


def test_general_barrier_matches_linear_gaussian_closed_form():
    """Closed-form mean and covariance of the double integrator; h_t = min_i -c_i(m_t) - nu_i
    sqrt(eta_i^T C_t eta_i) from them must match the oracle within Monte-Carlo error."""
    p = _quiet_di(1, 40000, 8, 0.01)
    p.Sigma_w = CORRELATED_W
    p.constraints = CONS
    x0 = np.array([0.2, 0.3, 1.0, -0.4], np.float32)
    Sig0 = np.diag([0.02, 0.03, 0.01, 0.01]).astype(np.float32)
    Sig0[0, 1] = Sig0[1, 0] = 0.015  # the disk's plane is correlated: the cross term of eta^T C eta counts
    v = workload.random_nominal(p, 8, scale=(1.0, 1.0))
    r = oracle.Oracle(p).solve(x0, v, ctr=4, Sigma0=Sig0, want_cov=True)
    A, B = _di_mats(float(np.float32(p.dt)))
    m, C = x0.astype(float), Sig0.astype(float)
    M = p.M
    for t in range(p.T + 1):
        if t > 0:
            m = A @ m + B @ v[t - 1].astype(float)
            C = A @ C @ A.T + CORRELATED_W
        hs, tol = [], 0.0
        for c in CONS:
            cv, eta = _c_and_eta(c, m)
            q = float(eta @ C @ eta)
            hs.append(-cv - _nu(c) * math.sqrt(q))
            lam = float(np.linalg.eigvalsh(C).max())
            tol = max(tol, 6.0 * (np.linalg.norm(eta) * math.sqrt(lam / M) + _nu(c) * math.sqrt(q / (2 * (M - 1))))
                      + 8.0 * lam / M)  # the disk's curvature adds (x - m)^2-order terms
        if t == 0:  # step 0 is evaluated on the given estimate, exactly
            assert abs(r["h"][0, 0] - min(hs)) < 1e-12
        else:
            assert abs(r["h"][0, t] - min(hs)) < tol, (t, r["h"][0, t], min(hs), tol)


def test_zero_spread_barrier_and_indicator_closed_form():
    """No disturbance and a known state: the covariance vanishes, h_t = min_i -c_i(x_t) exactly on
    the deterministic trajectory, and C_obs is charged at exactly the steps whose mean breaks a
    constraint (the trajectory crosses the disk)."""
    p = _quiet_di(1, 4, 12, 0.0)
    cons = (workload.disk(0, 1, (0.6, 0.0), 0.25, 0.05), workload.halfspace((0, 1, 0, 0), 3.0, 0.05))
    p.constraints = cons
    x0 = np.array([0.0, 0.05, 1.0, 0.0], np.float32)
    v = np.zeros((p.T, 2), np.float32)
    A, B = _di_mats(float(np.float32(p.dt)))
    xs = [x0.astype(float)]
    for t in range(p.T):
        xs.append(A @ xs[-1] + B @ v[t])
    h_ref = [min(-_c_and_eta(c, x)[0] for c in cons) for x in xs]
    costs = []
    for c_obs in (0.0, 1000.0):
        p.C_obs = c_obs
        r = oracle.Oracle(p).solve(x0, v, ctr=1, want_cov=True)
        np.testing.assert_allclose(r["h"][0], h_ref, rtol=0, atol=1e-12)
        costs.append(r["S"][0])
    broken = sum(1 for x in xs if any(_c_and_eta(c, x)[0] > 0 for c in cons))
    assert broken >= 3
    assert abs((costs[1] - costs[0]) - 1000.0 * broken) < 1e-6


def test_general_set_on_track_edges_ties_to_racing_barrier():
    """The racing barrier h_r = (w_T - nu sigma)^2 - e^2 and the general set {e - w_T < 0,
    -e - w_T < 0} with the same Gaussian nu satisfy h_r = h_g (h_g + 2 |e|) step by step; the
    particles (and so the moments) do not depend on the barrier."""
    p = workload.config0()
    p.K, p.M, p.T = 6, 12, 15
    x0, v = workload.random_state(p, 3), workload.random_nominal(p, 3)
    x0[4], x0[3] = 2.75, 0.1  # drifting out through the wall: h changes sign
    r_race = oracle.Oracle(p).solve(x0, v, ctr=6, want_cov=True)
    wT = float(np.float32(p.w_T))
    p.constraints = (workload.halfspace((0, 0, 0, 0, 1, 0), wT, p.delta),
                     workload.halfspace((0, 0, 0, 0, -1, 0), wT, p.delta))
    r_gen = oracle.Oracle(p).solve(x0, v, ctr=6, want_cov=True)
    np.testing.assert_array_equal(r_gen["mean"], r_race["mean"])
    e = np.abs(r_gen["mean"][..., 4])
    hg = r_gen["h"]
    np.testing.assert_allclose(r_race["h"], hg * (hg + 2 * e), rtol=1e-10, atol=1e-12)
    assert (hg < 0).any() and (hg > 0).any()


def test_cantelli_back_off_bounds_the_particles_violation_fraction():
    """Cantelli's inequality holds for any distribution, the particles' own included: at every step
    where h >= 0 for one half-space with nu = sqrt((1 - p)/p), at most a fraction p of the particles
    violate it. The particles are rebuilt from the stream-3 draws (no disturbance, exact linear steps)."""
    pl = 0.2
    p = _quiet_di(2, 50, 10, 0.0)
    c = workload.halfspace((0, 1, 0, 0), 0.9, pl, backoff="cantelli")
    p.constraints = (c,)
    x0 = np.array([0.0, 0.0, 0.5, 1.0], np.float32)
    Sig0 = np.diag([0.05, 0.05, 0.02, 0.04]).astype(np.float32)
    v = np.zeros((p.T, 2), np.float32)
    ctr = 13
    r = oracle.Oracle(p).solve(x0, v, ctr=ctr, Sigma0=Sig0, want_cov=True)
    A, _ = _di_mats(float(np.float32(p.dt)))
    L0 = np.linalg.cholesky(Sig0.astype(float))
    checked = 0
    for k in range(p.K):
        X = np.array([x0 + L0 @ _xi(p, 0, n, k, ctr, 4, stream=3) for n in range(p.M)])
        for t in range(1, p.T + 1):
            X = X @ A.T
            np.testing.assert_allclose(X.mean(axis=0), r["mean"][k, t], rtol=1e-10, atol=1e-12)
            if r["h"][k, t] >= 0:
                frac = np.mean(X[:, 1] - 0.9 >= 0)
                assert frac <= pl + 1e-12, (k, t, frac)
                checked += 1
    assert 0 < checked < p.K * p.T  # the bound was exercised, and h also went negative
