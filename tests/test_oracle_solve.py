"""Pins of the oracle's solve: belief moments, costs, weights, update and the repair adjoint.

Each test checks the oracle against something other than itself: a closed form (linear-Gaussian
moment propagation, a constant-barrier cost), a limit of the update law (lambda -> 0 / infinity),
an unbiasedness property, the literal brute-force restatement in tests/literal_bssmppi.py, or
central finite differences.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import workload
from tests import literal_bssmppi as lit


def _di_mats(dt):
    A = np.block([[np.eye(2), dt * np.eye(2)], [np.zeros((2, 2)), np.eye(2)]])
    B = np.vstack([0.5 * dt * dt * np.eye(2), dt * np.eye(2)])
    return A, B


CORRELATED_W = np.array([[0.010, 0.004, 0.002, 0.000],
                         [0.004, 0.020, 0.000, -0.003],
                         [0.002, 0.000, 0.015, 0.005],
                         [0.000, -0.003, 0.005, 0.012]])


@pytest.mark.parametrize("with_sigma0,correlated", [(False, False), (True, False), (False, True)])
def test_linear_gaussian_moments_match_closed_form(with_sigma0, correlated):
    """Linear dynamics with additive Gaussian noise: mean_{k+1} = A mean_k + B u_k and
    Cov_{k+1} = A Cov_k A^T + Sigma_w (the analytic belief dynamics mentioned in Sec. IV-C).
    Monte-Carlo moments must sit within a few standard errors of them."""
    p = workload.double_integrator_problem(K=2, M=40000, T=8, q_w=0.01)
    if correlated:
        p.Sigma_w = CORRELATED_W
    o = oracle.Oracle(p)
    x0 = np.array([0.5, -1.0, 1.0, 0.2], np.float32)
    v = workload.random_nominal(p, 3, scale=(1.0, 1.0))
    Sig0 = None
    if with_sigma0:
        Sig0 = np.diag([0.04, 0.09, 0.01, 0.02]).astype(np.float32)
        Sig0[0, 2] = Sig0[2, 0] = 0.005
    r = o.solve(x0, v, ctr=11, Sigma0=Sig0, want_cov=True)
    dt = float(np.float32(p.dt))
    A, B = _di_mats(dt)
    M = p.M
    zmax = 0.0
    for k in range(p.K):
        mean = x0.astype(float)
        cov = np.zeros((4, 4)) if Sig0 is None else Sig0.astype(float)
        for t in range(p.T):
            mean = A @ mean + B @ r["u"][k, t]
            cov = A @ cov @ A.T + np.asarray(p.Sigma_w)
            mc_mean, mc_cov = r["mean"][k, t + 1], r["cov"][k, t + 1]
            sd_mean = np.sqrt(np.diag(cov) / M)
            zmax = max(zmax, np.max(np.abs(mc_mean - mean) / sd_mean))
            d = np.diag(cov)
            sd_cov = np.sqrt((np.outer(d, d) + cov * cov) / (M - 1))
            zmax = max(zmax, np.max(np.abs(mc_cov - cov) / sd_cov))
    assert zmax < 5.5, zmax


def test_covariance_estimator_is_unbiased():
    """With M = 3 particles, the 1/(M-1) estimator averages to the true covariance over many
    independent samples (1/M would average to 2/3 of it)."""
    p = workload.double_integrator_problem(K=20000, M=3, T=1, q_w=0.01)
    o = oracle.Oracle(p)
    r = o.solve(np.zeros(4, np.float32), np.zeros((1, 2), np.float32), ctr=2, want_cov=True)
    c1 = r["cov"][:, 1]
    avg = c1.mean(axis=0)
    se = 0.01 * math.sqrt(2.0 / (3 - 1)) / math.sqrt(p.K)
    assert np.all(np.abs(np.diag(avg) - 0.01) < 5 * se)
    off = avg[~np.eye(4, dtype=bool)]
    assert np.all(np.abs(off) < 5 * 0.01 / math.sqrt(p.K))


def test_zero_disturbance_collapses_belief():
    """No disturbance and a known state: every particle coincides, the covariance vanishes, the
    barrier reduces to h = w_T^2 - mean_ey^2, and the cost does not depend on M."""
    costs = []
    for M in (2, 5, 8):
        p = workload.config0()
        p.K, p.M, p.T = 16, M, 12
        p.Sigma_w = np.zeros((6, 6))
        o = oracle.Oracle(p)
        x0 = workload.random_state(p, 4)
        v = workload.random_nominal(p, 4)
        r = o.solve(x0, v, ctr=5, want_cov=True)
        assert np.abs(r["cov"]).max() < 1e-20
        wT = float(np.float32(p.w_T))
        np.testing.assert_allclose(r["h"], wT * wT - r["mean"][:, :, 4] ** 2, rtol=1e-13, atol=1e-12)
        # the mean follows the deterministic model
        xd = x0.astype(float)
        for t in range(p.T):
            xd = o.model_step(xd, r["u"][0, t])
            np.testing.assert_allclose(r["mean"][0, t + 1], xd, rtol=1e-12, atol=1e-12)
        costs.append(r["S"])
    np.testing.assert_allclose(costs[1], costs[0], rtol=1e-12)
    np.testing.assert_allclose(costs[2], costs[0], rtol=1e-12)


def _quiet_di(T, y0, vy):
    """Double integrator without noise (disturbance 0, negligible control noise, no control cost)."""
    p = workload.double_integrator_problem(K=1, M=2, T=T, q_w=0.0)
    p.Sigma_eps = np.diag([1e-30, 1e-30])
    p.ctrl_w = 0.0
    p.C_safe = 100.0
    x0 = np.array([0.0, y0, 0.0, vy], np.float32)
    return p, x0


def test_cost_constant_barrier_inside_and_outside_safe_set():
    """A state at rest keeps h constant. Inside the safe set (h > 0) the DCBF condition
    h_k - (1 - gamma) h_{k-1} >= 0 holds and C_safe = 0; outside (h < 0) every step pays
    C gamma |h|, including step 0 where z_{-1} = z_0."""
    T = 7
    f = lambda x: float(np.float32(x))
    for y0, outside in ((1.0, False), (6.0, True)):
        p, x0 = _quiet_di(T, y0, 0.0)
        r = oracle.Oracle(p).solve(x0, np.zeros((T, 2), np.float32), ctr=0)
        wT, C, g = f(p.w_T), f(p.C_safe), f(p.gamma)
        q = f(0.1) * y0 * y0 + (f(p.C_obs) if outside else 0.0)
        h = wT * wT - y0 * y0
        expect = (T + 1) * q + (T + 1) * (C * g * (-h) if outside else 0.0)
        assert r["S"][0] == pytest.approx(expect, rel=1e-12)


def test_cost_moving_toward_boundary_closed_form():
    """Constant lateral velocity: p_y(k) = y0 + k dt v_y exactly, so h_k and the C_safe terms of
    every step follow in closed form; this pins the alignment of h_k with h_{k-1} and the
    terminal term."""
    T, y0, vy = 9, 1.0, 20.0
    p, x0 = _quiet_di(T, y0, vy)
    r = oracle.Oracle(p).solve(x0, np.zeros((T, 2), np.float32), ctr=0)
    f = lambda x: float(np.float32(x))
    dt, wT, C, g, Cobs = f(p.dt), f(p.w_T), f(p.C_safe), f(p.gamma), f(p.C_obs)
    ys = [y0 + k * dt * vy for k in range(T + 1)]
    hs = [wT * wT - y * y for y in ys]
    q = lambda y: f(0.1) * y * y + f(0.01) * vy * vy + (Cobs if abs(y) > wT else 0.0)
    penalties = [C * max(-hs[k] + (1 - g) * hs[max(k - 1, 0)], 0.0) for k in range(T + 1)]
    expect = sum(q(ys[k]) for k in range(T)) + q(ys[T]) + sum(penalties)
    assert sum(1 for x in penalties if x > 0) >= 3
    assert r["S"][0] == pytest.approx(expect, rel=1e-9)


def test_weights_closed_form_and_limits():
    rng = np.random.default_rng(0)
    K, T = 7, 4
    u = rng.normal(size=(K, T, 2))
    # two samples, S = (0, lambda ln 2): weights 2/3, 1/3
    lam = 0.7
    w, vp, diag = oracle.optimal_control(np.array([0.0, lam * math.log(2.0)]), u[:2], lam)
    np.testing.assert_allclose(w, [2 / 3, 1 / 3], rtol=1e-14)
    np.testing.assert_allclose(vp, (2 * u[0] + u[1]) / 3, rtol=1e-13)
    S = rng.uniform(10, 20, size=K)
    w, vp, diag = oracle.optimal_control(S, u, 1.0)
    assert w.sum() == pytest.approx(1.0, rel=1e-15)
    assert diag[0] == S.min() and diag[1] >= 1.0
    assert diag[2] == pytest.approx(1.0 / np.sum(w * w), rel=1e-14)
    # shift invariance (beta is subtracted)
    w2, vp2, _ = oracle.optimal_control(S + 1e3, u, 1.0)
    np.testing.assert_allclose(w2, w, rtol=1e-10)
    # lambda -> infinity: plain average; lambda -> 0: the minimum-cost sample
    _, vp_inf, _ = oracle.optimal_control(S, u, 1e9)
    np.testing.assert_allclose(vp_inf, u.mean(axis=0), rtol=1e-7, atol=1e-8)
    _, vp_0, _ = oracle.optimal_control(S, u, 1e-9)
    np.testing.assert_array_equal(vp_0, u[np.argmin(S)])
    # ties at the minimum under lambda -> 0 average the tied samples
    S2 = S.copy()
    S2[3] = S2[5] = S.min() - 1
    _, vp_tie, _ = oracle.optimal_control(S2, u, 1e-9)
    np.testing.assert_allclose(vp_tie, 0.5 * (u[3] + u[5]), rtol=1e-14)


@pytest.mark.parametrize("case", ["racing", "racing_crn", "racing_sigma_edge", "double_integrator"])
def test_oracle_matches_literal_brute_force(case):
    if case.startswith("racing"):
        p = workload.config0()
        p.K, p.M, p.T = 3, 3, 3
        p.crn_disturbance = int(case == "racing_crn")
        x0 = workload.random_state(p, 9)
        if case == "racing_sigma_edge":
            x0[4] = 2.9  # near the boundary so the barrier and hinge are active
            x0[3] = 0.1
    else:
        p = workload.double_integrator_problem(K=4, M=4, T=3)
        p.Sigma_w = CORRELATED_W
        x0 = workload.random_state(p, 9)
    v = workload.random_nominal(p, 10)
    r = oracle.Oracle(p).solve(x0, v, ctr=77, want_cov=True)
    P = lit.problem_dict(p, oracle.backoff_gaussian(float(np.float32(p.delta))))
    S, U, MEAN, COV, VP, W = lit.solve(P, [float(x) for x in x0], v.astype(float).tolist(), 77)
    np.testing.assert_allclose(r["S"], S, rtol=1e-11)
    np.testing.assert_allclose(r["u"], U, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(r["mean"], MEAN, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(r["cov"], COV, rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(r["v_plus"], VP, rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(r["w"], W, rtol=1e-10, atol=1e-15)


@pytest.mark.parametrize("backoff,clamp", [(1, 0), (0, 1), (1, 1)])
def test_backoff_and_clamped_margin_match_the_literal_restatement(backoff, clamp):
    """Remark 1's Cantelli back-off nu = sqrt((1 - delta) / delta) (computed here from delta, not by
    the oracle) and the clamped margin max(w_T - nu sigma, 0) against the pure-Python restatement,
    on a case where the back-off exceeds the half-width at some steps (large disturbance, narrow
    track), so the clamp is active."""
    p = workload.config0()
    p.K, p.M, p.T = 3, 4, 4
    p.backoff, p.clamp_margin = backoff, clamp
    p.w_T = 0.4
    p.Sigma_w = np.diag(np.array([0.02, 0.02, 0.01, 0.002, 0.3, 0.0]) ** 2)
    x0 = workload.random_state(p, 9)
    x0[4] = 0.1
    v = workload.random_nominal(p, 10)
    r = oracle.Oracle(p).solve(x0, v, ctr=31, want_cov=True)
    d = float(np.float32(p.delta))
    nu = math.sqrt((1.0 - d) / d) if backoff else oracle.backoff_gaussian(d)
    P = lit.problem_dict(p, nu)
    S, U, MEAN, COV, VP, W = lit.solve(P, [float(x) for x in x0], v.astype(float).tolist(), 31)
    np.testing.assert_allclose(r["S"], S, rtol=1e-11)
    np.testing.assert_allclose(r["v_plus"], VP, rtol=1e-11, atol=1e-14)
    sig = np.sqrt(r["cov"][:, :, 4, 4])
    assert np.any(nu * sig > float(np.float32(p.w_T)))  # the back-off passes the half-width somewhere
    if clamp:  # there the barrier is minus the squared mean, exactly
        wide = nu * sig >= float(np.float32(p.w_T))
        np.testing.assert_array_equal(r["h"][wide], -r["mean"][:, :, 4][wide] ** 2)


def _repair_case(model):
    if model == "racing":
        p = workload.config0()
        p.M, p.T = 8, 6
        x0 = np.array([9.0, 0.2, 0.1, 0.3, 2.7, 5.0], np.float32)
    else:
        p = workload.double_integrator_problem(K=1, M=8, T=6, q_w=0.05)
        p.w_T = 2.0
        x0 = np.array([0.0, 1.2, 0.5, 1.5], np.float32)
    v = workload.random_nominal(p, 21)
    return p, x0, v.astype(float)


@pytest.mark.parametrize("model", ["racing", "double_integrator"])
def test_repair_adjoint_matches_central_differences(model):
    p, x0, v = _repair_case(model)
    o = oracle.Oracle(p)
    J, g = o.repair_objective(x0, v, ctr=3)
    assert J > 0.0
    eps = 1e-4
    rng = np.random.default_rng(1)
    for _ in range(4):
        d = rng.normal(size=v.shape)
        fd = (o.repair_objective(x0, v + eps * d, 3, grad=False)
              - o.repair_objective(x0, v - eps * d, 3, grad=False)) / (2 * eps)
        assert float(np.sum(g * d)) == pytest.approx(fd, rel=2e-5, abs=1e-6 * abs(J))
    # a few single components
    for (t, j) in ((0, 0), (0, 1), (p.T // 2, 0), (p.T - 1, 1)):
        e = np.zeros_like(v)
        e[t, j] = 1.0
        fd = (o.repair_objective(x0, v + eps * e, 3, grad=False)
              - o.repair_objective(x0, v - eps * e, 3, grad=False)) / (2 * eps)
        assert g[t, j] == pytest.approx(fd, rel=2e-5, abs=1e-6 * abs(J))


@pytest.mark.parametrize("model", ["racing", "double_integrator"])
def test_repair_objective_equals_the_rollouts_barrier_penalty(model):
    """The value of J_r: the belief-DCBF penalty sum_{t=1..T} C max(-h_t + (1 - gamma) h_{t-1}, 0)
    (Eq. "cbfpenalty") of the M-particle rollout of the nominal v under sample 0's disturbance
    draws. The solve's rollout (whose moments, barrier and costs the other tests pin) forms the same
    barrier values h_t (Eq. "DCBF") when the control noise is zero and every sample shares sample 0's
    draws, so J_r and its hinge arguments must equal that sum built from the rollout's own h. A 1/M
    variance, a shifted h_0 or draws taken from another sample in the repair's separate rollout
    each break it."""
    p, x0, v = _repair_case(model)
    o_rep = oracle.Oracle(p)
    J, args = o_rep.repair_objective(x0, v, ctr=3, grad=False, want_args=True)
    q = dataclasses.replace(p, K=2, crn_disturbance=1, Sigma_eps=np.zeros((2, 2)))
    h = oracle.Oracle(q).solve(x0, v, 3, k_range=(1, 2))["h"][1]
    C, gam = float(np.float32(p.C_safe)), float(np.float32(p.gamma))
    arg_ref = -h[1:] + (1.0 - gam) * h[:-1]
    np.testing.assert_allclose(args[1:], arg_ref, rtol=1e-12, atol=1e-12 * np.abs(h).max())
    J_ref = float(np.sum(C * np.maximum(arg_ref, 0.0)))
    assert J_ref > 0.0  # the hinge is active in these cases
    assert J == pytest.approx(J_ref, rel=1e-12)


@pytest.mark.parametrize("case", ["racing", "resample", "sigma0"])
def test_threaded_oracle_equals_one_thread(case):
    """Samples spread over threads give every output of the one-thread solve bit for bit."""
    p = workload.config0()
    p.K, p.T = 67, 8
    Sig0 = None
    if case == "resample":
        p.resample = 1
    if case == "sigma0":
        Sig0 = np.eye(6) * 1e-3
    x0, v = workload.random_state(p, 4), workload.random_nominal(p, 4)
    o = oracle.Oracle(p)
    r1 = o.solve(x0, v, 5, Sigma0=Sig0, want_cov=True)
    r4 = o.solve(x0, v, 5, Sigma0=Sig0, want_cov=True, threads=4)
    for key in r1:
        assert np.array_equal(r1[key], r4[key]), key


def test_repair_objective_rejects_the_wheel_speed_model():
    p = workload.wheels_problem(4, 4, 3)
    with pytest.raises(ValueError):
        oracle.Oracle(p).repair_objective(workload.racing_x0(p), np.zeros((3, 2)), 0)


@pytest.mark.parametrize("cuts", [(), (1,), (37, 38, 100), (5, 17, 64, 65, 90, 120)])
def test_lse_partials_merge_to_the_full_update(cuts):
    """Splitting the samples into disjoint groups, taking each group's log-sum-exp partial and
    merging them reproduces the weights' normaliser and the update of the whole set (the exchange a
    sample-sharded solve makes), including groups whose best cost is far above the global best."""
    rng = np.random.default_rng(len(cuts))
    K, T, lam = 128, 6, 0.1
    S = rng.uniform(0.0, 50.0, K)
    S[90:] += 1e4  # a group that the merge rescales by exp(-1e5) (underflows to 0 weight)
    u = rng.normal(size=(K, T, 2))
    edges = (0,) + tuple(cuts) + (K,)
    parts = np.array([oracle.lse_partial(S, u, lam, (a, b)) for a, b in zip(edges[:-1], edges[1:])])
    vp, diag = oracle.lse_merge(parts, lam, K)
    w_ref, vp_ref, diag_ref = oracle.optimal_control(S, u, lam)
    np.testing.assert_allclose(vp, vp_ref, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(diag, diag_ref, rtol=1e-12)
