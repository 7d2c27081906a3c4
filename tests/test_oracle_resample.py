"""Pins of the oracle's literal reading of Algorithm 2 (particles re-drawn from N(mean, cov) before
every step, `resample` = 1).

Each test checks the oracle against something other than itself: the linear-Gaussian one-step
moment law, an exact identity built from the separately pinned Philox/Box-Muller primitives and
numpy's Cholesky factor, and the equivalence of both readings when the belief has no spread.
"""
import numpy as np
import pytest

import oracle
import workload
from tests.test_oracle_solve import CORRELATED_W, _di_mats


def _xi(p, k, n, sample, ctr, nx, stream=4):
    """The standard normals of the re-draw of particle n before step k (stream 4; stream 3 holds
    the initial particles)."""
    key = (int(p.seed) & 0xFFFFFFFF, int(p.seed) >> 32)
    out = []
    for i in range((nx + 1) // 2):
        w = oracle.philox((k | ((i // 2) << 16), n, sample, (stream << 28) | ctr), key)
        out.extend(oracle.gaussian_pair(int(w[2 * (i % 2)]), int(w[2 * (i % 2) + 1])))
    return np.array(out[:nx])


def test_resample_one_step_moments_follow_linear_gaussian_law():
    """Linear dynamics: given the Monte-Carlo moments (m_k, C_k) of step k, the re-drawn particles
    are N(m_k, C_k), so step k+1 has mean A m_k + B u_k and covariance A C_k A^T + Sigma_w, within
    Monte-Carlo error (the mean's error now includes the re-draw's own spread A C_k A^T / M)."""
    p = workload.double_integrator_problem(K=1, M=40000, T=8, q_w=0.01, resample=1)
    p.Sigma_w = CORRELATED_W
    o = oracle.Oracle(p)
    x0 = np.array([0.5, -1.0, 1.0, 0.2], np.float32)
    Sig0 = np.diag([0.04, 0.09, 0.01, 0.02]).astype(np.float32)
    Sig0[0, 2] = Sig0[2, 0] = 0.005
    v = workload.random_nominal(p, 3, scale=(1.0, 1.0))
    r = o.solve(x0, v, ctr=11, Sigma0=Sig0, want_cov=True)
    A, B = _di_mats(float(np.float32(p.dt)))
    M, zmax = p.M, 0.0
    for t in range(1, p.T):
        m, C = r["mean"][0, t], r["cov"][0, t]
        mean = A @ m + B @ r["u"][0, t]
        cov = A @ C @ A.T + CORRELATED_W
        sd_mean = np.sqrt(np.diag(cov) / M)
        zmax = max(zmax, np.max(np.abs(r["mean"][0, t + 1] - mean) / sd_mean))
        d = np.diag(cov)
        sd_cov = np.sqrt((np.outer(d, d) + cov * cov) / (M - 1))
        zmax = max(zmax, np.max(np.abs(r["cov"][0, t + 1] - cov) / sd_cov))
    assert zmax < 5.5, zmax


@pytest.mark.parametrize("crn", [0, 1])
def test_resample_draws_are_mean_plus_cholesky_times_stream4(crn):
    """Without disturbance the linear step is exact, so the moments of step k+1 are those of
    A (m_k + L_k xi^n) + B u_k, with L_k = numpy's Cholesky factor of the oracle's C_k and xi^n the
    stream-4 normals of (step k, particle n, sample k or 0). Step 0 keeps the initial particles."""
    p = workload.double_integrator_problem(K=3, M=16, T=4, q_w=0.0, resample=1, crn_disturbance=crn)
    o = oracle.Oracle(p)
    x0 = np.array([0.3, 0.1, -0.4, 0.8], np.float32)
    Sig0 = np.array([[0.05, 0.01, 0.0, 0.002], [0.01, 0.04, 0.003, 0.0],
                     [0.0, 0.003, 0.03, 0.001], [0.002, 0.0, 0.001, 0.02]], np.float32)
    v = workload.random_nominal(p, 5, scale=(1.0, 1.0))
    ctr = 21
    r = o.solve(x0, v, ctr=ctr, Sigma0=Sig0, want_cov=True)
    A, B = _di_mats(float(np.float32(p.dt)))
    for k in range(p.K):
        sample = 0 if crn else k
        for t in range(0, p.T):
            if t == 0:  # the initial particles x0 + L_0 xi^n (stream 3) are step 0's draw
                m, L, stream = x0.astype(float), np.linalg.cholesky(Sig0.astype(float)), 3
            else:
                m, L, stream = r["mean"][k, t], np.linalg.cholesky(r["cov"][k, t]), 4
            X = np.array([m + L @ _xi(p, t, n, sample, ctr, 4, stream) for n in range(p.M)])
            Xn = X @ A.T + B @ r["u"][k, t]
            np.testing.assert_allclose(r["mean"][k, t + 1], Xn.mean(axis=0), rtol=1e-10, atol=1e-12)
            np.testing.assert_allclose(r["cov"][k, t + 1], np.cov(Xn.T, ddof=1), rtol=1e-8, atol=1e-13)


def test_persistent_particles_are_not_redrawn():
    """Control for the test above: with persistent particles and no disturbance, the covariance
    maps exactly (C_{k+1} = A C_k A^T); with re-drawing it does not (the new draws have their own
    sample covariance)."""
    out = {}
    for rs in (0, 1):
        p = workload.double_integrator_problem(K=1, M=32, T=3, q_w=0.0, resample=rs)
        o = oracle.Oracle(p)
        r = o.solve(np.zeros(4, np.float32), np.zeros((3, 2), np.float32), ctr=3,
                    Sigma0=np.diag([0.1, 0.2, 0.3, 0.4]).astype(np.float32), want_cov=True)
        A, _ = _di_mats(float(np.float32(p.dt)))
        out[rs] = np.abs(r["cov"][0, 3] - A @ r["cov"][0, 2] @ A.T).max() / np.abs(r["cov"][0, 3]).max()
    assert out[0] < 1e-12
    assert out[1] > 1e-3


def test_resample_without_spread_equals_persistent():
    """A known state and no disturbance: the belief has no spread, the re-draw returns the mean,
    and both readings give identical costs, moments and update."""
    res = []
    for rs in (0, 1):
        p = workload.config0()
        p.K, p.M, p.T = 8, 4, 10
        p.Sigma_w = np.zeros((6, 6))
        p.resample = rs
        x0 = workload.random_state(p, 12)
        v = workload.random_nominal(p, 12)
        res.append(oracle.Oracle(p).solve(x0, v, ctr=9, want_cov=True))
    for key in ("S", "mean", "v_plus", "w"):
        np.testing.assert_array_equal(res[0][key], res[1][key])
