"""Parity of the single-track model with wheel speeds and combined slip (model 2, 8 states) against
the FP64 oracle, through the C ABI: one model step, whole solves (persistent particles, re-sampling,
a constraint set) and the benchmark-size solve sampled.

Tolerances are those of the bicycle model's tests: model step rel/abs 2e-5 (a few FP32 ulps through
n_sub = 10 Euler substeps, the tyre curve's hardware sine within 2^-21.4 of its unit amplitude);
solves as in tests/test_gpu_parity.py, except for the variances of large states (wheel_var_atol).
"""
import numpy as np
import pytest

import oracle
import workload
from tests.test_gpu_parity import _dev, assert_close, check_solve, gpu_solve
from tests.test_gpu_resample import redraw_atol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2408_00494_gb300 import bssmppi  # noqa: E402


def test_model_step_matches_oracle():
    p = workload.wheels_problem(1, 2, 1)
    c = bssmppi.Controller(p)
    o = oracle.Oracle(p)
    n = 4096
    rng = np.random.default_rng(11)
    xs = np.stack([workload.random_state(p, i) for i in range(n)])
    xs[: n // 4, 3:5] *= rng.uniform(0.5, 1.5, size=(n // 4, 2)).astype(np.float32)  # slipping wheels
    xs[n // 2:, 5] = np.linspace(-1.2, 1.2, n - n // 2, dtype=np.float32)           # both heading branches
    us = np.stack([rng.uniform(p.u_min, p.u_max) for _ in range(n)]).astype(np.float32)
    out = torch.zeros((n, p.nx), device="cuda")
    bssmppi.model_step(c.h, _dev(xs), _dev(us), out)
    c.close()
    g = out.cpu().numpy().astype(np.float64)
    ref = np.stack([o.model_step(xs[i].astype(np.float64), us[i].astype(np.float64)) for i in range(n)])
    assert_close(g, ref, 2e-5, 2e-5, "wheel-speed model step")


def wheel_var_atol(prob):
    """Absolute tolerance of state i's particle variances, derived from FP32 rounding. A state of
    magnitude X (the wheel speeds: about 50 rad/s) takes one rounding of relative size u = 2^-24
    per Euler substep, so after N = T n_sub substeps each particle carries an error e of order
    sqrt(N) u X (a random walk of roundings), bounded here by e = 4 sqrt(N) u X. To first order the
    unbiased variance then moves by 2/(M-1) sum (x_n - mean) e_n <= 2 sigma e sqrt(M/(M-1)) (Cauchy-
    Schwarz), plus e^2. For the wheel speeds (sigma ~ 1 rad/s) that is ~1e-4, above the flat 1e-5;
    for the other states it stays below it."""
    N = prob.T * prob.n_sub

    def atol(ref, i):
        X = np.abs(ref["mean"][..., i]).max()
        e = 4.0 * np.sqrt(N) * 2.0 ** -24 * X
        sigma = np.sqrt(np.maximum(np.diagonal(ref["cov"], axis1=2, axis2=3)[..., i], 0.0))
        M = prob.M
        return 1e-5 + 2.0 * sigma * e * np.sqrt(M / (M - 1)) + e * e

    return atol


@pytest.mark.parametrize("M,K,crn", [(16, 192, 0), (64, 192, 0), (128, 192, 0), (16, 193, 1), (5, 77, 0)])
def test_solve_matches_oracle(M, K, crn):
    p = workload.wheels_problem(K, M, 20, crn_disturbance=crn)
    x0, v = workload.random_state(p, 70 + M), workload.random_nominal(p, 70 + M, scale=(0.1, 0.5))
    check_solve(p, x0, v, ctr=4, var_atol=wheel_var_atol(p))


def test_solve_resampled_with_constraints():
    p = workload.wheels_problem(128, 32, 16, resample=1)
    x0, v = workload.random_state(p, 81), workload.random_nominal(p, 81, scale=(0.1, 0.5))
    p.constraints = (workload.halfspace((0, 0, 0, 0, 0, 0, 1, 0), 2.0, 0.05),
                     workload.halfspace((0, 0, 0, 0, 0, 0, -1, 0), 2.0, 0.05),
                     workload.disk(7, 6, (float(x0[7]) + 4.0, float(x0[6])), 0.6, 0.05, backoff="cantelli"))
    check_solve(p, x0, v, ctr=2, mean_atol=redraw_atol, var_atol=wheel_var_atol(p))


def test_full_size_sampled_parity():
    """K=4096, M=64, T=40 (n_sub = 10): sampled costs against the oracle, the update against the
    oracle's update from the GPU's costs."""
    p = workload.wheels_problem(4096, 64, 40, seed=5)
    x0, v = workload.random_state(p, 82), workload.random_nominal(p, 82, scale=(0.1, 0.5))
    g = gpu_solve(p, x0, v, ctr=17, record=False)
    o = oracle.Oracle(p)
    for k in (0, 77, 2048, 4095):
        r = o.solve(x0, v, 17, k_range=(k, k + 1))
        assert_close(g["eps"][k], r["eps"][k], 0.0, 1e-6, f"eps[{k}]")
        if r["margin"][k] > 1e-3:
            assert abs(g["S"][k] - r["S"][k]) <= 1e-4 * max(1.0, abs(r["S"][k])), k
    u_gpu = v.astype(np.float64)[None] + g["eps"]
    w_iso, vp_iso, _ = oracle.optimal_control(g["S"], u_gpu, float(np.float32(p.lam)))
    assert_close(g["w"], w_iso, 1e-5, 1e-7, "weights")
    assert_close(g["v_plus"], vp_iso, 1e-4, 1e-5, "v+")


def test_limits_of_the_wheel_speed_model():
    p = workload.wheels_problem(64, 129, 10)
    with pytest.raises(bssmppi.BssmppiError):
        bssmppi.Controller(p)
    p = workload.wheels_problem(64, 16, 10)
    c = bssmppi.Controller(p)
    try:
        with pytest.raises(bssmppi.BssmppiError):  # no 8-state adjoint for the repair
            bssmppi.repair_grad(c.h, _dev(workload.racing_x0(p)), None, torch.zeros(p.T, 2, device="cuda"))
    finally:
        c.close()
