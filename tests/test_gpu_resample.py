"""Parity of the re-sampling rollout (Algorithm 2 read literally: particles re-drawn from
N(mean, cov) before every step) against the FP64 oracle, through the C ABI.

Tolerances are those of the persistent-particle parity tests (moments rel 1e-4 / abs 1e-5, costs
rel 1e-4 away from the collision indicator, weights and update from the GPU's own costs), with one
addition for the means. Every step re-draws the particles through an FP32 Cholesky factor of the
sample covariance. The factorisation is backward stable: the computed factor is exact for a
covariance perturbed by about nx 2^-24 ||C||, so a re-drawn particle can move by up to
sqrt(nx 2^-24) sigma_i along state i. That is small for a well-conditioned covariance, but it is
reached in its near-null directions, which appear when M is close to nx: with 8 particles in 6
states the correlation matrix's condition number reaches ~1e6 on these inputs. The means are
therefore compared with abs 1e-5 + sqrt(nx 2^-24) sigma_i, with sigma_i the oracle's largest
standard deviation of state i over the horizon.
"""
import numpy as np
import pytest

import oracle
import workload
from tests.test_gpu_parity import assert_close, check_solve, gpu_solve
from tests.test_oracle_solve import CORRELATED_W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2408_00494_gb300 import bssmppi  # noqa: E402


def redraw_atol(ref):
    """Per-state absolute tolerance of the means: 1e-5 + sqrt(nx 2^-24) max_t sigma_i."""
    nx = ref["cov"].shape[-1]
    sig = np.sqrt(np.max(np.diagonal(ref["cov"], axis1=2, axis2=3), axis=(0, 1)))
    return 1e-5 + np.sqrt(nx * 2.0 ** -24) * sig


def test_resample_double_integrator_with_initial_covariance():
    p = workload.double_integrator_problem(K=64, M=32, T=16, q_w=0.01, resample=1)
    p.Sigma_w = CORRELATED_W
    x0 = workload.random_state(p, 31)
    v = workload.random_nominal(p, 31, scale=(1.0, 1.0))
    Sig0 = np.diag([0.04, 0.09, 0.01, 0.02]).astype(np.float32)
    check_solve(p, x0, v, ctr=5, Sigma0=Sig0, mean_atol=redraw_atol)


@pytest.mark.parametrize("M", [8, 20, 32, 64, 128])
def test_resample_racing_particle_counts(M):
    p = workload.config0()
    p.M, p.resample = M, 1
    x0, v = workload.random_state(p, 40 + M), workload.random_nominal(p, 40 + M)
    check_solve(p, x0, v, ctr=3, mean_atol=redraw_atol)


def test_resample_racing_crn_and_ragged_K():
    p = workload.config0()
    p.K, p.M, p.T, p.resample, p.crn_disturbance = 333, 24, 30, 1, 1
    x0, v = workload.random_state(p, 77), workload.random_nominal(p, 77)
    check_solve(p, x0, v, ctr=9, mean_atol=redraw_atol)


def test_resample_without_spread_matches_persistent_kernel():
    """No disturbance and a known state: both kernels see zero covariance, the re-draw returns the
    mean, and their costs agree to rounding."""
    out = []
    for rs in (0, 1):
        p = workload.config0()
        p.Sigma_w = np.zeros((6, 6))
        p.resample = rs
        out.append(gpu_solve(p, workload.random_state(p, 5), workload.random_nominal(p, 5), ctr=2, record=False))
    assert_close(out[1]["S"], out[0]["S"], 1e-5, 1e-5, "S, re-sampled vs persistent without spread")


def test_resample_full_size_sampled_parity():
    """The benchmark's workload (K=4096, M=64, T=40) with re-sampling: sampled costs against the
    oracle sample by sample, the update against the oracle's update from the GPU's costs."""
    p = workload.config1()
    p.resample = 1
    x0, v = workload.random_state(p, 15), workload.random_nominal(p, 15)
    g = gpu_solve(p, x0, v, ctr=321, record=False)
    o = oracle.Oracle(p)
    for k in (0, 1, 33, 2048, 4095):
        r = o.solve(x0, v, 321, k_range=(k, k + 1))
        assert_close(g["eps"][k], r["eps"][k], 0.0, 1e-6, f"eps[{k}]")
        if r["margin"][k] > 1e-3:
            assert abs(g["S"][k] - r["S"][k]) <= 1e-4 * max(1.0, abs(r["S"][k])), k
    u_gpu = v.astype(np.float64)[None] + g["eps"]
    w_iso, vp_iso, _ = oracle.optimal_control(g["S"], u_gpu, float(np.float32(p.lam)))
    assert_close(g["w"], w_iso, 1e-5, 1e-7, "weights")
    assert_close(g["v_plus"], vp_iso, 1e-4, 1e-5, "v+")


def test_resample_not_offered_by_repair_and_server():
    p = workload.config0()
    p.resample = 1
    c = bssmppi.Controller(p)
    try:
        x0 = torch.as_tensor(workload.racing_x0(p), device="cuda")
        g = torch.zeros(p.T, 2, device="cuda")
        with pytest.raises(bssmppi.BssmppiError):
            bssmppi.repair_grad(c.h, x0, None, g)
    finally:
        c.close()
    s = bssmppi.server_create(4)
    try:
        with pytest.raises(bssmppi.BssmppiError):
            bssmppi.server_add_controller(s, bssmppi.make_params(p))
    finally:
        bssmppi.server_destroy(s)
