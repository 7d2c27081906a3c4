"""Parity of the general constraint set (half-spaces and disk obstacles with per-constraint chance
levels and back-off rules; h = min_q h_q) against the FP64 oracle, through the C ABI.

Tolerances are those of the persistent-particle parity tests. Samples whose mean passes within 1e-4
of a constraint's boundary (the oracle's margin) are excluded from the cost comparison, because
there the C_obs indicator may be decided differently in FP32 and FP64.
"""
import numpy as np
import pytest

import oracle
import workload
from tests.test_gpu_parity import assert_close, check_solve, check_unrecorded, gpu_solve
from tests.test_gpu_resample import redraw_atol
from tests.test_oracle_solve import CORRELATED_W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2408_00494_gb300 import bssmppi  # noqa: E402

DI_CONS = (workload.halfspace((0, 1, 0, 0), 1.2, 0.05),
           workload.halfspace((1, 1, 0, 0), 2.5, 0.1, backoff="cantelli"),
           workload.disk(0, 1, (0.8, 0.1), 0.35, 0.02))


def _racing_cons(p, x0):
    """Track edges as two half-spaces on e_y plus a disk obstacle 6 m ahead on the (s, e_y) plane."""
    wT = float(p.w_T)
    return (workload.halfspace((0, 0, 0, 0, 1, 0), wT, 0.05),
            workload.halfspace((0, 0, 0, 0, -1, 0), wT, 0.05),
            workload.disk(5, 4, (float(x0[5]) + 6.0, float(x0[4]) + 0.3), 1.0, 0.05, backoff="cantelli"))


def test_constraints_double_integrator():
    p = workload.double_integrator_problem(K=96, M=32, T=16, q_w=0.01)
    p.Sigma_w = CORRELATED_W
    p.constraints = DI_CONS
    x0 = np.array([0.0, 0.2, 1.0, 0.3], np.float32)
    v = workload.random_nominal(p, 12, scale=(1.0, 1.0))
    Sig0 = np.diag([0.02, 0.03, 0.01, 0.01]).astype(np.float32)
    check_solve(p, x0, v, ctr=7, Sigma0=Sig0)


@pytest.mark.parametrize("resample", [0, 1])
def test_constraints_racing_obstacle_ahead(resample):
    p = workload.config0()
    p.M, p.resample = 32, resample
    x0, v = workload.random_state(p, 51), workload.random_nominal(p, 51)
    x0[4] = 0.2
    p.constraints = _racing_cons(p, x0)
    check_solve(p, x0, v, ctr=11, mean_atol=redraw_atol if resample else None)


@pytest.mark.parametrize("M", [20, 64, 128])
def test_constraints_on_the_road_plane_without_recording(M):
    """A set on e_y and s only (track edges and an obstacle), with the racing cost and no recording:
    the build that keeps four means and the (e_y, s) covariance, against the oracle on every sample
    (costs, weights, v+ isolated and end to end). M = 20 leaves lanes empty; M = 128 puts four
    particles in a lane."""
    p = workload.config0()
    p.K, p.M, p.T = 384, M, 16
    x0, v = workload.random_state(p, 60 + M), workload.random_nominal(p, 60 + M)
    x0[4] = 0.2
    p.constraints = _racing_cons(p, x0)
    check_unrecorded(p, x0, v, ctr=13 + M)


def test_constraints_full_size_sampled_parity():
    """K=4096, M=64, T=40 with the obstacle set: sampled costs against the oracle sample by sample,
    the update against the oracle's update from the GPU's costs."""
    p = workload.config1()
    x0, v = workload.random_state(p, 16), workload.random_nominal(p, 16)
    x0[4] = 0.0
    p.constraints = _racing_cons(p, x0)
    g = gpu_solve(p, x0, v, ctr=77, record=False)
    o = oracle.Oracle(p)
    for k in (0, 5, 1024, 4095):
        r = o.solve(x0, v, 77, k_range=(k, k + 1))
        if r["margin"][k] > 1e-3:
            assert abs(g["S"][k] - r["S"][k]) <= 1e-4 * max(1.0, abs(r["S"][k])), k
    u_gpu = v.astype(np.float64)[None] + g["eps"]
    w_iso, vp_iso, _ = oracle.optimal_control(g["S"], u_gpu, float(np.float32(p.lam)))
    assert_close(g["w"], w_iso, 1e-5, 1e-7, "weights")
    assert_close(g["v_plus"], vp_iso, 1e-4, 1e-5, "v+")


def test_empty_set_restores_racing_barrier_and_bad_sets_are_rejected():
    p = workload.config0()
    x0, v = workload.random_state(p, 2), workload.random_nominal(p, 2)
    base = gpu_solve(p, x0, v, ctr=3, record=False)
    c = bssmppi.Controller(p)
    try:
        bad = (dict(DI_CONS[0], p=0.6), dict(DI_CONS[1], p=0.0), dict(DI_CONS[2], i=1, j=1),
               dict(DI_CONS[2], radius=-1.0), dict(DI_CONS[0], backoff="cantelli", p=1.0))
        for b in bad:
            with pytest.raises(bssmppi.BssmppiError):
                bssmppi.set_constraints(c.h, [b])
        with pytest.raises(bssmppi.BssmppiError):
            bssmppi.set_constraints(c.h, [DI_CONS[0]] * 9)
        bssmppi.set_constraints(c.h, _racing_cons(p, x0))
        bssmppi.set_constraints(c.h, [])
        bssmppi.set_counter(c.h, 3)
        vt = torch.as_tensor(v, device="cuda")
        bssmppi.solve(c.h, torch.as_tensor(x0, device="cuda"), None, vt)
        S = c.buffer(bssmppi.BUF_S).cpu().numpy()
        np.testing.assert_array_equal(S, base["S"].astype(np.float32))
        with pytest.raises(bssmppi.BssmppiError):  # the repair differentiates the racing barrier only
            bssmppi.set_constraints(c.h, _racing_cons(p, x0))
            bssmppi.repair_grad(c.h, torch.as_tensor(x0, device="cuda"), None, torch.zeros(p.T, 2, device="cuda"))
    finally:
        c.close()


def test_switching_barriers_matches_fresh_handles():
    """One handle switched racing -> constraint set -> racing -> constraint set gives, solve by
    solve, the costs of fresh handles built for each configuration (same counter)."""
    p = workload.config0()
    x0, v = workload.random_state(p, 9), workload.random_nominal(p, 9)
    cons = _racing_cons(p, x0)
    expect = {}
    for name, cs in (("racing", ()), ("set", cons)):
        q = workload.Problem(**{**p.__dict__, "constraints": cs})
        expect[name] = gpu_solve(q, x0, v, ctr=12, record=False)["S"]
    c = bssmppi.Controller(p)
    try:
        for name in ("racing", "set", "racing", "set"):
            bssmppi.set_constraints(c.h, cons if name == "set" else [])
            bssmppi.set_counter(c.h, 12)
            bssmppi.solve(c.h, torch.as_tensor(x0, device="cuda"), None, torch.as_tensor(v, device="cuda"))
            S = c.buffer(bssmppi.BUF_S).cpu().numpy().astype(np.float64)
            np.testing.assert_array_equal(S, expect[name])
    finally:
        c.close()
