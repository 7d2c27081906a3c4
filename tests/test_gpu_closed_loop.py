"""Closed-loop parity on the small racing workload (K=256, M=16, T=20, track seed 0): 50
receding-horizon steps of Algorithm 1 (solve, apply u_0, shift the nominal by one step).

At every step the GPU's solve of the current state, nominal and solve counter is checked against
the FP64 oracle's solve of the same inputs, with the tolerances of tests/test_gpu_parity.py
(Philox draws, perturbations, moments, costs, weights, update). The loop then advances on the GPU's
outputs: u_0 into the plant (the FP64 model step plus a seeded N(0, Sigma_w) disturbance, rounded
to FP32), and v+ shifted by one step as the next nominal. So the 50 checks follow the controller
along its own trajectory, including the states it drives the car into.
"""
import numpy as np
import pytest

import oracle
import workload
from tests.test_gpu_parity import check_solve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fifty_closed_loop_steps_match_the_oracle_at_every_step():
    p = workload.config0()
    o = oracle.Oracle(p)
    x = workload.racing_x0(p)
    v = np.zeros((p.T, 2), np.float32)
    rng = np.random.default_rng(50)
    std = np.sqrt(np.diag(np.asarray(p.Sigma_w, dtype=np.float64)))
    ey = []
    for k in range(50):
        g, _ = check_solve(p, x, v, ctr=k)
        u0 = g["u0"].astype(np.float32)
        v = np.concatenate([g["v_plus"][1:], g["v_plus"][-1:]]).astype(np.float32)
        x = (o.model_step(x.astype(np.float64), u0.astype(np.float64))
             + rng.standard_normal(p.nx) * std).astype(np.float32)
        ey.append(float(x[4]))
    # the controller kept the car on the track and made progress along it
    assert np.max(np.abs(ey)) < p.w_T
    assert x[5] > 50 * p.dt * 0.5 * p.x_goal[0]
