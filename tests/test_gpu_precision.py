"""Precision study: FP32 with compensated reductions vs FP32 naive vs the FP64 oracle.

Compensated (the default): per-lane two-pass moments merged across lanes with Chan's pairwise
update, Neumaier-compensated cost sums, compensated weight and update sums. Naive: one-pass sums of
x and x^2 (variance = (sum x^2 - M mean^2) / (M - 1)) and plain sums. The tests assert the
compensated path's tolerances, assert that the naive variance loses accuracy where cancellation is
expected, and print every measured error (run with -s or -rA to read them).
"""
import numpy as np
import pytest

import oracle
import workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.test_gpu_parity import gpu_solve  # noqa: E402


def _rel(a, b, floor):
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


def test_variance_cancellation_near_the_boundary():
    """Mean e_y ~ 2.5 m with sigma ~ cm: sum x^2 - M mean^2 cancels ~3 digits in FP32."""
    p = workload.config0()
    p.K, p.M, p.T = 256, 64, 20
    x0 = workload.random_state(p, 21)
    x0[4], x0[3] = 2.5, 0.0
    v = np.zeros((p.T, 2), np.float32)
    ref = oracle.Oracle(p).solve(x0, v, 3, want_cov=True)
    ref_var = ref["cov"][:, 1:, 4, 4]
    errs = {}
    for comp in (1, 0):
        p.compensated = comp
        g = gpu_solve(p, x0, v, ctr=3)
        errs[comp] = _rel(g["var"][:, 1:, 4], ref_var, 1e-12)
    print(f"[precision] Var(e_y) rel err, mean e_y ~ 2.5 m: compensated max {errs[1].max():.2e} "
          f"median {np.median(errs[1]):.2e}; naive max {errs[0].max():.2e} median {np.median(errs[0]):.2e}")
    assert errs[1].max() < 1e-4
    assert np.median(errs[0]) > 10 * np.median(errs[1])


def test_linear_gaussian_closed_form_with_offset():
    """Double integrator at p_y = 100 m: Cov_{k+1} = A Cov_k A^T + 0.01 I in closed form. The
    average over K samples of the GPU's per-sample variances must sit within a few standard
    errors of it when compensated. The naive one-pass variance of each sample carries a
    cancellation error of a few percent (sum x^2 ~ 2.6e6 against (M - 1) Var ~ 25); its signs vary,
    so it shows per sample rather than in the K-average."""
    p = workload.double_integrator_problem(K=2048, M=256, T=20, q_w=0.01)
    p.w_T = 1000.0
    x0 = np.array([50.0, 100.0, 1.0, -0.5], np.float32)
    v = np.zeros((p.T, 2), np.float32)
    dt = float(np.float32(p.dt))
    A = np.block([[np.eye(2), dt * np.eye(2)], [np.zeros((2, 2)), np.eye(2)]])
    cov = np.zeros((4, 4))
    exact = []
    for _ in range(p.T):
        cov = A @ cov @ A.T + 0.01 * np.eye(4)
        exact.append(np.diag(cov).copy())
    exact = np.array(exact)                                 # (T, 4)
    se = exact * np.sqrt(2.0 / (p.M - 1)) / np.sqrt(p.K)    # standard error of the K-average
    out, per_sample = {}, {}
    for comp in (1, 0):
        p.compensated = comp
        g = gpu_solve(p, x0, v, ctr=8)
        avg = g["var"][:, 1:, :].mean(axis=0)               # (T, 4)
        out[comp] = np.abs(avg - exact) / se
        per_sample[comp] = g["var"][:, 1:, 1]               # Var(p_y), the offset component
    dev = np.sqrt(np.mean(((per_sample[0] - per_sample[1]) / per_sample[1]) ** 2))
    print(f"[precision] linear-Gaussian Var vs closed form (K-average), |z| max: compensated "
          f"{out[1].max():.2f}, naive {out[0].max():.2f}; per-sample RMS relative deviation of the "
          f"naive Var(p_y) from the compensated one {dev:.2e} (positions ~100 m)")
    assert out[1].max() < 5.5
    assert dev > 1e-3


@pytest.mark.parametrize("lam", [0.1, 1.0, 10.0])
def test_precision_large_workload(lam):
    """K=16384, M=128, T=60 on every sample, compensated and naive against the FP64 oracle: costs,
    means and Var(e_y) of every step, the weights and update against FP64 weights/update of the GPU's
    own costs and perturbations (isolated), and the end-to-end v+ against the oracle's own v+ next to
    the first-order bound sum_k w_k |dS_k - <dS>| / lambda |u_k - v+| of the measured cost errors."""
    p = workload.config3(lam)
    x0 = workload.racing_x0(p)
    # steer that follows the mean curvature (wheelbase x 2 pi / track length), so the samples stay
    # on the track and the weights spread over many samples
    v = np.zeros((p.T, 2), np.float32)
    v[:, 0] = (p.lf + p.lr) * 2 * np.pi / p.track_len
    ref = oracle.Oracle(p).solve(x0, v, 6, want_cov=True, threads=oracle.host_threads())
    ok = ref["margin"] > 1e-4
    scale = np.maximum(np.abs(ref["S"]), 1.0)
    ref_vey = ref["cov"][:, 1:, 4, 4]
    lam32 = float(np.float32(lam))
    rows = []
    for comp in (1, 0):
        p.compensated = comp
        g = gpu_solve(p, x0, v, ctr=6)
        dS = g["S"] - ref["S"]
        dSr = np.max(np.abs(dS[ok]) / scale[ok])
        dm = np.max(_rel(g["mean"], ref["mean"], 0.1))
        dv = np.max(_rel(g["var"][:, 1:, 4], ref_vey, 1e-6))
        u = v.astype(np.float64)[None] + g["eps"]
        w64, vp64, _ = oracle.optimal_control(g["S"], u, lam32)
        big = w64 > 1e-6
        dw = np.max(np.abs(g["w"][big] - w64[big]) / w64[big])
        dvp = np.max(np.abs(g["v_plus"] - vp64))
        dSc = np.where(ok, dS, 0.0)
        dev = np.abs(dSc - np.sum(ref["w"] * dSc)) / lam32
        bound = np.einsum("k,kti->ti", ref["w"] * dev, np.abs(ref["u"] - ref["v_plus"][None]))
        e2e = np.abs(g["v_plus"] - ref["v_plus"])
        w_e2e = np.max(np.abs(g["w"] - ref["w"])[ref["w"] > 1e-6] / ref["w"][ref["w"] > 1e-6])
        rows.append((comp, dSr, dm, dv, dw, dvp, e2e.max(), bound.max(), w_e2e, g["diag"][2], int(big.sum())))
        if comp:
            assert dSr < 1e-4
            assert dv < 1e-3
            assert dvp < 1e-5 + 1e-4 * np.abs(vp64).max()
            assert np.all(e2e <= 1e-5 + 1e-4 * np.abs(ref["v_plus"]) + 2 * bound)
    for comp, dSr, dm, dv, dw, dvp, e2e, bnd, w_e2e, ess, nbig in rows:
        print(f"[precision] K=16384 M=128 T=60 lambda={lam:g} {'compensated' if comp else 'naive'} (all {p.K} "
              f"samples, {int((~ok).sum())} within 1e-4 of the wall): S rel {dSr:.2e}, mean rel {dm:.2e}, "
              f"Var(e_y) rel {dv:.2e}, weights rel {dw:.2e} ({nbig} weights > 1e-6, ESS {ess:.0f}), v+ abs "
              f"{dvp:.2e} (isolated); end to end: v+ abs {e2e:.2e} (first-order bound {bnd:.2e}), weights rel "
              f"{w_e2e:.2e}")
