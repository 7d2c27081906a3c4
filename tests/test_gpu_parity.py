"""Parity of the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (FP32 kernels against the FP64 oracle on identical inputs and identical Philox integers):
  * Philox words: bit-exact.
  * Box-Muller Gaussians: |dz| <= 2e-6 (|z| + 1e-3), from single-rounding errors of logf, sqrtf and
    sincospif on exactly representable uniforms.
  * Control perturbations eps_eff = clamp(v + eps) - v: atol 1e-6 (a few FP32 ulps of |u| <= 3).
  * Particle means and variances of every step: rel 1e-4 / abs 1e-5 (the stated moment tolerance).
  * Trajectory costs S: rel 1e-4 of the cost scale, on samples whose mean e_y stays at least 1e-4
    away from the collision boundary (the C_obs indicator is a jump; a sample within rounding of it
    may legitimately flip and is counted, not compared).
  * Weights from the GPU's own costs (isolates the weight kernel): rel 1e-5 / abs 1e-7.
  * Update from the GPU's own costs and perturbations (isolates the update kernel): rel 1e-4 / abs 1e-5.
  * End-to-end v+ against the oracle's own v+: within abs 1e-5 + rel 1e-4 plus twice the first-order
    bound sum_k w_k |dS_k - <dS>| / lambda |u_k - v+| that the measured cost differences imply.
"""
import numpy as np
import pytest

import oracle
import workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2408_00494_gb300 import bssmppi  # noqa: E402


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def gpu_solve(prob, x0, v, ctr=0, Sigma0=None, record=True, solves=1):
    c = bssmppi.Controller(prob, record_moments=record)
    try:
        bssmppi.set_counter(c.h, ctr)
        xt, vt = _dev(x0), _dev(v)
        S0 = None if Sigma0 is None else _dev(Sigma0)
        u0 = torch.zeros(2, device="cuda")
        for _ in range(solves):
            vt = _dev(v)
            bssmppi.solve(c.h, xt, S0, vt, u0)
        torch.cuda.synchronize()
        out = {"v_plus": vt.cpu().numpy().astype(np.float64), "u0": u0.cpu().numpy().astype(np.float64)}
        for name, buf in (("S", bssmppi.BUF_S), ("w", bssmppi.BUF_W), ("eps", bssmppi.BUF_EPS),
                          ("diag", bssmppi.BUF_DIAG)):
            out[name] = c.buffer(buf).cpu().numpy().astype(np.float64)
        if record:
            out["mean"] = c.buffer(bssmppi.BUF_MEAN).cpu().numpy().astype(np.float64)
            out["var"] = c.buffer(bssmppi.BUF_VAR).cpu().numpy().astype(np.float64)
        out["counter"] = bssmppi.get_counter(c.h)
        return out
    finally:
        c.close()


def assert_close(a, b, rtol, atol, what):
    a, b = np.asarray(a, float), np.asarray(b, float)
    err = np.abs(a - b)
    bad = err > atol + rtol * np.abs(b)
    assert not bad.any(), f"{what}: {bad.sum()} of {bad.size} outside tolerance, max err {err.max():.3e}"


def check_solve(prob, x0, v, ctr=0, Sigma0=None, mean_atol=None, var_atol=None):
    """mean_atol(ref) and var_atol(ref, i) may widen the absolute tolerances of the means and of
    state i's variances. The oracle runs on all host cores (the same results as one thread)."""
    o = oracle.Oracle(prob)
    ref = o.solve(x0, v, ctr, Sigma0=Sigma0, want_cov=True, threads=oracle.host_threads())
    g = gpu_solve(prob, x0, v, ctr, Sigma0=Sigma0)
    T = prob.T
    # control perturbations
    assert_close(g["eps"], ref["eps"], 0.0, 1e-6, "eps_eff")
    # moments of every step
    assert_close(g["mean"], ref["mean"], 1e-4, 1e-5 if mean_atol is None else mean_atol(ref), "particle means")
    ref_var = np.diagonal(ref["cov"], axis1=2, axis2=3)
    for i in range(ref_var.shape[-1]):
        assert_close(g["var"][..., i], ref_var[..., i], 1e-4, 1e-5 if var_atol is None else var_atol(ref, i),
                     f"particle variances of state {i}")
    # costs, away from the collision-indicator jump (FP32 moves the mean e_y by ~1e-6, so only a
    # sample whose mean passes within 1e-4 of the wall can see the indicator decided differently)
    ok = ref["margin"] > 1e-4
    scale = np.maximum(np.abs(ref["S"]), 1.0)
    dS = g["S"] - ref["S"]
    assert np.all(np.abs(dS[ok]) <= 1e-4 * scale[ok]), f"S: max rel err {np.max(np.abs(dS[ok]) / scale[ok]):.3e}"
    # A mean that moves ~0.1 m per step lands within 1e-4 of the wall at a given crossing with
    # probability ~2e-3, so even when every sample crosses, the exclusions stay a small share.
    assert (~ok).sum() <= max(2, prob.K // 100), f"{(~ok).sum()} samples within 1e-4 of the wall"
    # weights from the GPU's costs
    u_gpu = v.astype(np.float64)[None] + g["eps"]
    w_iso, vp_iso, diag_iso = oracle.optimal_control(g["S"], u_gpu, float(np.float32(prob.lam)))
    assert_close(g["w"], w_iso, 1e-5, 1e-7, "weights (from GPU costs)")
    assert_close(g["v_plus"], vp_iso, 1e-4, 1e-5, "v+ (from GPU costs and eps)")
    assert_close(g["u0"], vp_iso[0], 1e-4, 1e-5, "u0")
    assert_close(g["diag"][:3], diag_iso[:3], 1e-4, 1e-6, "diagnostics")
    # end to end, with the bound implied by the measured cost differences
    lam = float(np.float32(prob.lam))
    wr = ref["w"]
    dSc = np.where(ok, dS, 0.0)
    dev = np.abs(dSc - np.sum(wr * dSc)) / lam
    bound = np.einsum("k,kti->ti", wr * dev, np.abs(ref["u"] - ref["v_plus"][None]))
    err = np.abs(g["v_plus"] - ref["v_plus"])
    assert np.all(err <= 1e-5 + 1e-4 * np.abs(ref["v_plus"]) + 2 * bound), f"v+ e2e max err {err.max():.3e}"
    assert g["counter"] == ctr + 1
    rel = lambda a, b: float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-3)))
    print(f"[parity K={prob.K} M={prob.M} T={prob.T}] S max rel {np.max(np.abs(dS[ok]) / scale[ok]):.2e}; "
          f"mean max abs {np.abs(g['mean'] - ref['mean']).max():.2e}; var max abs {np.abs(g['var'] - ref_var).max():.2e}; "
          f"v+ iso max rel {rel(g['v_plus'], vp_iso):.2e}; v+ e2e max abs {err.max():.2e} (bound {bound.max():.2e}); "
          f"indicator-margin exclusions {(~ok).sum()}")
    return g, ref


def test_philox_bit_exact():
    rng = np.random.default_rng(0)
    n = 1 << 20
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    # the layout the solve uses: steps, calls, particles, samples, streams, counters
    ctr[:4096, 0] = np.arange(4096) % 256 | ((np.arange(4096) // 256 % 2) << 16)
    ctr[:4096, 3] = (np.arange(4096) % 4 << 28) | 7
    for seed in (0, 0x0123456789ABCDEF):
        key = (seed & 0xFFFFFFFF, seed >> 32)
        out = torch.zeros(n * 4, dtype=torch.int32, device="cuda")
        bssmppi.philox4x32_10(torch.as_tensor(ctr.view(np.int32).reshape(-1), device="cuda"), seed, out)
        gpu = out.cpu().numpy().view(np.uint32).reshape(n, 4)
        ref = oracle.philox_batch(ctr, key)
        assert np.array_equal(gpu, ref)


def test_box_muller_matches_oracle():
    rng = np.random.default_rng(1)
    n = 1 << 16
    words = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    words[:4] = [[0xFFFFFFFF, 0], [0, 0], [0, 1 << 30], [0x000000FF, 0xFFFFFFFF]]
    z = torch.zeros(2 * n, dtype=torch.float32, device="cuda")
    bssmppi.box_muller(torch.as_tensor(words.view(np.int32).reshape(-1), device="cuda"), z)
    zg = z.cpu().numpy().reshape(n, 2).astype(np.float64)
    zr = np.array([oracle.gaussian_pair(int(a), int(b)) for a, b in words])
    r = np.hypot(zr[:, 0], zr[:, 1])
    assert np.all(np.abs(zg - zr) <= 2e-6 * (r[:, None] + 1e-3))
    assert zg[0, 0] == 0.0 and zg[0, 1] == 0.0


def test_slip_angle_arctangent_within_an_ulp():
    """The substeps' slip-angle arctangent against atan in FP64: within one FP32 ulp on the
    polynomial's range |t| <= 1/2 (the fit gives 0.72), within the library atanf's documented 2 ulp
    beyond it, exact at 0 and odd."""
    pos = np.linspace(0.0, 0.5, 1 << 19, dtype=np.float32)
    inner = np.concatenate([pos, -pos])
    edge = np.nextafter(np.float32(0.5), np.float32([0.0, 1.0])).astype(np.float32)
    outer = np.concatenate([np.geomspace(0.5, 1e6, 1 << 16), -np.geomspace(0.5, 1e6, 1 << 16)]).astype(np.float32)
    t = np.concatenate([inner, edge, -edge, outer, np.float32([0.0, 1e-30, -1e-30])])
    y = torch.zeros(t.size, device="cuda")
    bssmppi.slip_atan(_dev(t), y)
    y = y.cpu().numpy()
    ref = np.arctan(t.astype(np.float64))
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    err = np.abs(y - ref) / ulp
    small = np.abs(t) <= 0.5
    assert err[small].max() <= 1.0, err[small].max()
    assert err[~small].max() <= 2.0, err[~small].max()
    assert y[t == 0].max() == 0.0
    n = pos.size
    assert np.array_equal(y[:n], -y[n:2 * n])


@pytest.mark.parametrize("C", [1.9, 1.6])
def test_tyre_curve_against_fp64(C):
    """The substep's tyre curve sin(C atan x): the polynomial on |x| <= 1 within 4e-7 of FP64 (and
    odd bit for bit), the library route beyond within 2e-6 (atanf's 2 ulp times C, plus the hardware
    sine's 2^-21.4)."""
    p = workload.wheels_problem(8, 4, 3) if C == 1.6 else workload.config0()
    assert abs(p.tire_C - C) < 1e-12
    c = bssmppi.Controller(p)
    pos = np.linspace(0.0, 1.0, 1 << 18, dtype=np.float32)
    inner = np.concatenate([pos, -pos])
    outer = np.concatenate([np.geomspace(1.0, 1e4, 1 << 14), -np.geomspace(1.0, 1e4, 1 << 14)]).astype(np.float32)
    outer = outer[np.abs(outer) > 1.0]
    x = np.concatenate([inner, outer])
    y = torch.zeros(x.size, device="cuda")
    bssmppi.tyre_curve(c.h, _dev(x), y)
    c.close()
    y = y.cpu().numpy().astype(np.float64)
    ref = np.sin(float(np.float32(C)) * np.arctan(x.astype(np.float64)))
    n = inner.size
    assert np.abs(y[:n] - ref[:n]).max() <= 4e-7, np.abs(y[:n] - ref[:n]).max()
    assert np.abs(y[n:] - ref[n:]).max() <= 2e-6, np.abs(y[n:] - ref[n:]).max()
    assert np.array_equal(y[:n // 2], -y[n // 2:n])


@pytest.mark.parametrize("which", ["bicycle", "wheels"])
def test_rear_tyre_against_fp64(which):
    """The substep's rear tyre curve sin(C atan(-B atan t)) as one polynomial in t / tau, taken in
    packed pairs as the solve takes them: within 4e-7 of FP64 on |t| < tau (and odd bit for bit); the
    route beyond (slip_atan, then the library's atanf and hardware sine) within 3e-6 (B times the
    slip angle's ulp through the tyre curve, plus atanf's and the sine's errors); pairs with one
    value on each side take each value's own route."""
    p = workload.config0() if which == "bicycle" else workload.wheels_problem(8, 4, 3)
    B, C = float(np.float32(p.tire_B)), float(np.float32(p.tire_C))
    _, tau = bssmppi.rear_tyre_coefficients(B, C)
    pos = np.linspace(0.0, tau * (1.0 - 1e-6), 1 << 18).astype(np.float32)
    inner = np.concatenate([pos, -pos])
    far = np.concatenate([np.geomspace(tau * 1.0001, 1e4, 1 << 14), -np.geomspace(tau * 1.0001, 1e4, 1 << 14)])
    far = far.astype(np.float32)
    mixed = np.stack([pos[::16][:far.size // 2], far[:far.size // 2]], axis=1).reshape(-1)
    t = np.concatenate([inner, far, mixed])
    c = bssmppi.Controller(p)
    y = torch.zeros(t.size, device="cuda")
    bssmppi.rear_tyre(c.h, _dev(t), y)
    c.close()
    y = y.cpu().numpy().astype(np.float64)
    ref = np.sin(C * np.arctan(-B * np.arctan(t.astype(np.float64))))
    n, m = inner.size, inner.size + far.size
    assert np.abs(y[:n] - ref[:n]).max() <= 4e-7, np.abs(y[:n] - ref[:n]).max()
    assert np.abs(y[n:m] - ref[n:m]).max() <= 3e-6, np.abs(y[n:m] - ref[n:m]).max()
    assert np.abs(y[m:] - ref[m:]).max() <= 3e-6, np.abs(y[m:] - ref[m:]).max()
    assert np.array_equal(y[:n // 2], -y[n // 2:n])


@pytest.mark.parametrize("model", ["bicycle", "double_integrator"])
def test_model_step_matches_oracle(model):
    if model == "bicycle":
        p = workload.config1()
    else:
        p = workload.double_integrator_problem(1, 2, 1)
    c = bssmppi.Controller(p)
    o = oracle.Oracle(p)
    n = 4096
    xs = np.stack([workload.random_state(p, i) for i in range(n)])
    if model == "bicycle":  # heading errors on both sides of the series' range |e_psi| <= pi/4, and
        # several turns away (the fallback's reduction by multiples of 2 pi)
        xs[n // 2:, 3] = np.linspace(-1.5, 1.5, n - n // 2, dtype=np.float32)
        xs[n // 4: n // 2, 3] = np.linspace(-40.0, 40.0, n // 4, dtype=np.float32)
    us = np.stack([workload.random_nominal(p, i)[0] for i in range(n)]) * 3.0
    us = np.clip(us, p.u_min, p.u_max).astype(np.float32)
    out = torch.zeros((n, p.nx), device="cuda")
    bssmppi.model_step(c.h, _dev(xs), _dev(us), out)
    g = out.cpu().numpy().astype(np.float64)
    ref = np.stack([o.model_step(xs[i].astype(np.float64), us[i].astype(np.float64)) for i in range(n)])
    assert_close(g, ref, 2e-5, 2e-5, "model step")
    # with an additive disturbance: x_next = f(x, u) + w
    w = np.random.default_rng(2).normal(0, 0.1, size=xs.shape).astype(np.float32)
    out_w = torch.zeros((n, p.nx), device="cuda")
    bssmppi.model_step(c.h, _dev(xs), _dev(us), out_w, _dev(w))
    c.close()
    assert np.array_equal(out_w.cpu().numpy(), (out.cpu().numpy() + w).astype(np.float32))


def test_solve_config0_from_start():
    p = workload.config0()
    check_solve(p, workload.racing_x0(p), np.zeros((p.T, 2), np.float32), ctr=0)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_solve_config0_random_states(seed):
    p = workload.config0()
    check_solve(p, workload.random_state(p, seed), workload.random_nominal(p, seed), ctr=100 + seed)


@pytest.mark.parametrize("M", [2, 5, 20, 32, 50, 64, 128])
def test_solve_particle_counts(M):
    """Segments narrower than a warp, ragged lanes (M not a multiple of the segment) and P > 1."""
    p = workload.config0()
    p.K, p.M, p.T = 200, M, 12
    check_solve(p, workload.random_state(p, M), workload.random_nominal(p, M), ctr=M)


def check_unrecorded(prob, x0, v, ctr):
    """A solve that keeps no moments (the launch the benchmark and the controllers use) against the
    oracle: every sample's perturbations and cost, the weights from the GPU's costs, and v+ and u0
    isolated and end to end."""
    g = gpu_solve(prob, x0, v, ctr, record=False)
    ref = oracle.Oracle(prob).solve(x0, v, ctr, threads=oracle.host_threads())
    assert_close(g["eps"], ref["eps"], 0.0, 1e-6, "eps_eff")
    ok = ref["margin"] > 1e-4
    assert (~ok).sum() <= max(2, prob.K // 100), f"{(~ok).sum()} samples within 1e-4 of the wall"
    scale = np.maximum(np.abs(ref["S"]), 1.0)
    dS = g["S"] - ref["S"]
    assert np.all(np.abs(dS[ok]) <= 1e-4 * scale[ok]), f"S: max rel err {np.max(np.abs(dS[ok]) / scale[ok]):.3e}"
    lam = float(np.float32(prob.lam))
    w_iso, vp_iso, _ = oracle.optimal_control(g["S"], v.astype(np.float64)[None] + g["eps"], lam)
    assert_close(g["w"], w_iso, 1e-5, 1e-7, "weights (from GPU costs)")
    assert_close(g["v_plus"], vp_iso, 1e-4, 1e-5, "v+ (from GPU costs and eps)")
    assert_close(g["u0"], vp_iso[0], 1e-4, 1e-5, "u0")
    dSc = np.where(ok, dS, 0.0)
    dev = np.abs(dSc - np.sum(ref["w"] * dSc)) / lam
    bound = np.einsum("k,kti->ti", ref["w"] * dev, np.abs(ref["u"] - ref["v_plus"][None]))
    err = np.abs(g["v_plus"] - ref["v_plus"])
    assert np.all(err <= 1e-5 + 1e-4 * np.abs(ref["v_plus"]) + 2 * bound), f"v+ e2e max err {err.max():.3e}"
    assert g["counter"] == ctr + 1


@pytest.mark.parametrize("M", [2, 16, 50, 64, 96, 256])
@pytest.mark.parametrize("compensated", [1, 0])
def test_unrecorded_solve_particle_counts(M, compensated):
    """Without recording, a cost that weights only v_x, e_psi and e_y (the racing cost) runs a build
    that merges those three means only (compensated), or the run-time set of the plain sums (naive):
    segments narrower than a warp, full warps, ragged lanes and one to eight particles per lane."""
    p = workload.config0()
    p.K, p.M, p.T, p.compensated = 200, M, 12, compensated
    check_unrecorded(p, workload.random_state(p, 300 + M), workload.random_nominal(p, 300 + M), ctr=M + 5)


@pytest.mark.parametrize("K,M", [(4096, 32), (4096, 20), (8192, 16), (16384, 8)])
def test_two_particles_per_lane_mapping(K, M):
    """From 8 to 32 particles a solve with enough samples for about 12 warps per SM runs two
    particles per lane in segments of the next power of two >= M / 2 lanes (ragged at M = 20): the
    recorded solve (every step's means and variances) and the unrecorded one (the racing-cost build)
    against the oracle."""
    p = workload.config0()
    p.K, p.M, p.T = K, M, 10
    x0, v = workload.random_state(p, 500 + M), workload.random_nominal(p, 500 + M)
    check_solve(p, x0, v, ctr=M + 1)
    check_unrecorded(p, x0, v, ctr=M + 2)


@pytest.mark.parametrize("K,M", [(4096, 32), (4096, 20)])
def test_two_particles_per_lane_mapping_naive_sums(K, M):
    """The same mapping with the naive (uncompensated) reductions, unrecorded, against the oracle."""
    p = workload.config0()
    p.K, p.M, p.T, p.compensated = K, M, 10, 0
    x0, v = workload.random_state(p, 600 + M), workload.random_nominal(p, 600 + M)
    check_unrecorded(p, x0, v, ctr=M + 3)


def test_unrecorded_solve_with_every_state_weighted():
    """A cost that weights every state (the build with the run-time set of merged means)."""
    p = workload.config0()
    p.K, p.M, p.T = 200, 64, 12
    p.Q = p.Qf = (1.0, 0.5, 0.2, 1.0, 0.1, 1e-4)
    check_unrecorded(p, workload.random_state(p, 41), workload.random_nominal(p, 41), ctr=9)


@pytest.mark.parametrize("model,K,M,T", [("double_integrator", 70, 2, 256), ("bicycle", 70, 2, 64),
                                         ("bicycle", 40, 256, 6), ("bicycle", 33, 3, 7)])
def test_solve_extreme_shapes(model, K, M, T):
    """Sixteen samples per warp over the longest horizon, the largest particle count (8 per lane),
    and a ragged odd case. The 256-step horizon runs on the linear model: with open-loop controls
    for 12.8 s the vehicle leaves the track and nears the road-frame singularity 1 - kappa e_y = 0,
    where FP32 and FP64 trajectories separate for reasons of conditioning, not of the kernel."""
    if model == "bicycle":
        p = workload.config0()
        p.K, p.M, p.T = K, M, T
    else:
        p = workload.double_integrator_problem(K, M, T)
    check_solve(p, workload.random_state(p, K), workload.random_nominal(p, K), ctr=K)


def test_maximum_sample_count_sampled_parity():
    """K = BSSMPPI_K_MAX = 2^20 samples (65,536 groups of 16 two-particle samples per warp, through
    the persistent grid and its 152-block tail): sampled perturbations and costs against the oracle,
    the weights and update against the oracle's from the GPU's own costs."""
    p = workload.config0()
    p.K, p.M, p.T = 1 << 20, 2, 3
    x0, v = workload.random_state(p, 9), workload.random_nominal(p, 9)
    g = gpu_solve(p, x0, v, ctr=1, record=False)
    o = oracle.Oracle(p)
    for k in (0, 1, 15, 16, 777777, p.K - 1):
        r = o.solve(x0, v, 1, k_range=(k, k + 1))
        assert_close(g["eps"][k], r["eps"][k], 0.0, 1e-6, f"eps[{k}]")
        if r["margin"][k] > 1e-3:
            assert abs(g["S"][k] - r["S"][k]) <= 1e-4 * max(1.0, abs(r["S"][k])), k
    u_gpu = v.astype(np.float64)[None] + g["eps"]
    w_iso, vp_iso, _ = oracle.optimal_control(g["S"], u_gpu, float(np.float32(p.lam)))
    assert_close(g["w"], w_iso, 1e-5, 1e-7, "weights")
    assert_close(g["v_plus"], vp_iso, 1e-4, 1e-5, "v+")
    assert g["counter"] == 2


@pytest.mark.parametrize("n_track,M,T", [(2, 16, 20), (16384, 256, 32)])
def test_curvature_table_sizes(n_track, M, T):
    """The smallest curvature table (two entries) and the largest (BSSMPPI_NTRACK_MAX = 2^14
    entries: 128 KiB of (value, difference) pairs staged in shared memory beside the largest particle
    count's buffers)."""
    p = workload.config0()
    p.M, p.T = M, T
    p.kappa, p.track_len = workload.make_track(7, n_s=n_track)
    check_solve(p, workload.random_state(p, 3), workload.random_nominal(p, 3), ctr=2)


@pytest.mark.parametrize("case", ["no_disturbance", "small_lambda", "large_lambda", "gamma_near_0",
                                  "gamma_near_1", "delta_near_half", "delta_small"])
def test_solve_degenerate_settings(case):
    """The method's limiting settings against the oracle: no disturbance (every particle identical,
    so the belief collapses to a point: zero variance, and the barrier is the deterministic one),
    lambda -> 0 (the weights pick the best sample) and large (near-uniform weights), gamma at both
    ends of (0, 1), and chance levels delta near 1/2 (nu -> 0, no back-off) and small (large nu)."""
    p = workload.config0()
    if case == "no_disturbance":
        p.Sigma_w = np.zeros_like(np.asarray(p.Sigma_w))
    elif case == "small_lambda":
        p.lam = 1e-3
    elif case == "large_lambda":
        p.lam = 1e4
    elif case == "gamma_near_0":
        p.gamma = 1e-3
    elif case == "gamma_near_1":
        p.gamma = 0.999
    elif case == "delta_near_half":
        p.delta = 0.499
    elif case == "delta_small":
        p.delta = 1e-4
    x0, v = workload.random_state(p, 31), workload.random_nominal(p, 31)
    g, ref = check_solve(p, x0, v, ctr=5)
    if case == "no_disturbance":
        assert np.all(g["var"] == 0.0)
    lam = float(np.float32(p.lam))
    S = np.sort(g["S"])
    if case == "small_lambda":
        # Eq. "Weights" gives w_best = 1 / (1 + sum_{k != best} exp(-(S_k - S_min)/lambda)), at least
        # 1 / (1 + (K - 1) exp(-gap/lambda)) with gap the two lowest costs' difference: the weights
        # reach the argmin limit as gap/lambda grows (here gap/lambda is printed)
        bound = 1.0 / (1.0 + (p.K - 1) * np.exp(-(S[1] - S[0]) / lam))
        print(f"[degenerate] lambda={lam:g}: gap/lambda {(S[1] - S[0]) / lam:.1f}, w_best {g['w'].max():.6f}")
        assert g["w"][np.argmin(g["S"])] >= bound * (1 - 1e-5) - 1e-7
    if case == "large_lambda":
        # every omega lies in [exp(-R/lambda), 1] with R the cost range, so the effective sample size
        # (sum w)^2 / sum w^2 is at least K exp(-2R/lambda): it tends to K as lambda grows
        w = g["w"] / g["w"].sum()
        ess, bound = 1.0 / np.sum(w * w), p.K * np.exp(-2.0 * (S[-1] - S[0]) / lam)
        print(f"[degenerate] lambda={lam:g}: ESS {ess:.1f} of K={p.K}, bound {bound:.1f}")
        assert ess >= bound * (1 - 1e-5)


@pytest.mark.parametrize("backoff,clamp", [(1, 0), (0, 1), (1, 1)])
def test_solve_backoff_and_clamped_margin(backoff, clamp):
    """Remark 1's Cantelli back-off and the clamped barrier margin max(w_T - nu sigma, 0) against the
    oracle: a 1 m half-width with a lateral disturbance of 0.1 m per step, so that Cantelli's
    back-off (nu = 4.36) passes the half-width within the horizon and the clamp decides h."""
    p = workload.config0()
    p.K, p.M, p.T = 256, 32, 20
    p.w_T, p.backoff, p.clamp_margin = 1.0, backoff, clamp
    p.Sigma_w = np.diag(np.array([0.02, 0.02, 0.01, 0.002, 0.1, 0.0]) ** 2)
    x0 = workload.random_state(p, 41)
    x0[3], x0[4] = 0.0, 0.0
    g, ref = check_solve(p, x0, workload.random_nominal(p, 41), ctr=12)
    if backoff:
        nu = float(np.sqrt((1 - np.float32(p.delta)) / np.float32(p.delta)))
        assert np.any(nu * np.sqrt(ref["cov"][:, :, 4, 4]) > 1.0)  # the margin is negative somewhere


def test_solve_ragged_K_and_long_horizon():
    p = workload.config1()
    p.K, p.M, p.T = 1001, 64, 40
    check_solve(p, workload.random_state(p, 5), workload.random_nominal(p, 5), ctr=3)


def test_solve_single_sample_and_single_step():
    p = workload.config0()
    p.K, p.M, p.T = 1, 16, 1
    g, ref = check_solve(p, workload.random_state(p, 6), workload.random_nominal(p, 6), ctr=0)
    assert g["w"][0] == 1.0


def test_solve_with_initial_covariance():
    p = workload.config0()
    p.K, p.T = 128, 10
    Sig0 = np.diag([0.05, 0.01, 0.01, 0.001, 0.04, 0.1]).astype(np.float32) ** 2
    check_solve(p, workload.random_state(p, 7), workload.random_nominal(p, 7), ctr=9, Sigma0=Sig0)


def test_solve_common_random_numbers():
    p = workload.config0()
    p.K, p.T = 96, 15
    p.crn_disturbance = 1
    check_solve(p, workload.random_state(p, 8), workload.random_nominal(p, 8), ctr=4)


def test_solve_near_boundary_with_active_barrier():
    p = workload.config0()
    p.K, p.T = 256, 20
    x0 = workload.random_state(p, 9)
    x0[4], x0[3] = 2.6, 0.3
    g, ref = check_solve(p, x0, workload.random_nominal(p, 9), ctr=2)
    one_m_gamma = 1.0 - float(np.float32(p.gamma))
    assert np.any(-ref["h"][:, 1:] + one_m_gamma * ref["h"][:, :-1] > 0)  # the DCBF penalty is active


def test_solve_double_integrator():
    p = workload.double_integrator_problem(K=300, M=40, T=16)
    check_solve(p, workload.random_state(p, 10), workload.random_nominal(p, 10), ctr=5)


def test_consecutive_solves_advance_counter():
    p = workload.config0()
    p.K, p.T = 64, 8
    x0, v = workload.random_state(p, 11), workload.random_nominal(p, 11)
    g = gpu_solve(p, x0, v, ctr=41, solves=2)
    ref = oracle.Oracle(p).solve(x0, v, 42)
    assert g["counter"] == 43
    assert_close(g["eps"], ref["eps"], 0.0, 1e-6, "eps of the second solve")


def test_shift_matches_definition():
    p = workload.config0()
    c = bssmppi.Controller(p)
    v = workload.random_nominal(p, 12)
    for n in (1, 3, p.T):
        vt = _dev(v)
        bssmppi.shift(c.h, vt, n)
        exp = v[np.minimum(np.arange(p.T) + n, p.T - 1)]
        assert np.array_equal(vt.cpu().numpy(), exp)
    c.close()


@pytest.mark.parametrize("case", ["plain", "sigma0", "resident", "wheels8"])
def test_solve_host_matches_device_path(case):
    """The host-buffer solve (one H2D of x0 | v | Sigma0, one D2H of v+ | u0) gives bit for bit the
    device-buffer solve's v+ and u0."""
    p = workload.wheels_problem(96, 16, 12) if case == "wheels8" else workload.config0()
    x0, v = workload.random_state(p, 13), workload.random_nominal(p, 13)
    Sig0 = None
    if case in ("sigma0", "wheels8"):
        Sig0 = (np.eye(p.nx) * 0.01).astype(np.float32)
        Sig0[0, 1] = Sig0[1, 0] = 0.002
    g = gpu_solve(p, x0, v, ctr=7, Sigma0=Sig0, record=False)
    c = bssmppi.Controller(p)
    try:
        bssmppi.set_counter(c.h, 7)
        u0 = np.zeros(2, np.float32)
        if case == "resident":
            bssmppi.set_nominal(c.h, _dev(v))
            bssmppi.solve_host(c.h, x0.astype(np.float32), None, None, u0)
            vh = c.buffer(bssmppi.BUF_V).cpu().numpy()
        else:
            vh = v.copy()
            bssmppi.solve_host(c.h, x0.astype(np.float32), Sig0, vh, u0)
    finally:
        c.close()
    assert np.array_equal(vh.astype(np.float64), g["v_plus"])
    assert np.array_equal(u0.astype(np.float64), g["u0"])


def test_host_solve_graph_follows_the_handle_state():
    """The host-buffer solve replays a captured graph (H2D, solve kernel, D2H). Replays must read the
    current solve counter and nominal, a new constraint set must replace the graph (the kernel takes
    the set by value), and with timing events on the plain path must run: each result equals the
    device-buffer solve of the same state bit for bit."""
    p = workload.config0()
    x0, v = workload.random_state(p, 21), workload.random_nominal(p, 21)
    cons = (workload.halfspace((0, 0, 0, 0, 1, 0), p.w_T, p.delta),
            workload.disk(5, 4, (float(x0[5]) + 5.0, 0.2), 0.8, 0.05))
    c = bssmppi.Controller(p)
    try:
        bssmppi.set_counter(c.h, 7)
        got = []
        for step in range(4):
            if step == 2:
                bssmppi.set_constraints(c.h, cons)
            if step == 3:
                bssmppi.timing(c.h, 2)
            vh, u0 = v.copy(), np.zeros(2, np.float32)
            bssmppi.solve_host(c.h, x0.astype(np.float32), None, vh, u0)
            got.append((vh.astype(np.float64), u0.astype(np.float64)))
        roll_ms, _ = bssmppi.timing_read(c.h, 2)
        assert len(roll_ms) == 1 and roll_ms[0] > 0.0
    finally:
        c.close()
    for step, (vh, u0) in enumerate(got):
        q = workload.config0()
        if step >= 2:
            q.constraints = cons
        g = gpu_solve(q, x0, v, ctr=7 + step, record=False)
        assert np.array_equal(vh, g["v_plus"]), step
        assert np.array_equal(u0, g["u0"]), step


def test_full_size_config1_sampled_parity():
    """The benchmark's workload and launch configuration (K=4096, M=64, T=40, moments not kept):
    sampled costs and perturbations against the oracle sample by sample, the update against the
    oracle's update from the GPU's costs, and properties of the weights."""
    p = workload.config1()
    x0, v = workload.random_state(p, 14), workload.random_nominal(p, 14)
    g = gpu_solve(p, x0, v, ctr=123, record=False)
    o = oracle.Oracle(p)
    picks = [0, 1, 31, 32, 1000, 2047, 4064, 4095]
    for k in picks:
        r = o.solve(x0, v, 123, k_range=(k, k + 1))
        assert_close(g["eps"][k], r["eps"][k], 0.0, 1e-6, f"eps[{k}]")
        if r["margin"][k] > 1e-3:
            assert abs(g["S"][k] - r["S"][k]) <= 1e-4 * max(1.0, abs(r["S"][k])), k
    u_gpu = v.astype(np.float64)[None] + g["eps"]
    w_iso, vp_iso, _ = oracle.optimal_control(g["S"], u_gpu, float(np.float32(p.lam)))
    assert_close(g["w"], w_iso, 1e-5, 1e-7, "weights")
    assert_close(g["v_plus"], vp_iso, 1e-4, 1e-5, "v+")
    assert abs(g["w"].sum() - 1.0) < 1e-5 and g["w"].min() >= 0.0
    lo, hi = np.asarray(p.u_min), np.asarray(p.u_max)
    assert np.all(u_gpu >= lo - 1e-6) and np.all(u_gpu <= hi + 1e-6)


@pytest.mark.parametrize("n", [0, 1, 3, 20])
def test_solve_shift_equals_solve_then_shift(n):
    """The fused call leaves the resident nominal and u0 exactly as a solve followed by a shift."""
    p = workload.config0()
    x0, v = workload.random_state(p, 17), workload.random_nominal(p, 17)
    out = []
    for fused in (False, True):
        c = bssmppi.Controller(p)
        try:
            bssmppi.set_counter(c.h, 4)
            bssmppi.set_nominal(c.h, _dev(v))
            u0 = torch.zeros(2, device="cuda")
            xt = _dev(x0)
            if fused:
                bssmppi.solve_shift(c.h, xt, None, u0, n)
            else:
                bssmppi.solve(c.h, xt, None, None, u0)
                bssmppi.shift(c.h, None, n)
            out.append((c.buffer(bssmppi.BUF_V).cpu().numpy(), u0.cpu().numpy(), bssmppi.get_counter(c.h)))
        finally:
            c.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] == 5


def test_full_size_config1_whole_solve_parity():
    """The benchmark's workload (K=4096, M=64, T=40, disturbance x2) compared on every sample: the
    perturbations, the costs, the means and variances of every step, the weights and the update
    (isolated and end to end against the oracle's own v+)."""
    p = workload.config1()
    check_solve(p, workload.random_state(p, 14), workload.random_nominal(p, 14), ctr=123)


def test_full_size_config1_benchmark_launch_parity():
    """The launch the benchmark times: solve and warm-start shift in one launch on the resident
    nominal, moments not kept. Every sample's perturbations and cost, the weights, u0 and the
    shifted nominal against the oracle's solve followed by its shift."""
    p = workload.config1()
    x0, v = workload.random_state(p, 15), workload.random_nominal(p, 15)
    c = bssmppi.Controller(p)
    try:
        bssmppi.set_counter(c.h, 77)
        bssmppi.set_nominal(c.h, _dev(v))
        u0 = torch.zeros(2, device="cuda")
        bssmppi.solve_shift(c.h, _dev(x0), None, u0, 1)
        torch.cuda.synchronize()
        S, w = c.buffer(bssmppi.BUF_S).cpu().numpy().astype(np.float64), c.buffer(bssmppi.BUF_W).cpu().numpy()
        eps = c.buffer(bssmppi.BUF_EPS).cpu().numpy().astype(np.float64)
        v_shift = c.buffer(bssmppi.BUF_V).cpu().numpy().astype(np.float64)
        u0 = u0.cpu().numpy().astype(np.float64)
    finally:
        c.close()
    ref = oracle.Oracle(p).solve(x0, v, 77, threads=oracle.host_threads())
    assert_close(eps, ref["eps"], 0.0, 1e-6, "eps_eff")
    ok = ref["margin"] > 1e-4
    assert (~ok).sum() <= max(2, p.K // 100)
    assert np.all(np.abs(S - ref["S"])[ok] <= 1e-4 * np.maximum(np.abs(ref["S"][ok]), 1.0))
    lam = float(np.float32(p.lam))
    w_iso, vp_iso, _ = oracle.optimal_control(S, v.astype(np.float64)[None] + eps, lam)
    assert_close(w, w_iso, 1e-5, 1e-7, "weights (from GPU costs)")
    dS = np.where(ok, S - ref["S"], 0.0)
    dev = np.abs(dS - np.sum(ref["w"] * dS)) / lam
    bound = np.einsum("k,kti->ti", ref["w"] * dev, np.abs(ref["u"] - ref["v_plus"][None]))
    vp_ref = ref["v_plus"].copy()
    err_u0 = np.abs(u0 - vp_ref[0])
    assert np.all(err_u0 <= 1e-5 + 1e-4 * np.abs(vp_ref[0]) + 2 * bound[0]), err_u0
    shifted_ref = vp_ref.copy()
    shifted_bound = bound.copy()
    for arr in (shifted_ref, shifted_bound):
        arr[:-1] = arr[1:].copy()
    err = np.abs(v_shift - shifted_ref)
    assert np.all(err <= 1e-5 + 1e-4 * np.abs(shifted_ref) + 2 * shifted_bound), f"shifted v+ max err {err.max():.3e}"
    print(f"[bench-launch parity K={p.K} M={p.M} T={p.T}] S max rel "
          f"{np.max(np.abs(S - ref['S'])[ok] / np.maximum(np.abs(ref['S'][ok]), 1.0)):.2e}, u0 err {err_u0.max():.2e}, "
          f"shifted v+ max err {err.max():.2e} (bound {shifted_bound.max():.2e})")


@pytest.mark.parametrize("lam", [0.1, 1.0, 10.0])
def test_full_size_config3_whole_solve_parity(lam):
    """The precision study's scale (K=16384, M=128, T=60) on every sample, for each temperature:
    perturbations, costs, the means and variances of every step, weights and update, and the
    end-to-end v+ against the oracle's own within the first-order |dS|/lambda bound."""
    p = workload.config3(lam)
    v = np.zeros((p.T, 2), np.float32)
    v[:, 0] = (p.lf + p.lr) * 2 * np.pi / p.track_len  # follows the mean curvature
    check_solve(p, workload.racing_x0(p), v, ctr=6)
