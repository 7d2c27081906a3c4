"""Seeded synthetic inputs for the BSS-MPPI solve: race tracks, problem constants, initial states.

This module is the only code shared by the FP64 oracle's tests and the CUDA path's tests and
benchmark. It produces inputs only: it holds none of the controller's arithmetic (no dynamics,
no sampling, no costs, no weights). Everything here is plain numpy in FP64, seeded by
``numpy.random.default_rng``.

Track (a stand-in for the paper's race course, Sec. V-A; the AutoRally track itself is not
available): a closed curve in polar form r(theta) = R + sum_{j=2..6} A_j cos(j theta + phi_j) with
A_j ~ U(0, 1.2) m (so the radial perturbation is at most 6 m) and phi_j ~ U(0, 2 pi). The centre
line is re-parametrised by arc length s and its signed curvature kappa(s) is tabulated on n_s
uniform points of [0, L). Both the oracle and the CUDA path receive that table (as float32) and
interpolate it linearly with wrap-around.

Problem constants follow the racing configurations used throughout the tests and the benchmark:
6-state dynamic bicycle [v_x, v_y, yaw rate r, heading error e_psi, lateral error e_y, progress s],
controls [steer, accel] bounded by +-0.4 rad and +-3 m/s^2, dt = 0.05 s, m = 1500 kg,
Iz = 2500 kg m^2, l_f = 1.2 m, l_r = 1.4 m, Pacejka B = 10, C = 1.9, D = mu F_z with mu = 1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

NU = 2
MODEL_BICYCLE6 = 0
MODEL_DOUBLE_INT4 = 1
MODEL_WHEELS8 = 2


def make_track(seed: int, radius: float = 60.0, n_s: int = 4096, n_theta: int = 1 << 16,
               amp_max: float = 1.2):
    """Curvature table kappa[n_s] (float32) and length L (m) of a seeded Fourier-perturbed circle.

    Arc length uses the periodic trapezoid rule on n_theta points (spectrally accurate for a
    smooth periodic integrand); the polar-curve curvature formula
    kappa = (r^2 + 2 r'^2 - r r'') / (r^2 + r'^2)^{3/2} is evaluated analytically at theta(s).
    """
    rng = np.random.default_rng(seed)
    js = np.arange(2, 7, dtype=np.float64)
    amp = rng.uniform(0.0, amp_max, size=js.size)
    phase = rng.uniform(0.0, 2.0 * math.pi, size=js.size)

    def radial(th):
        th = np.asarray(th, dtype=np.float64)[..., None]
        c = np.cos(js * th + phase)
        s = np.sin(js * th + phase)
        r = radius + (amp * c).sum(-1)
        dr = (-amp * js * s).sum(-1)
        ddr = (-amp * js * js * c).sum(-1)
        return r, dr, ddr

    theta = np.arange(n_theta, dtype=np.float64) * (2.0 * math.pi / n_theta)
    r, dr, _ = radial(theta)
    speed = np.sqrt(r * r + dr * dr)  # ds/dtheta
    h = 2.0 * math.pi / n_theta
    cum = np.concatenate([[0.0], np.cumsum(0.5 * h * (speed + np.roll(speed, -1)))])
    length = float(cum[-1])
    theta_ext = np.concatenate([theta, [2.0 * math.pi]])
    s_grid = np.arange(n_s, dtype=np.float64) * (length / n_s)
    th_s = np.interp(s_grid, cum, theta_ext)
    r, dr, ddr = radial(th_s)
    kappa = (r * r + 2.0 * dr * dr - r * ddr) / np.power(r * r + dr * dr, 1.5)
    return kappa.astype(np.float32), length


@dataclasses.dataclass
class Problem:
    """One controller's problem constants (names follow the paper where it gives them)."""

    K: int = 256                 # control samples (the paper's M)
    M: int = 16                  # disturbance particles per sample (the paper's N)
    T: int = 20                  # horizon steps (the paper's K)
    n_sub: int = 5               # explicit-Euler substeps per dt
    model: int = MODEL_BICYCLE6
    dt: float = 0.05
    mass: float = 1500.0
    Iz: float = 2500.0
    lf: float = 1.2
    lr: float = 1.4
    tire_B: float = 10.0
    tire_C: float = 1.9
    mu: float = 1.0
    g: float = 9.81
    vx_floor: float = 1.0
    wheel_radius: float = 0.3        # wheel-speed model (model 2) only
    wheel_inertia: float = 1.0
    mu_x: float = 1.0
    tau_max: float = 0.0
    slip_floor: float = 2.0
    u_min: tuple = (-0.4, -3.0)
    u_max: tuple = (0.4, 3.0)
    Sigma_eps: np.ndarray = None     # 2x2 control-noise covariance
    Sigma_w: np.ndarray = None       # nx x nx disturbance covariance (PSD)
    lam: float = 1.0                 # temperature lambda
    delta: float = 0.05              # per-boundary chance level
    gamma: float = 0.3               # DCBF decay rate (the paper's beta in (1 - beta))
    ctrl_w: float = 1.0              # weight of v^T Sigma_eps^-1 u in S (the paper's gamma)
    C_safe: float = 100.0            # safe-violation weight C
    C_obs: float = 1000.0            # collision penalty
    w_T: float = 3.0                 # track half-width
    x_goal: tuple = (10.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    Q: tuple = (1.0, 0.0, 0.0, 1.0, 0.1, 0.0)
    Qf: tuple = (1.0, 0.0, 0.0, 1.0, 0.1, 0.0)
    ey_index: int = 4                # state component constrained by |x_i| <= w_T
    kappa: np.ndarray = None         # float32 curvature table
    track_len: float = 1.0
    seed: int = 0
    crn_disturbance: int = 0
    resample: int = 0                # 1: re-draw particles from N(mean, cov) before every step (Alg. 2 literal)
    constraints: tuple = ()          # general constraint set (halfspace()/disk() entries); () = racing barrier
    compensated: int = 1
    backoff: int = 0                 # racing barrier's nu: 0 Gaussian, 1 Cantelli (Remark 1)
    clamp_margin: int = 0            # 1: h = max(w_T - nu sigma, 0)^2 - mean_ey^2

    @property
    def nx(self) -> int:
        return {MODEL_BICYCLE6: 6, MODEL_DOUBLE_INT4: 4, MODEL_WHEELS8: 8}[self.model]


def _diag(std):
    std = np.asarray(std, dtype=np.float64)
    return np.diag(std * std)


def racing_problem(K, M, T, track_seed, noise_scale=1.0, lam=1.0, seed=0, **kw) -> Problem:
    """The dynamic-bicycle racing problem on a seeded track."""
    kappa, length = make_track(track_seed)
    p = Problem(K=K, M=M, T=T, lam=lam, ctrl_w=lam, kappa=kappa, track_len=length, seed=seed)
    p.Sigma_eps = _diag([0.05, 0.5])
    p.Sigma_w = _diag(np.array([0.02, 0.02, 0.01, 0.002, 0.02, 0.0]) * noise_scale)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def wheels_problem(K, M, T, track_seed=2, noise_scale=1.0, lam=1.0, seed=0, **kw) -> Problem:
    """The single-track model with wheel speeds and combined slip at AutoRally scale (a 22 kg,
    1 m vehicle) on a seeded track of radius 25 m, goal speed 6 m/s, half-width 2 m. The paper does
    not publish the model's parameters; these are chosen to be plausible for such a vehicle."""
    kappa, length = make_track(track_seed, radius=25.0, amp_max=0.5)
    p = Problem(K=K, M=M, T=T, model=MODEL_WHEELS8, n_sub=10, lam=lam, ctrl_w=lam, kappa=kappa, track_len=length,
                seed=seed, mass=22.0, Iz=1.1, lf=0.34, lr=0.23, tire_B=8.0, tire_C=1.6, mu=0.9, mu_x=1.0,
                wheel_radius=0.095, wheel_inertia=0.05, tau_max=8.0, slip_floor=2.0,
                u_min=(-0.35, -1.0), u_max=(0.35, 1.0), w_T=2.0, ey_index=6,
                x_goal=(6.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0), Q=(1.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.1, 0.0),
                Qf=(1.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.1, 0.0))
    p.Sigma_eps = _diag([0.05, 0.3])
    p.Sigma_w = _diag(np.array([0.02, 0.02, 0.01, 0.05, 0.05, 0.002, 0.02, 0.0]) * noise_scale)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def double_integrator_problem(K, M, T, q_w=0.01, seed=0, **kw) -> Problem:
    """Planar double integrator x = [p_x, p_y, v_x, v_y], u = [a_x, a_y], additive N(0, q_w I).

    Its particle moments have the closed form mean_{k+1} = A mean_k + B u_k,
    Cov_{k+1} = A Cov_k A^T + q_w I, which pins the Monte-Carlo moment machinery.
    """
    p = Problem(K=K, M=M, T=T, model=MODEL_DOUBLE_INT4, n_sub=1, lam=1.0, ctrl_w=1.0, seed=seed,
                u_min=(-1e3, -1e3), u_max=(1e3, 1e3), x_goal=(0.0,) * 6,
                Q=(0.1, 0.1, 0.01, 0.01, 0.0, 0.0), Qf=(0.1, 0.1, 0.01, 0.01, 0.0, 0.0),
                ey_index=1, w_T=5.0, kappa=np.zeros(16, np.float32), track_len=1.0)
    p.Sigma_eps = _diag([0.3, 0.3])
    p.Sigma_w = q_w * np.eye(4)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def halfspace(a, b, p, backoff="gaussian") -> dict:
    """Constraint a^T x - b < 0 held with probability 1 - p."""
    return {"kind": "halfspace", "a": tuple(float(x) for x in a), "b": float(b), "p": float(p), "backoff": backoff}


def disk(i, j, center, radius, p, backoff="gaussian") -> dict:
    """Disk obstacle in the plane of states (i, j): feasible outside, with probability 1 - p."""
    return {"kind": "disk", "i": int(i), "j": int(j), "center": (float(center[0]), float(center[1])),
            "radius": float(radius), "p": float(p), "backoff": backoff}


def racing_x0(p: Problem) -> np.ndarray:
    """Start on the centre line at the goal speed (wheels rolling freely for the wheel-speed model)."""
    x = np.zeros(p.nx, dtype=np.float32)
    if p.model in (MODEL_BICYCLE6, MODEL_WHEELS8):
        x[0] = p.x_goal[0]
    if p.model == MODEL_WHEELS8:
        x[3] = x[4] = p.x_goal[0] / p.wheel_radius
    return x


def random_state(p: Problem, seed: int) -> np.ndarray:
    """A seeded plausible state near the centre line (for parity cases away from the start)."""
    rng = np.random.default_rng(seed)
    if p.model == MODEL_WHEELS8:
        vx = rng.uniform(4.0, 7.0)
        x = np.array([vx, rng.normal(0, 0.1), rng.normal(0, 0.1), vx / p.wheel_radius * (1 + rng.normal(0, 0.02)),
                      vx / p.wheel_radius * (1 + rng.normal(0, 0.02)), rng.normal(0, 0.05), rng.uniform(-1.0, 1.0),
                      rng.uniform(0, p.track_len)])
        return x.astype(np.float32)
    if p.model == MODEL_BICYCLE6:
        x = np.array([rng.uniform(7.0, 12.0), rng.normal(0, 0.3), rng.normal(0, 0.2),
                      rng.normal(0, 0.05), rng.uniform(-2.0, 2.0), rng.uniform(0, p.track_len)])
    else:
        x = rng.normal(0.0, 1.0, size=4)
    return x.astype(np.float32)


def random_nominal(p: Problem, seed: int, scale=(0.1, 1.0)) -> np.ndarray:
    """A seeded smooth nominal control sequence inside the bounds."""
    rng = np.random.default_rng(seed)
    t = np.arange(p.T, dtype=np.float64)
    out = np.zeros((p.T, NU))
    for j in range(NU):
        a, f, ph = rng.uniform(0.2, 1.0), rng.uniform(0.05, 0.3), rng.uniform(0, 2 * math.pi)
        out[:, j] = scale[j] * a * np.sin(f * t + ph)
    lo, hi = np.asarray(p.u_min), np.asarray(p.u_max)
    return np.clip(out, lo, hi).astype(np.float32)


# The five workload configurations (sizes and constants).
def config0() -> Problem:
    """Plain BSS-MPPI, one controller: K=256, M=16, T=20, track seed 0, solve seed 0."""
    return racing_problem(256, 16, 20, track_seed=0, noise_scale=1.0, lam=1.0, seed=0)


def config1() -> Problem:
    """Single-controller racing scale: K=4096, M=64, T=40, disturbance std x2, track seed 1."""
    return racing_problem(4096, 64, 40, track_seed=1, noise_scale=2.0, lam=1.0, seed=1)


def config3(lam: float = 1.0) -> Problem:
    """Precision study scale: K=16384, M=128, T=60, lambda in {0.1, 1, 10}, track seed 1."""
    return racing_problem(16384, 128, 60, track_seed=1, noise_scale=2.0, lam=lam, seed=3)


SERVE_K = (512, 2048, 4096, 8192)
SERVE_M = (8, 32, 64, 128)
SERVE_T = (20, 40, 60)


def serving_requests(n_ctrl=512, rate_hz=20.0, duration_s=1.0, seed=4):
    """Poisson arrivals of solve requests from n_ctrl controllers, each with a (K, M, T) class.

    Returns a list of (t_arrival_s, controller_id, K, M, T) sorted by arrival time.
    """
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_ctrl):
        t = rng.exponential(1.0 / rate_hz)
        while t < duration_s:
            out.append((t, c, int(rng.choice(SERVE_K)), int(rng.choice(SERVE_M)),
                        int(rng.choice(SERVE_T))))
            t += rng.exponential(1.0 / rate_hz)
    out.sort(key=lambda r: r[0])
    return out
