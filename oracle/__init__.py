"""FP64 reference oracle for the BSS-MPPI solve (ctypes wrapper around bssmppi_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use it to check and to time against; the product path never imports it. It shares no code
with the CUDA library: the two receive the same seeded inputs from ``workload`` and nothing else.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_DIR = os.path.join(_HERE, "_lib")
_LIB_PATH = os.path.join(_LIB_DIR, "liboracle.so")
_SRC = os.path.join(_HERE, "bssmppi_oracle.c")

_dp = ctypes.POINTER(ctypes.c_double)


class OrcConstraint(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("backoff", ctypes.c_int), ("i", ctypes.c_int), ("j", ctypes.c_int),
                ("p", ctypes.c_double), ("b", ctypes.c_double), ("a", ctypes.c_double * 8),
                ("center", ctypes.c_double * 2), ("radius", ctypes.c_double)]


class OrcProblem(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int), ("M", ctypes.c_int), ("T", ctypes.c_int), ("n_sub", ctypes.c_int),
        ("model", ctypes.c_int),
        ("dt", ctypes.c_double), ("mass", ctypes.c_double), ("Iz", ctypes.c_double),
        ("lf", ctypes.c_double), ("lr", ctypes.c_double), ("tire_B", ctypes.c_double),
        ("tire_C", ctypes.c_double), ("mu", ctypes.c_double), ("g", ctypes.c_double),
        ("vx_floor", ctypes.c_double),
        ("wheel_radius", ctypes.c_double), ("wheel_inertia", ctypes.c_double), ("mu_x", ctypes.c_double),
        ("tau_max", ctypes.c_double), ("slip_floor", ctypes.c_double),
        ("u_min", ctypes.c_double * 2), ("u_max", ctypes.c_double * 2),
        ("Sigma_eps", ctypes.c_double * 4), ("Sigma_w", ctypes.c_double * 64),
        ("lam", ctypes.c_double), ("delta", ctypes.c_double), ("gamma", ctypes.c_double),
        ("ctrl_w", ctypes.c_double), ("C_safe", ctypes.c_double), ("C_obs", ctypes.c_double),
        ("w_T", ctypes.c_double),
        ("x_goal", ctypes.c_double * 8), ("Q", ctypes.c_double * 8), ("Qf", ctypes.c_double * 8),
        ("ey_index", ctypes.c_int),
        ("kappa", _dp), ("n_track", ctypes.c_int), ("track_len", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("crn_disturbance", ctypes.c_int), ("resample", ctypes.c_int),
        ("n_con", ctypes.c_int), ("con", ctypes.POINTER(OrcConstraint)),
        ("backoff", ctypes.c_int), ("clamp_margin", ctypes.c_int),
    ]


class OrcOutputs(ctypes.Structure):
    _fields_ = [(n, _dp) for n in ("S", "u", "w", "v_plus", "mean", "cov", "margin", "h", "diag")]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE double: no contraction, no fast-math), with OpenMP
    for the optional threads over samples when the compiler has it (one thread otherwise)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                "-o", _LIB_PATH, _SRC, "-lm"]
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.run(base, check=True)
    return _LIB_PATH


def host_threads() -> int:
    """Threads the oracle may use on this host: the CPUs this process may run on."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_philox4x32_10_batch.argtypes = [ctypes.c_int64, u32p, u32p, u32p]
        L.orc_gaussian_pair.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _dp]
        L.orc_backoff_gaussian.restype = ctypes.c_double
        L.orc_backoff_gaussian.argtypes = [ctypes.c_double]
        L.orc_backoff_cantelli.restype = ctypes.c_double
        L.orc_backoff_cantelli.argtypes = [ctypes.c_double]
        L.orc_track_kappa.restype = ctypes.c_double
        L.orc_track_kappa.argtypes = [ctypes.POINTER(OrcProblem), ctypes.c_double]
        L.orc_model_step.argtypes = [ctypes.POINTER(OrcProblem), _dp, _dp, _dp]
        L.orc_rollout.argtypes = [ctypes.POINTER(OrcProblem), _dp, _dp, _dp, ctypes.c_uint32,
                                  ctypes.c_int, ctypes.c_int, ctypes.POINTER(OrcOutputs)]
        L.orc_optimal_control.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp,
                                          _dp, _dp, _dp]
        L.orc_lse_partial.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]
        L.orc_lse_merge.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp, _dp]
        L.orc_solve.argtypes = [ctypes.POINTER(OrcProblem), _dp, _dp, _dp, ctypes.c_uint32,
                                ctypes.POINTER(OrcOutputs)]
        L.orc_rollout_threads.argtypes = [ctypes.POINTER(OrcProblem), _dp, _dp, _dp, ctypes.c_uint32,
                                          ctypes.c_int, ctypes.c_int, ctypes.POINTER(OrcOutputs), ctypes.c_int]
        L.orc_solve_threads.argtypes = [ctypes.POINTER(OrcProblem), _dp, _dp, _dp, ctypes.c_uint32,
                                        ctypes.POINTER(OrcOutputs), ctypes.c_int]
        L.orc_repair_objective.restype = ctypes.c_double
        L.orc_repair_objective.argtypes = [ctypes.POINTER(OrcProblem), _dp, _dp, ctypes.c_uint32, _dp, _dp]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _f32(x):
    """Inputs are handed to the CUDA path as float32; the oracle takes the same rounded values."""
    return float(np.float32(x))


class Oracle:
    """Holds one problem in the oracle's own struct (keeps the arrays it points to alive)."""

    def __init__(self, prob):
        self.prob = prob
        p = OrcProblem()
        for name in ("K", "M", "T", "n_sub", "model", "ey_index", "crn_disturbance", "resample"):
            setattr(p, name, int(getattr(prob, name)))
        p.backoff = int(getattr(prob, "backoff", 0))
        p.clamp_margin = int(getattr(prob, "clamp_margin", 0))
        for name in ("dt", "mass", "Iz", "lf", "lr", "tire_B", "tire_C", "mu", "g", "vx_floor",
                     "wheel_radius", "wheel_inertia", "mu_x", "tau_max", "slip_floor",
                     "delta", "gamma", "ctrl_w", "C_safe", "C_obs", "w_T"):
            setattr(p, name, _f32(getattr(prob, name)))
        p.lam = _f32(prob.lam)
        for i in range(2):
            p.u_min[i] = _f32(prob.u_min[i])
            p.u_max[i] = _f32(prob.u_max[i])
        se = np.asarray(prob.Sigma_eps, dtype=np.float64).reshape(2, 2)
        for i in range(4):
            p.Sigma_eps[i] = se.flat[i]
        nx = prob.nx
        sw = np.asarray(prob.Sigma_w, dtype=np.float64).reshape(nx, nx)
        for i in range(nx * nx):
            p.Sigma_w[i] = sw.flat[i]
        for i in range(min(8, len(prob.x_goal))):
            p.x_goal[i] = _f32(prob.x_goal[i])
            p.Q[i] = _f32(prob.Q[i])
            p.Qf[i] = _f32(prob.Qf[i])
        self._kappa = np.ascontiguousarray(np.asarray(prob.kappa, dtype=np.float32), dtype=np.float64)
        p.kappa = _ptr(self._kappa)
        p.n_track = int(self._kappa.size)
        p.track_len = _f32(prob.track_len)
        p.seed = int(prob.seed) & 0xFFFFFFFFFFFFFFFF
        cons = list(getattr(prob, "constraints", ()) or ())
        self._con = (OrcConstraint * max(1, len(cons)))()
        for q, c in enumerate(cons):
            oc = self._con[q]
            oc.kind = {"halfspace": 0, "disk": 1}[c["kind"]]
            oc.backoff = {"gaussian": 0, "cantelli": 1}[c.get("backoff", "gaussian")]
            oc.p = _f32(c["p"])
            if oc.kind == 0:
                for l in range(8):
                    oc.a[l] = _f32(c["a"][l]) if l < len(c["a"]) else 0.0
                oc.b = _f32(c["b"])
            else:
                oc.i, oc.j = int(c["i"]), int(c["j"])
                oc.center[0], oc.center[1] = _f32(c["center"][0]), _f32(c["center"][1])
                oc.radius = _f32(c["radius"])
        p.n_con = len(cons)
        p.con = ctypes.cast(self._con, ctypes.POINTER(OrcConstraint))
        self.p = p
        self.nx = nx

    def solve(self, x0, v, ctr, Sigma0=None, want_cov=False, k_range=None, threads=1):
        """Full solve (or rollout of samples k_range=(k0, k1) only). Returns a dict of arrays.
        threads > 1 spreads whole samples over OpenMP threads (the same results bit for bit)."""
        K, T, nx = self.prob.K, self.prob.T, self.nx
        x0 = np.ascontiguousarray(np.asarray(x0, dtype=np.float32), dtype=np.float64)
        v = np.ascontiguousarray(np.asarray(v, dtype=np.float32).reshape(T, 2), dtype=np.float64)
        S0 = None
        if Sigma0 is not None:
            S0 = np.ascontiguousarray(np.asarray(Sigma0, dtype=np.float32).reshape(nx, nx), dtype=np.float64)
        r = {
            "S": np.zeros(K), "u": np.zeros((K, T, 2)), "w": np.zeros(K), "v_plus": np.zeros((T, 2)),
            "mean": np.zeros((K, T + 1, nx)), "margin": np.zeros(K), "h": np.zeros((K, T + 1)),
            "diag": np.zeros(4),
        }
        if want_cov:
            r["cov"] = np.zeros((K, T + 1, nx, nx))
        o = OrcOutputs(*[_ptr(r.get(name)) for name, _ in OrcOutputs._fields_])
        if k_range is None:
            rc = lib().orc_solve_threads(ctypes.byref(self.p), _ptr(x0), _ptr(S0), _ptr(v), ctypes.c_uint32(ctr),
                                         ctypes.byref(o), int(threads))
        else:
            rc = lib().orc_rollout_threads(ctypes.byref(self.p), _ptr(x0), _ptr(S0), _ptr(v), ctypes.c_uint32(ctr),
                                           int(k_range[0]), int(k_range[1]), ctypes.byref(o), int(threads))
        if rc != 0:
            raise ValueError("oracle rejected the problem")
        r["eps"] = r["u"] - v[None]
        return r

    def model_step(self, x, u):
        x = np.ascontiguousarray(x, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.zeros(self.nx)
        lib().orc_model_step(ctypes.byref(self.p), _ptr(x), _ptr(u), _ptr(out))
        return out

    def kappa_at(self, s):
        return lib().orc_track_kappa(ctypes.byref(self.p), float(s))

    def repair_objective(self, x0, v, ctr, grad=True, want_args=False):
        """J_r(v) and (optionally) its gradient dJ/dv [T, 2] and the hinge arguments [T + 1]."""
        if self.prob.model == 2:
            raise ValueError("the repair objective has no adjoint for the wheel-speed model")
        T = self.prob.T
        x0 = np.ascontiguousarray(np.asarray(x0, dtype=np.float64))
        v = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(T, 2))
        g = np.zeros((T, 2)) if grad else None
        a = np.zeros(T + 1) if want_args else None
        J = lib().orc_repair_objective(ctypes.byref(self.p), _ptr(x0), _ptr(v), ctypes.c_uint32(ctr), _ptr(g),
                                       _ptr(a))
        out = (J, g) if grad else (J,)
        if want_args:
            out = out + (a,)
        return out if len(out) > 1 else out[0]


def optimal_control(S, u, lam):
    """Weights and update from given costs S[K] and clamped samples u[K, T, 2]."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    K, T = u.shape[0], u.shape[1]
    w = np.zeros(K)
    vp = np.zeros((T, 2))
    diag = np.zeros(4)
    lib().orc_optimal_control(K, T, float(lam), _ptr(S), _ptr(u), _ptr(w), _ptr(vp), _ptr(diag))
    return w, vp, diag


def lse_partial(S, u, lam, k_range):
    """Log-sum-exp partial {beta, eta, q, U[2T]} of the samples k_range = (k0, k1)."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    T = u.shape[1]
    part = np.zeros(3 + 2 * T)
    lib().orc_lse_partial(int(k_range[0]), int(k_range[1]), T, float(lam), _ptr(S), _ptr(u), _ptr(part))
    return part


def lse_merge(parts, lam, K_total):
    """Merge of G partials (rows of parts) into (v+ [T, 2], diag[4])."""
    parts = np.ascontiguousarray(parts, dtype=np.float64)
    G, n = parts.shape
    T = (n - 3) // 2
    vp, diag = np.zeros((T, 2)), np.zeros(4)
    lib().orc_lse_merge(G, T, float(lam), int(K_total), _ptr(parts), _ptr(vp), _ptr(diag))
    return vp, diag


def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    out = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, out)
    return np.array(list(out), dtype=np.uint32)


def philox_batch(ctr, key):
    """Philox of n counters (uint32 array of shape (n, 4))."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
    out = np.zeros_like(ctr)
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib().orc_philox4x32_10_batch(ctr.shape[0], ctr.ctypes.data_as(u32p), k, out.ctypes.data_as(u32p))
    return out


def gaussian_pair(a, b):
    z = np.zeros(2)
    lib().orc_gaussian_pair(ctypes.c_uint32(a), ctypes.c_uint32(b), _ptr(z))
    return z


def backoff_gaussian(p):
    return lib().orc_backoff_gaussian(float(p))


def backoff_cantelli(p):
    return lib().orc_backoff_cantelli(float(p))
