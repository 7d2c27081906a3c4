"""Thin Python binding of the C ABI in include/bssmppi.h (argument marshalling only).

Every function has the C entry point's name without the ``bssmppi_`` prefix and takes torch CUDA
tensors where the C function takes device pointers (the tensor's storage is passed as is) and
numpy arrays where it takes host pointers. All compute happens in libbssmppi.so; if the library is
missing or cannot be loaded, every call raises. There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

NU = 2
NDIAG = 4
BUF_S, BUF_W, BUF_EPS, BUF_MEAN, BUF_VAR, BUF_DIAG, BUF_V = range(7)
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "EBUSY", -6: "ENOTSUP"}


class BssmppiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    """Mirror of struct bssmppi_params (layout checked against bssmppi_params_size())."""

    _fields_ = [
        ("K", ctypes.c_int32), ("M", ctypes.c_int32), ("T", ctypes.c_int32), ("n_sub", ctypes.c_int32),
        ("model", ctypes.c_int32), ("ey_index", ctypes.c_int32),
        ("dt", ctypes.c_float), ("mass", ctypes.c_float), ("Iz", ctypes.c_float), ("lf", ctypes.c_float),
        ("lr", ctypes.c_float), ("tire_B", ctypes.c_float), ("tire_C", ctypes.c_float), ("mu", ctypes.c_float),
        ("g", ctypes.c_float), ("vx_floor", ctypes.c_float),
        ("wheel_radius", ctypes.c_float), ("wheel_inertia", ctypes.c_float), ("mu_x", ctypes.c_float),
        ("tau_max", ctypes.c_float), ("slip_floor", ctypes.c_float),
        ("u_min", ctypes.c_float * 2), ("u_max", ctypes.c_float * 2),
        ("lam", ctypes.c_float), ("delta", ctypes.c_float), ("gamma", ctypes.c_float), ("ctrl_w", ctypes.c_float),
        ("C_safe", ctypes.c_float), ("C_obs", ctypes.c_float), ("w_T", ctypes.c_float),
        ("x_goal", ctypes.c_float * 8), ("Q", ctypes.c_float * 8), ("Qf", ctypes.c_float * 8),
        ("track_len", ctypes.c_float), ("n_track", ctypes.c_int32),
        ("track_kappa", ctypes.POINTER(ctypes.c_float)),
        ("Sigma_eps", ctypes.c_double * 4), ("Sigma_w", ctypes.c_double * 64),
        ("seed", ctypes.c_uint64),
        ("crn_disturbance", ctypes.c_int32), ("compensated", ctypes.c_int32),
        ("record_moments", ctypes.c_int32), ("resample", ctypes.c_int32),
        ("backoff", ctypes.c_int32), ("clamp_margin", ctypes.c_int32),
    ]


class Constraint(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("backoff", ctypes.c_int32), ("i", ctypes.c_int32), ("j", ctypes.c_int32),
                ("p", ctypes.c_float), ("b", ctypes.c_float), ("a", ctypes.c_float * 8),
                ("center", ctypes.c_float * 2), ("radius", ctypes.c_float), ("reserved", ctypes.c_int32)]


CON_HALFSPACE, CON_DISK = 0, 1
BACKOFF_GAUSSIAN, BACKOFF_CANTELLI = 0, 1


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_controllers", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("T_max", ctypes.c_int32),
                ("slots", ctypes.c_int32), ("use_graphs", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_size_t), ("max_batch_work", ctypes.c_int64)]


class Result(ctypes.Structure):
    _fields_ = [("req_id", ctypes.c_uint64), ("ctrl_id", ctypes.c_int32), ("status", ctypes.c_int32),
                ("u0", ctypes.c_float * 2), ("beta", ctypes.c_float), ("K", ctypes.c_int32), ("M", ctypes.c_int32),
                ("T", ctypes.c_int32), ("t_submit_us", ctypes.c_double), ("t_start_us", ctypes.c_double),
                ("t_done_us", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "superseded", "admitted", "completed", "batches",
                                               "max_batch_seen", "queued")] + [("now_us", ctypes.c_double)]


_lib = None


def load(build_if_missing: bool = True):
    """Load libbssmppi.so from the package's _lib/ directory (building it first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB_PATH
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, i32, i64, u32, u64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                  ctypes.c_uint64, ctypes.c_size_t)
    sig = {
        "bssmppi_abi_version": (u32, []),
        "bssmppi_params_size": (sz, []),
        "bssmppi_create": (ctypes.c_int, [ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]),
        "bssmppi_solve": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "bssmppi_solve_host": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "bssmppi_shift": (ctypes.c_int, [vp, vp, i32]),
        "bssmppi_set_constraints": (ctypes.c_int, [vp, vp, i32]),
        "bssmppi_solve_shift": (ctypes.c_int, [vp, vp, vp, vp, i32]),
        "bssmppi_set_sample_range": (ctypes.c_int, [vp, i32, i32]),
        "bssmppi_solve_partial": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "bssmppi_merge_partials": (ctypes.c_int, [vp, vp, i32, vp, vp]),
        "bssmppi_destroy": (ctypes.c_int, [vp]),
        "bssmppi_last_error": (ctypes.c_char_p, [vp]),
        "bssmppi_set_counter": (ctypes.c_int, [vp, u32]),
        "bssmppi_get_counter": (ctypes.c_int, [vp, ctypes.POINTER(u32)]),
        "bssmppi_set_nominal": (ctypes.c_int, [vp, vp]),
        "bssmppi_read": (ctypes.c_int, [vp, i32, vp, sz]),
        "bssmppi_timing": (ctypes.c_int, [vp, i32]),
        "bssmppi_timing_read": (ctypes.c_int, [vp, vp, vp, i32, ctypes.POINTER(i32)]),
        "bssmppi_update_noalloc": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, i32, i32, ctypes.c_float, i32, vp]),
        "bssmppi_server_create": (ctypes.c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]),
        "bssmppi_server_add_controller": (ctypes.c_int, [vp, ctypes.POINTER(Params), ctypes.POINTER(i32)]),
        "bssmppi_server_submit": (ctypes.c_int, [vp, i32, vp, i32, i32, i32, u64]),
        "bssmppi_server_poll": (ctypes.c_int, [vp, ctypes.POINTER(Result), i32, ctypes.POINTER(i32)]),
        "bssmppi_server_drain": (ctypes.c_int, [vp, i32]),
        "bssmppi_server_get_state": (ctypes.c_int, [vp, i32, vp, ctypes.POINTER(u32)]),
        "bssmppi_server_set_state": (ctypes.c_int, [vp, i32, vp, u32]),
        "bssmppi_server_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(ServerStats)]),
        "bssmppi_fp32_peak": (ctypes.c_int, [i32, i32, vp, ctypes.POINTER(ctypes.c_float),
                                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]),
        "bssmppi_server_capture": (ctypes.c_int, [vp, i32, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
        "bssmppi_server_last_error": (ctypes.c_char_p, [vp]),
        "bssmppi_server_destroy": (ctypes.c_int, [vp]),
        "bssmppi_repair_grad": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "bssmppi_repair": (ctypes.c_int, [vp, vp, vp, i32, ctypes.c_float, vp]),
        "bssmppi_model_step": (ctypes.c_int, [vp, vp, vp, vp, vp, i64]),
        "bssmppi_philox4x32_10": (ctypes.c_int, [vp, u64, vp, i64, vp]),
        "bssmppi_box_muller": (ctypes.c_int, [vp, vp, i64, vp]),
        "bssmppi_slip_atan": (ctypes.c_int, [vp, vp, i64, vp]),
        "bssmppi_tyre_curve": (ctypes.c_int, [vp, vp, vp, i64, vp]),
        "bssmppi_tyre_curve_coefficients": (ctypes.c_int, [ctypes.c_double, vp, i32]),
        "bssmppi_rear_tyre": (ctypes.c_int, [vp, vp, vp, i64, vp]),
        "bssmppi_rear_tyre_coefficients": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, vp, i32, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    if L.bssmppi_params_size() != ctypes.sizeof(Params):
        raise RuntimeError("bssmppi_params layout mismatch between the binding and the library")
    _lib = L
    return L


def _ptr(t):
    """Device pointer of a contiguous torch CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    if a is None:
        return None
    if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous):
        raise ValueError("expected a contiguous float32 numpy array")
    return ctypes.c_void_p(a.__array_interface__["data"][0])


def _check(rc, h=None):
    if rc != 0:
        msg = load().bssmppi_last_error(h)
        raise BssmppiError(rc, msg.decode() if msg else "")


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def make_params(prob, record_moments: bool = False, compensated: bool | None = None) -> Params:
    """Fill the C struct from a problem description (workload.Problem or any object with its fields)."""
    p = Params()
    for name in ("K", "M", "T", "n_sub", "model", "ey_index"):
        setattr(p, name, int(getattr(prob, name)))
    for name in ("dt", "mass", "Iz", "lf", "lr", "tire_B", "tire_C", "mu", "g", "vx_floor", "delta", "gamma",
                 "ctrl_w", "C_safe", "C_obs", "w_T"):
        setattr(p, name, float(getattr(prob, name)))
    for name, default in (("wheel_radius", 0.3), ("wheel_inertia", 1.0), ("mu_x", 1.0), ("tau_max", 0.0),
                          ("slip_floor", 2.0)):
        setattr(p, name, float(getattr(prob, name, default)))
    p.lam = float(prob.lam)
    for i in range(2):
        p.u_min[i] = float(prob.u_min[i])
        p.u_max[i] = float(prob.u_max[i])
    for i in range(min(8, len(prob.x_goal))):
        p.x_goal[i] = float(prob.x_goal[i])
        p.Q[i] = float(prob.Q[i])
        p.Qf[i] = float(prob.Qf[i])
    kappa = np.ascontiguousarray(np.asarray(prob.kappa, dtype=np.float32))
    p._kappa_keepalive = kappa
    p.track_kappa = kappa.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    p.n_track = int(kappa.size)
    p.track_len = float(prob.track_len)
    se = np.asarray(prob.Sigma_eps, dtype=np.float64).reshape(-1)
    for i in range(4):
        p.Sigma_eps[i] = float(se[i])
    sw = np.asarray(prob.Sigma_w, dtype=np.float64).reshape(-1)
    for i in range(sw.size):
        p.Sigma_w[i] = float(sw[i])
    p.seed = int(prob.seed) & 0xFFFFFFFFFFFFFFFF
    p.crn_disturbance = int(prob.crn_disturbance)
    p.compensated = int(prob.compensated if compensated is None else compensated)
    p.record_moments = int(record_moments)
    p.resample = int(getattr(prob, "resample", 0))
    p.backoff = int(getattr(prob, "backoff", 0))
    p.clamp_margin = int(getattr(prob, "clamp_margin", 0))
    return p


# ---- the C entry points, one Python function each ---------------------------------------------

def abi_version() -> int:
    return load().bssmppi_abi_version()


def params_size() -> int:
    return load().bssmppi_params_size()


def create(params: Params, stream=None):
    h = ctypes.c_void_p()
    _check(load().bssmppi_create(ctypes.byref(params), _stream_handle(stream), ctypes.byref(h)))
    return h


def solve(h, x0, Sigma0=None, v=None, u0=None):
    _check(load().bssmppi_solve(h, _ptr(x0), _ptr(Sigma0), _ptr(v), _ptr(u0)), h)


def solve_shift(h, x0, Sigma0=None, u0=None, n: int = 1):
    """Solve on the resident nominal and shift it by n steps, in one launch (u0 = v+_0)."""
    _check(load().bssmppi_solve_shift(h, _ptr(x0), _ptr(Sigma0), _ptr(u0), int(n)), h)


def solve_host(h, x0, Sigma0=None, v=None, u0=None):
    _check(load().bssmppi_solve_host(h, _hptr(x0), _hptr(Sigma0), _hptr(v), _hptr(u0)), h)


def make_constraints(cons):
    """ctypes array of bssmppi_constraint from {"kind": "halfspace" | "disk", ...} descriptions."""
    arr = (Constraint * max(1, len(cons)))()
    for q, c in enumerate(cons):
        k = arr[q]
        k.kind = {"halfspace": CON_HALFSPACE, "disk": CON_DISK}[c["kind"]]
        k.backoff = {"gaussian": BACKOFF_GAUSSIAN, "cantelli": BACKOFF_CANTELLI}[c.get("backoff", "gaussian")]
        k.p = float(c["p"])
        if k.kind == CON_HALFSPACE:
            for l, x in enumerate(c["a"]):
                k.a[l] = float(x)
            k.b = float(c["b"])
        else:
            k.i, k.j = int(c["i"]), int(c["j"])
            k.center[0], k.center[1] = float(c["center"][0]), float(c["center"][1])
            k.radius = float(c["radius"])
    return arr


def set_constraints(h, cons):
    """Selects the general constraint set (an empty list restores the racing barrier)."""
    cons = list(cons or ())
    _check(load().bssmppi_set_constraints(h, ctypes.cast(make_constraints(cons), ctypes.c_void_p), len(cons)), h)


def set_sample_range(h, k_begin: int, K_total: int):
    _check(load().bssmppi_set_sample_range(h, int(k_begin), int(K_total)), h)


def solve_partial(h, x0, Sigma0, v, partial):
    _check(load().bssmppi_solve_partial(h, _ptr(x0), _ptr(Sigma0), _ptr(v), _ptr(partial)), h)


def merge_partials(h, partials, v=None, u0=None):
    G = partials.shape[0] if partials.dim() > 1 else 1
    _check(load().bssmppi_merge_partials(h, _ptr(partials), int(G), _ptr(v), _ptr(u0)), h)


def sharded_solve(h, x0, T, Sigma0=None, v=None, u0=None, group=None):
    """One solve whose samples are split over the ranks of a torch.distributed group (each rank's
    handle covers its range, set with set_sample_range): partial, one all-gather of the partials,
    merge. Every rank ends with the whole solve's update in its resident nominal (and v, u0).
    With NCCL the partials are gathered on the device; with gloo (CPU collectives) they are staged
    through host memory: 4 (3 + 2T) bytes per rank each way."""
    import torch
    import torch.distributed as dist
    part = torch.empty(3 + 2 * T, dtype=torch.float32, device=x0.device)
    solve_partial(h, x0, Sigma0, v, part)
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    if world == 1:
        parts = part.view(1, -1)
    elif dist.get_backend(group) == "nccl":
        parts = torch.empty(world, 3 + 2 * T, dtype=torch.float32, device=x0.device)
        dist.all_gather_into_tensor(parts, part, group=group)
    else:
        host = part.cpu()
        gathered = [torch.empty_like(host) for _ in range(world)]
        dist.all_gather(gathered, host, group=group)
        parts = torch.stack(gathered).to(x0.device)
    merge_partials(h, parts, v, u0)


def shift(h, v=None, n: int = 1):
    _check(load().bssmppi_shift(h, _ptr(v), int(n)), h)


def destroy(h):
    _check(load().bssmppi_destroy(h))


def last_error(h=None) -> str:
    msg = load().bssmppi_last_error(h)
    return msg.decode() if msg else ""


def set_counter(h, counter: int):
    _check(load().bssmppi_set_counter(h, ctypes.c_uint32(counter)), h)


def get_counter(h) -> int:
    c = ctypes.c_uint32()
    _check(load().bssmppi_get_counter(h, ctypes.byref(c)), h)
    return c.value


def set_nominal(h, v):
    _check(load().bssmppi_set_nominal(h, _ptr(v)), h)


def read(h, which: int, dst):
    _check(load().bssmppi_read(h, int(which), _ptr(dst), dst.numel() * dst.element_size()), h)


def timing(h, n: int):
    _check(load().bssmppi_timing(h, int(n)), h)


def timing_read(h, max_n: int = 4096):
    """Durations (ms) of the solves recorded since timing(h, n): (solve kernel, update) arrays; the update
    is fused into the solve kernel, so its entries are 0."""
    roll = np.zeros(max_n, np.float32)
    upd = np.zeros(max_n, np.float32)
    n = ctypes.c_int32()
    _check(load().bssmppi_timing_read(h, ctypes.c_void_p(roll.ctypes.data), ctypes.c_void_p(upd.ctypes.data),
                                      int(max_n), ctypes.byref(n)), h)
    return roll[: n.value].copy(), upd[: n.value].copy()


def update_noalloc(S, eps, v, w, u0=None, diag=None, counter=None, lam=1.0, compensated=True, stream=None):
    """Weights and update with no device allocation (scratch in the library's static array).
    K and T are taken from the shapes of S [K] and eps [K, T, 2]."""
    K, T = int(S.numel()), int(eps.numel() // (2 * max(1, S.numel())))
    _check(load().bssmppi_update_noalloc(_ptr(S), _ptr(eps), _ptr(v), _ptr(w), _ptr(u0), _ptr(diag), _ptr(counter),
                                         K, T, ctypes.c_float(lam), int(bool(compensated)), _stream_handle(stream)))


def repair_grad(h, x0, v, grad, J=None):
    _check(load().bssmppi_repair_grad(h, _ptr(x0), _ptr(v), _ptr(grad), _ptr(J)), h)


def repair(h, x0, v=None, iters=5, step=2e-6, J=None):
    _check(load().bssmppi_repair(h, _ptr(x0), _ptr(v), int(iters), ctypes.c_float(step), _ptr(J)), h)


def _repair_objective_function():
    import torch

    class RepairObjective(torch.autograd.Function):
        """J_r(v) of bssmppi_repair_grad as a differentiable torch function of the nominal v [T, 2].

        forward runs the library's forward rollout and adjoint sweep once and keeps dJ/dv; backward
        scales it by the incoming gradient. x0 and the handle are not differentiated."""

        @staticmethod
        def forward(ctx, v, x0, handle):
            v = v.contiguous()
            J = torch.empty(1, dtype=torch.float32, device=v.device)
            grad = torch.empty_like(v)
            repair_grad(handle, x0.contiguous(), v, grad, J)
            ctx.save_for_backward(grad)
            return J[0]

        @staticmethod
        def backward(ctx, gJ):
            (grad,) = ctx.saved_tensors
            return gJ * grad, None, None

    return RepairObjective


_RepairObjective = None


def repair_objective(v, x0, handle):
    """Differentiable repair objective J_r(v) (a torch.autograd.Function backed by the adjoint kernel)."""
    global _RepairObjective
    if _RepairObjective is None:
        _RepairObjective = _repair_objective_function()
    return _RepairObjective.apply(v, x0, handle)


def fp32_peak(packed=False, iters=1 << 14, stream=None) -> dict:
    """Measured FP32 multiply-add rate of the current device (bssmppi_fp32_peak)."""
    ms, tf, sms = ctypes.c_float(0.0), ctypes.c_double(0.0), ctypes.c_int32(0)
    _check(load().bssmppi_fp32_peak(int(bool(packed)), int(iters), _stream_handle(stream), ctypes.byref(ms),
                                    ctypes.byref(tf), ctypes.byref(sms)))
    return {"tflops": tf.value, "ms": ms.value, "sms": sms.value, "packed": bool(packed)}


def model_step(h, x, u, x_next, w=None):
    """x_next = f(x, u) + w for n states (rows of x); w may be None."""
    n = x.shape[0] if x.dim() > 1 else 1
    _check(load().bssmppi_model_step(h, _ptr(x), _ptr(u), _ptr(w), _ptr(x_next), n), h)


def philox4x32_10(ctr, seed: int, out, stream=None):
    _check(load().bssmppi_philox4x32_10(_ptr(ctr), ctypes.c_uint64(seed), _ptr(out), ctr.numel() // 4,
                                        _stream_handle(stream)))


def box_muller(words, z, stream=None):
    _check(load().bssmppi_box_muller(_ptr(words), _ptr(z), words.numel() // 2, _stream_handle(stream)))


def tyre_curve(h, x, y, stream=None):
    """y = sin(C atan x) as the substep evaluates it, for the handle's tyre shape factor C."""
    _check(load().bssmppi_tyre_curve(h, _ptr(x), _ptr(y), x.numel(), _stream_handle(stream)), h)


def rear_tyre(h, t, y, stream=None):
    """y = sin(C atan(-B atan t)), the rear tyre's curve at slip argument t as the substep evaluates it."""
    _check(load().bssmppi_rear_tyre(h, _ptr(t), _ptr(y), t.numel(), _stream_handle(stream)), h)


def rear_tyre_coefficients(B, C):
    """(c_0..c_9, tau) of the rear tyre's polynomial in x = t / tau for B and C (host only)."""
    c = np.zeros(10, np.float32)
    tau = ctypes.c_double(0.0)
    _check(load().bssmppi_rear_tyre_coefficients(float(B), float(C), ctypes.c_void_p(c.ctypes.data), 10,
                                                 ctypes.byref(tau)))
    return c, tau.value


def tyre_curve_coefficients(C) -> np.ndarray:
    """c_0..c_9 of the tyre curve's polynomial for shape factor C (host only)."""
    c = np.zeros(10, np.float32)
    _check(load().bssmppi_tyre_curve_coefficients(float(C), ctypes.c_void_p(c.ctypes.data), 10))
    return c


def slip_atan(t, y, stream=None):
    """y = atan(t) as the substeps take the slip angles (float32 device tensors of equal size)."""
    _check(load().bssmppi_slip_atan(_ptr(t), _ptr(y), t.numel(), _stream_handle(stream)))


class Controller:
    """Owns one handle: the problem, its device buffers and its stream (convenience wrapper)."""

    def __init__(self, prob, record_moments=False, compensated=None, stream=None):
        import torch
        self.prob = prob
        self.params = make_params(prob, record_moments=record_moments, compensated=compensated)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = create(self.params, self.stream)
        self.nx = prob.nx
        if getattr(prob, "constraints", ()):
            set_constraints(self.h, prob.constraints)

    def close(self):
        if self.h is not None:
            destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def buffer(self, which):
        import torch
        K, T, nx = self.prob.K, self.prob.T, self.nx
        shape = {BUF_S: (K,), BUF_W: (K,), BUF_EPS: (K, T, 2), BUF_MEAN: (K, T + 1, nx),
                 BUF_VAR: (K, T + 1, nx), BUF_DIAG: (NDIAG,), BUF_V: (T, 2)}[which]
        out = torch.empty(shape, dtype=torch.float32, device="cuda")
        read(self.h, which, out)
        return out


# ---- serving ----------------------------------------------------------------------------------

def _srv_check(rc, s):
    if rc != 0:
        msg = load().bssmppi_server_last_error(s)
        raise BssmppiError(rc, msg.decode() if msg else "")


def server_create(max_controllers, max_batch=256, T_max=60, slots=2, use_graphs=True, hbm_budget_bytes=1 << 30,
                  max_batch_work=0):
    cfg = ServerConfig(int(max_controllers), int(max_batch), int(T_max), int(slots), int(bool(use_graphs)), 0,
                       int(hbm_budget_bytes), int(max_batch_work))
    s = ctypes.c_void_p()
    _srv_check(load().bssmppi_server_create(ctypes.byref(cfg), ctypes.byref(s)), None)
    return s


def server_add_controller(s, params: Params) -> int:
    cid = ctypes.c_int32()
    _srv_check(load().bssmppi_server_add_controller(s, ctypes.byref(params), ctypes.byref(cid)), s)
    return cid.value


def server_submit(s, ctrl_id, x0, K, M, T, req_id):
    x = np.ascontiguousarray(np.asarray(x0, dtype=np.float32).reshape(-1)[:6])
    _srv_check(load().bssmppi_server_submit(s, int(ctrl_id), ctypes.c_void_p(x.ctypes.data), int(K), int(M), int(T),
                                            ctypes.c_uint64(req_id)), s)


def server_poll(s, max_n=4096):
    buf = (Result * max_n)()
    n = ctypes.c_int32()
    _srv_check(load().bssmppi_server_poll(s, buf, int(max_n), ctypes.byref(n)), s)
    return [buf[i] for i in range(n.value)]


def server_drain(s, timeout_ms=60000):
    _srv_check(load().bssmppi_server_drain(s, int(timeout_ms)), s)


def server_get_state(s, ctrl_id, T_max):
    v = np.zeros((T_max, 2), np.float32)
    c = ctypes.c_uint32()
    _srv_check(load().bssmppi_server_get_state(s, int(ctrl_id), ctypes.c_void_p(v.ctypes.data), ctypes.byref(c)), s)
    return v, c.value


def server_set_state(s, ctrl_id, v, counter):
    v = np.ascontiguousarray(v, dtype=np.float32)
    _srv_check(load().bssmppi_server_set_state(s, int(ctrl_id), ctypes.c_void_p(v.ctypes.data), int(counter)), s)


def server_get_stats(s) -> dict:
    st = ServerStats()
    _srv_check(load().bssmppi_server_get_stats(s, ctypes.byref(st)), s)
    return {name: getattr(st, name) for name, _ in ServerStats._fields_}


class ServerCapture:
    """Host buffers that receive one served request's S, weights and eps_eff (bssmppi_server_capture)."""

    def __init__(self, K_max, T_max):
        self.buf = np.zeros(K_max * (2 + 2 * T_max), np.float32)
        self.written = ctypes.c_int64(0)

    def result(self, K, T):
        """(S[K], w[K], eps[K, T, 2]) once the request completed, else None."""
        n = self.written.value
        if n == 0:
            return None
        if n < 0:
            raise BssmppiError(n, "capture did not fit" if n == -1 else "capture copy failed")
        assert n == K * (2 + 2 * T)
        b = self.buf
        return b[:K].copy(), b[K:2 * K].copy(), b[2 * K:2 * K + 2 * K * T].reshape(K, T, 2).copy()


def server_capture(s, ctrl_id, K_max, T_max) -> ServerCapture:
    cap = ServerCapture(K_max, T_max)
    _srv_check(load().bssmppi_server_capture(s, int(ctrl_id), ctypes.c_void_p(cap.buf.ctypes.data), cap.buf.size,
                                             ctypes.byref(cap.written)), s)
    return cap


def server_destroy(s):
    _srv_check(load().bssmppi_server_destroy(s), None)
