"""Coefficients of the slip-angle arctangent in csrc/device.cuh (`slip_atan`).

atan t = t + t z p(z), z = t^2, with p of degree 4, for |t| <= 1/2. The coefficients minimise the
maximum relative error of atan t over (0, 1/2] by Lawson's algorithm (iteratively reweighted least
squares, whose weights converge to the minimax solution). Reference values come from mpmath at 30
digits. The script prints the coefficients, the relative error in exact arithmetic and the error in
FP32 ulps of the kernel's evaluation (Horner's rule with fused multiply-adds, emulated in float64
and rounded to float32 after every operation).

Run: python paper_2408_00494_gb300/fit_slip_atan.py   (needs numpy and mpmath; not part of the build)
"""
import numpy as np


def fit(n_coef=5, r_max=0.5, iters=300):
    import mpmath as mp
    mp.mp.dps = 30
    u = np.unique(np.concatenate([r_max * np.cos(np.linspace(0, np.pi / 2, 8001))[::-1],
                                  np.linspace(1e-4, r_max, 8001)]))
    u = u[u > 1e-4]
    at = np.array([float(mp.atan(mp.mpf(float(x)))) for x in u])
    z = u * u
    y = (at / u - 1.0) / z                      # p(z) should equal this
    A = np.vander(z, n_coef, increasing=True)
    s = u * z / at                              # turns an error in p into a relative error of atan
    w = np.ones_like(u)
    for _ in range(iters):
        sw = np.sqrt(w) * s
        c, *_ = np.linalg.lstsq(A * sw[:, None], y * sw, rcond=None)
        e = s * (A @ c - y)
        w = w * np.abs(e)
        w /= w.sum()
    return c, float(np.max(np.abs(e)))


def fp32_ulp_error(c, r_max=0.5, n=2_000_000):
    c32 = np.asarray(c, dtype=np.float32)
    t = np.linspace(0, r_max, n + 1, dtype=np.float32)[1:]
    z = (t * t).astype(np.float32)
    p = np.full_like(z, c32[-1])
    for k in range(len(c32) - 2, -1, -1):
        p = (p.astype(np.float64) * z + c32[k]).astype(np.float32)      # one rounding: a fused multiply-add
    tz = (t * z).astype(np.float32)
    r = (tz.astype(np.float64) * p + t).astype(np.float32)
    ref = np.arctan(t.astype(np.float64))
    return float(np.max(np.abs(r - ref) / np.spacing(ref.astype(np.float32)).astype(np.float64)))


if __name__ == "__main__":
    c, rel = fit()
    print("coefficients c_0..c_4:", ", ".join(f"{x:.10e}" for x in c))
    print(f"max relative error (exact arithmetic): {rel:.2e}")
    print(f"max error of the FP32 evaluation: {fp32_ulp_error(c):.2f} ulp")
