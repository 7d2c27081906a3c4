"""The tyre curve's polynomial, fitted by the library on the host (no GPU needed): for the shape
factors of the workloads and around them, x p(x^2) with the FP32-rounded coefficients stays within
4e-7 of sin(C atan x) on |x| <= 1 (the hardware sine it replaces is within 2^-21.4 = 3.6e-7), p(0) is
C (the slope B C of the lateral force at zero slip, in units of B D), and bad shape factors are
rejected."""
import numpy as np
import pytest

from paper_2408_00494_gb300 import bssmppi


@pytest.mark.parametrize("C", [1.3, 1.6, 1.9, 2.2])
def test_fit_reproduces_the_curve(C):
    c = bssmppi.tyre_curve_coefficients(C).astype(np.float64)
    x = np.linspace(-1.0, 1.0, 40001)
    y = x * np.polyval(c[::-1], x * x)
    err = np.abs(y - np.sin(C * np.arctan(x)))
    assert err.max() <= 4e-7, err.max()
    assert abs(c[0] - C) <= 1e-7 * C
    assert np.abs(c).max() <= 2 * C  # coefficients of the order of C: Horner's rule in FP32 cancels little


def test_fit_rejects_bad_shape_factors():
    for C in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(bssmppi.BssmppiError):
            bssmppi.tyre_curve_coefficients(C)
