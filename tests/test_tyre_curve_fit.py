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


@pytest.mark.parametrize("B,C", [(10.0, 1.9), (8.0, 1.6), (14.0, 2.2), (1.5, 1.3)])
def test_rear_fit_reproduces_the_composite_curve(B, C):
    """The rear tyre's curve sin(C atan(-B atan t)) from one polynomial in x = t / tau: within 4e-7 of
    the composite on |t| <= tau, tau = tan(1/B) (where |B atan t| reaches 1) or 1/2 if that is less,
    with the slope -B C tau at x = 0."""
    c, tau = bssmppi.rear_tyre_coefficients(B, C)
    assert tau == pytest.approx(np.tan(1.0 / B) if 1.0 / B < np.arctan(0.5) else 0.5, rel=1e-15)
    c = c.astype(np.float64)
    t = np.linspace(-tau, tau, 40001)
    x = t / tau
    err = np.abs(x * np.polyval(c[::-1], x * x) - np.sin(C * np.arctan(-B * np.arctan(t))))
    assert err.max() <= 4e-7, err.max()
    assert abs(c[0] + B * C * tau) <= 1e-6 * B * C * tau
    assert np.abs(c).max() <= 2 * C


def test_rear_fit_rejects_bad_parameters():
    for B, C in ((0.0, 1.9), (10.0, 0.0), (-1.0, 1.9), (float("nan"), 1.9), (10.0, float("inf"))):
        with pytest.raises(bssmppi.BssmppiError):
            bssmppi.rear_tyre_coefficients(B, C)
