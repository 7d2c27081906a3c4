"""The slip-angle arctangent's coefficients in csrc/device.cuh are the ones the committed fit
produces (paper_2408_00494_gb300/fit_slip_atan.py: Lawson's iteratively reweighted least squares
for the least maximum relative error of atan on (0, 1/2]), and their FP32 evaluation stays within
one ulp of atan. The GPU's own evaluation is checked in tests/test_gpu_parity.py."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _kernel_coefficients():
    src = open(os.path.join(ROOT, "paper_2408_00494_gb300", "csrc", "device.cuh")).read()
    body = src[src.index("float slip_atan_coef(int i)"):]
    body = body[: body.index("}")]
    lits = [float(x) for x in re.findall(r"(-?\d\.\d+e-?\d+)f", body)]
    # Horner order in the source (the coefficient function slip_atan reads): c_4 first, then c_3 .. c_0
    assert len(lits) == 5
    return np.array(lits[::-1])


def test_kernel_coefficients_are_the_fit():
    pytest.importorskip("mpmath")
    from paper_2408_00494_gb300 import fit_slip_atan
    c, rel = fit_slip_atan.fit()
    assert rel < 1e-8
    k = _kernel_coefficients()
    assert np.allclose(k, c, rtol=1e-9, atol=0.0), (k, c)


def test_fp32_evaluation_within_one_ulp():
    from paper_2408_00494_gb300 import fit_slip_atan
    assert fit_slip_atan.fp32_ulp_error(_kernel_coefficients().astype(np.float32)) <= 1.0
