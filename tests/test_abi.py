"""The C-ABI library builds, loads and exports every entry point include/*.h declares (CPU only).

No compute call runs here; without a GPU, create() must fail loudly instead of falling back.
"""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import workload
from paper_2408_00494_gb300 import _build, bssmppi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(bssmppi_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("bssmppi_create", "bssmppi_solve", "bssmppi_shift", "bssmppi_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_build.build())
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_params_layout_and_version():
    L = bssmppi.load()
    assert L.bssmppi_abi_version() == 3
    assert L.bssmppi_params_size() == ctypes.sizeof(bssmppi.Params)


def test_invalid_parameters_rejected_on_host():
    """Validation happens before any CUDA call, so it works without a GPU."""
    L = bssmppi.load()
    p = workload.config0()
    for field, bad in (("M", 1), ("K", 0), ("T", 0), ("delta", 0.7), ("gamma", 1.5), ("lam", 0.0)):
        prm = bssmppi.make_params(p)
        setattr(prm, field, bad)
        h = ctypes.c_void_p()
        rc = L.bssmppi_create(ctypes.byref(prm), None, ctypes.byref(h))
        assert rc == -1, field
        assert h.value is None
        assert bssmppi.last_error(None)
    prm = bssmppi.make_params(p)
    prm.Sigma_w[0] = -1.0
    assert L.bssmppi_create(ctypes.byref(prm), None, ctypes.byref(ctypes.c_void_p())) == -1
    for field, bad in (("backoff", 2), ("backoff", -1), ("clamp_margin", 3)):
        prm = bssmppi.make_params(p)
        setattr(prm, field, bad)
        assert L.bssmppi_create(ctypes.byref(prm), None, ctypes.byref(ctypes.c_void_p())) == -1, field
        assert field in bssmppi.last_error(None)
    for resample, compensated in ((2, 1), (1, 0)):  # re-sampling runs with compensated reductions only
        prm = bssmppi.make_params(p)
        prm.resample, prm.compensated = resample, compensated
        assert L.bssmppi_create(ctypes.byref(prm), None, ctypes.byref(ctypes.c_void_p())) == -1
        assert "resample" in bssmppi.last_error(None)


def test_no_cpu_fallback_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = bssmppi.load()
    prm = bssmppi.make_params(workload.config0())
    h = ctypes.c_void_p()
    rc = L.bssmppi_create(ctypes.byref(prm), None, ctypes.byref(h))
    assert rc == -3  # ECUDA: the library refuses to run anywhere but on a CUDA device
    assert "CUDA" in bssmppi.last_error(None) or "device" in bssmppi.last_error(None)


def test_measurement_and_checking_entry_points_validate_arguments_on_host():
    """Argument errors come back as EINVAL before any CUDA call, so they need no GPU."""
    L = bssmppi.load()
    ms, tf, sms = ctypes.c_float(), ctypes.c_double(), ctypes.c_int32()
    for iters in (0, (1 << 24) + 1):
        rc = L.bssmppi_fp32_peak(0, iters, None, ctypes.byref(ms), ctypes.byref(tf), ctypes.byref(sms))
        assert rc == -1 and "iters" in bssmppi.last_error(None)
    assert L.bssmppi_fp32_peak(0, 16, None, None, ctypes.byref(tf), ctypes.byref(sms)) == -1
    assert L.bssmppi_tyre_curve(None, None, None, 4, None) == -1
    assert L.bssmppi_rear_tyre(None, None, None, 4, None) == -1
    c = (ctypes.c_float * 10)()
    assert L.bssmppi_tyre_curve_coefficients(1.9, c, 9) == -1  # room for fewer than ten coefficients
