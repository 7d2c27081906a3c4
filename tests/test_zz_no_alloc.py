"""The allocation-free weights/update entry point (bssmppi_update_noalloc) against bssmppi_solve.

Callers that cannot allocate device memory at run time (hard real-time loops, plugins whose host
process owns the device memory) use bssmppi_update_noalloc, whose scratch is a fixed array in the
library. This checks, through the C ABI, that two calls in a row give the same weights, v+, first
control, diagnostics and counter advance as the update inside bssmppi_solve, within the update
tolerance of the parity tests (rel 1e-4 / abs 1e-5 for v+, rel 1e-5 / abs 1e-7 for weights),
and the same against the FP64 oracle's weights and update of the same costs and perturbations.
This file is collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import oracle
import workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2408_00494_gb300 import bssmppi  # noqa: E402


def _solve_reference(prob, x0, v, ctr):
    """One bssmppi_solve; returns its inputs to the update (S, eps) and its outputs."""
    c = bssmppi.Controller(prob)
    try:
        bssmppi.set_counter(c.h, ctr)
        vt = torch.as_tensor(v, device="cuda").contiguous()
        u0 = torch.zeros(2, device="cuda")
        bssmppi.solve(c.h, torch.as_tensor(x0, device="cuda"), None, vt, u0)
        out = {name: c.buffer(buf) for name, buf in (("S", bssmppi.BUF_S), ("eps", bssmppi.BUF_EPS),
                                                     ("w", bssmppi.BUF_W), ("diag", bssmppi.BUF_DIAG))}
        out["v_plus"], out["u0"] = vt, u0
        out["counter"] = bssmppi.get_counter(c.h)
        torch.cuda.synchronize()
        return out
    finally:
        c.close()


def _close(a, b, rtol, atol):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    assert np.all(np.abs(a - b) <= atol + rtol * np.abs(b)), np.abs(a - b).max()


def test_update_noalloc_matches_solve_on_two_calls_in_a_row():
    p = workload.config0()
    p.K, p.T = 1000, 24  # several update blocks and a ragged last chunk
    cases = []
    for seed in (1, 2):
        x0 = workload.random_state(p, seed)
        v = workload.random_nominal(p, seed)
        cases.append((v, _solve_reference(p, x0, v, ctr=10 + seed)))
    for v, ref in cases:  # two calls in a row, sharing the library's scratch
        v_io = torch.as_tensor(v, device="cuda").contiguous()
        w = torch.full((p.K,), -1.0, device="cuda")
        u0 = torch.zeros(2, device="cuda")
        diag = torch.zeros(bssmppi.NDIAG, device="cuda")
        counter = torch.tensor([7], dtype=torch.int32, device="cuda")
        bssmppi.update_noalloc(ref["S"], ref["eps"], v_io, w, u0, diag, counter, lam=float(p.lam))
        torch.cuda.synchronize()
        _close(v_io, ref["v_plus"], 1e-4, 1e-5)
        _close(u0, ref["u0"], 1e-4, 1e-5)
        _close(w, ref["w"], 1e-5, 1e-7)
        _close(diag, ref["diag"], 1e-5, 1e-7)
        assert int(counter.item()) == 8
        # and against the FP64 weights and update of the same costs and perturbations
        S64, eps64 = ref["S"].double().cpu().numpy(), ref["eps"].double().cpu().numpy()
        w64, vp64, _ = oracle.optimal_control(S64, v.astype(np.float64)[None] + eps64, float(np.float32(p.lam)))
        _close(v_io, torch.as_tensor(vp64), 1e-4, 1e-5)
        _close(w, torch.as_tensor(w64), 1e-5, 1e-7)


def test_update_noalloc_without_optional_outputs_and_size_limit():
    p = workload.config0()
    x0, v = workload.random_state(p, 3), workload.random_nominal(p, 3)
    ref = _solve_reference(p, x0, v, ctr=1)
    v_io = torch.as_tensor(v, device="cuda").contiguous()
    w = torch.empty(p.K, device="cuda")
    bssmppi.update_noalloc(ref["S"], ref["eps"], v_io, w, lam=float(p.lam))
    torch.cuda.synchronize()
    _close(v_io, ref["v_plus"], 1e-4, 1e-5)
    # sizes beyond the static scratch's limits are rejected before any launch
    L = bssmppi.load()
    null = None
    rc = L.bssmppi_update_noalloc(null, null, null, null, null, null, null, 1 << 21, 10, 1.0, 1, null)
    assert rc == -1 and "K out of range" in bssmppi.last_error(None)
    rc = L.bssmppi_update_noalloc(null, null, null, null, null, null, null, 100, 257, 1.0, 1, null)
    assert rc == -1 and "T out of range" in bssmppi.last_error(None)
