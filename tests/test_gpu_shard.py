"""Sample-sharded solve on one GPU: several handles split the K samples of one solve
(bssmppi_set_sample_range), each reduces its range to a log-sum-exp partial
(bssmppi_solve_partial), and the merge (bssmppi_merge_partials) must reproduce the single-handle
solve. Per-sample work is identical (random streams keyed by the global sample index), so the costs
match bit for bit; the update and weights differ only by the order of the sums (FP32 rel 1e-5).
"""
import numpy as np
import pytest

import oracle
import workload
from tests.test_gpu_parity import assert_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2408_00494_gb300 import bssmppi  # noqa: E402


def _full(p, x0, v, ctr):
    c = bssmppi.Controller(p)
    try:
        bssmppi.set_counter(c.h, ctr)
        vt, u0 = torch.as_tensor(v, device="cuda"), torch.zeros(2, device="cuda")
        bssmppi.solve(c.h, torch.as_tensor(x0, device="cuda"), None, vt, u0)
        torch.cuda.synchronize()
        return {"v": vt.cpu().numpy(), "u0": u0.cpu().numpy(), "S": c.buffer(bssmppi.BUF_S).cpu().numpy(),
                "w": c.buffer(bssmppi.BUF_W).cpu().numpy(), "diag": c.buffer(bssmppi.BUF_DIAG).cpu().numpy()}
    finally:
        c.close()


def _sharded(p, x0, v, ctr, sizes):
    K_total = sum(sizes)
    ctls, parts, out = [], [], []
    try:
        begin = 0
        for n in sizes:
            q = workload.Problem(**{**p.__dict__, "K": n})
            c = bssmppi.Controller(q)
            bssmppi.set_sample_range(c.h, begin, K_total)
            bssmppi.set_counter(c.h, ctr)
            ctls.append(c)
            begin += n
        xt = torch.as_tensor(x0, device="cuda")
        for c in ctls:
            part = torch.empty(3 + 2 * p.T, device="cuda")
            bssmppi.solve_partial(c.h, xt, None, torch.as_tensor(v, device="cuda"), part)
            parts.append(part)
        allp = torch.stack(parts)
        for c in ctls:
            vt, u0 = torch.empty(p.T, 2, device="cuda"), torch.zeros(2, device="cuda")
            bssmppi.merge_partials(c.h, allp, vt, u0)
            torch.cuda.synchronize()
            out.append({"v": vt.cpu().numpy(), "u0": u0.cpu().numpy(), "S": c.buffer(bssmppi.BUF_S).cpu().numpy(),
                        "w": c.buffer(bssmppi.BUF_W).cpu().numpy(), "diag": c.buffer(bssmppi.BUF_DIAG).cpu().numpy(),
                        "ctr": bssmppi.get_counter(c.h)})
        return out
    finally:
        for c in ctls:
            c.close()


@pytest.mark.parametrize("sizes,variant", [((128, 128), "racing"), ((100, 123, 33), "racing"), ((1, 255), "racing"),
                                           ((96, 160), "constraints"), ((200, 56), "resample")])
def test_shards_merge_to_the_single_handle_solve(sizes, variant):
    p = workload.config0()
    p.K = sum(sizes)
    if variant == "resample":
        p.resample = 1
    if variant == "constraints":
        p.constraints = (workload.halfspace((0, 0, 0, 0, 1, 0), 2.5, 0.05),
                         workload.disk(5, 4, (40.0, 0.5), 1.0, 0.1, backoff="cantelli"))
    x0, v = workload.random_state(p, 61), workload.random_nominal(p, 61)
    full = _full(p, x0, v, ctr=5)
    shards = _sharded(p, x0, v, 5, sizes)
    np.testing.assert_array_equal(np.concatenate([s["S"] for s in shards]), full["S"])
    assert_close(np.concatenate([s["w"] for s in shards]), full["w"], 1e-5, 1e-7, "weights")
    for s in shards:
        assert s["ctr"] == 6
        assert_close(s["v"], full["v"], 1e-5, 1e-6, "v+")
        assert_close(s["u0"], full["u0"], 1e-5, 1e-6, "u0")
        assert s["diag"][0] == full["diag"][0]  # beta: the minimum of the same costs
        assert_close(s["diag"][1:], full["diag"][1:], 1e-5, 1e-6, "eta, ESS, free energy")


def test_sharded_solve_matches_oracle_full_size():
    """K=4096, M=64, T=40 split over 4 handles: the merged update against the oracle's update from
    the GPU's costs and perturbations (isolates the partial and merge arithmetic)."""
    p = workload.config1()
    x0, v = workload.random_state(p, 62), workload.random_nominal(p, 62)
    shards = _sharded(p, x0, v, 9, (1024,) * 4)
    full = _full(p, x0, v, ctr=9)
    S = np.concatenate([s["S"] for s in shards]).astype(np.float64)
    c = bssmppi.Controller(p)
    try:
        bssmppi.set_counter(c.h, 9)
        bssmppi.solve(c.h, torch.as_tensor(x0, device="cuda"), None, torch.as_tensor(v, device="cuda"))
        eps = c.buffer(bssmppi.BUF_EPS).cpu().numpy().astype(np.float64)
    finally:
        c.close()
    _, vp_iso, _ = oracle.optimal_control(S, v.astype(np.float64)[None] + eps, float(np.float32(p.lam)))
    for s in shards:
        assert_close(s["v"], vp_iso, 1e-4, 1e-5, "sharded v+ (from GPU costs)")
        assert_close(s["v"], full["v"], 1e-5, 1e-6, "sharded v+ against the single-handle v+")


def test_sample_range_validation_and_single_rank_helper():
    p = workload.config0()
    c = bssmppi.Controller(p)
    try:
        for k0, kt in ((-1, 512), (300, 512), (0, 100), (0, 1 << 21)):
            with pytest.raises(bssmppi.BssmppiError):
                bssmppi.set_sample_range(c.h, k0, kt)
        bssmppi.set_sample_range(c.h, 0, p.K)
        x0 = torch.as_tensor(workload.random_state(p, 3), device="cuda")
        v = workload.random_nominal(p, 3)
        bssmppi.set_counter(c.h, 2)
        vt = torch.as_tensor(v, device="cuda")
        bssmppi.sharded_solve(c.h, x0, p.T, v=vt)  # one rank: partial + merge
        torch.cuda.synchronize()
        full = _full(p, workload.random_state(p, 3), v, ctr=2)
        assert_close(vt.cpu().numpy(), full["v"], 1e-5, 1e-6, "single-rank sharded v+")
    finally:
        c.close()
