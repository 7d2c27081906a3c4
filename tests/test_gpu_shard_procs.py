"""The product's sample-sharded solve across processes: two ranks (spawned processes on the one
GPU, gloo on the host) each own a handle covering half of the K=4096 samples, and
bssmppi.sharded_solve runs the partial kernel, gathers the 3 + 2T partials through host memory and
merges them. No kernel waits on the other process: each rank's launches finish before the host
exchange. Every rank must end with the single-handle solve's costs (bit for bit), update, u0 and
diagnostics (FP32 rel 1e-5: only the order of the sums differs), and an advanced counter.
"""
import os
import socket

import numpy as np
import pytest

import workload
from tests.test_gpu_parity import assert_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2408_00494_gb300 import bssmppi  # noqa: E402

CTR = 13


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    p = workload.config1()
    return p, workload.random_state(p, 71), workload.random_nominal(p, 71)


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        p, x0, v = _case()
        k0, k1 = rank * p.K // world, (rank + 1) * p.K // world
        c = bssmppi.Controller(workload.Problem(**{**p.__dict__, "K": k1 - k0}))
        try:
            bssmppi.set_sample_range(c.h, k0, p.K)
            bssmppi.set_counter(c.h, CTR)
            vt, u0 = torch.as_tensor(v, device="cuda"), torch.zeros(2, device="cuda")
            bssmppi.sharded_solve(c.h, torch.as_tensor(x0, device="cuda"), p.T, v=vt, u0=u0)
            torch.cuda.synchronize()
            q.put((rank, k0, vt.cpu().numpy(), u0.cpu().numpy(), c.buffer(bssmppi.BUF_S).cpu().numpy(),
                   c.buffer(bssmppi.BUF_W).cpu().numpy(), c.buffer(bssmppi.BUF_DIAG).cpu().numpy(),
                   bssmppi.get_counter(c.h)))
        finally:
            c.close()
    finally:
        dist.destroy_process_group()


def test_two_processes_shard_one_solve_through_the_library():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    p, x0, v = _case()
    c = bssmppi.Controller(p)
    try:
        bssmppi.set_counter(c.h, CTR)
        vt, u0 = torch.as_tensor(v, device="cuda"), torch.zeros(2, device="cuda")
        bssmppi.solve(c.h, torch.as_tensor(x0, device="cuda"), None, vt, u0)
        torch.cuda.synchronize()
        full = {"v": vt.cpu().numpy(), "u0": u0.cpu().numpy(), "S": c.buffer(bssmppi.BUF_S).cpu().numpy(),
                "w": c.buffer(bssmppi.BUF_W).cpu().numpy(), "diag": c.buffer(bssmppi.BUF_DIAG).cpu().numpy()}
    finally:
        c.close()
    np.testing.assert_array_equal(np.concatenate([o[4] for o in out]), full["S"])
    assert_close(np.concatenate([o[5] for o in out]), full["w"], 1e-5, 1e-7, "weights")
    for rank, k0, v_r, u0_r, _, _, diag_r, ctr_r in out:
        assert ctr_r == CTR + 1
        assert_close(v_r, full["v"], 1e-5, 1e-6, f"rank {rank} v+")
        assert_close(u0_r, full["u0"], 1e-5, 1e-6, f"rank {rank} u0")
        assert diag_r[0] == full["diag"][0]
        assert_close(diag_r[1:], full["diag"][1:], 1e-5, 1e-6, f"rank {rank} eta, ESS, free energy")
