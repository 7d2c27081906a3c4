"""Multi-rank paths on CPU with two gloo ranks.

1. Replicas (the benchmark): each rank measures its own controller; the job's time is the slowest
   rank's and its throughput all ranks' units over that time (the aggregation bench.py uses under
   torchrun).
2. A sample-sharded solve: each rank rolls out its own range of the K samples and takes the
   log-sum-exp partial of its weights and update; one all-gather of the partials (3 + 2T values per
   rank) and a merge give every rank the whole solve's update. Run here with the FP64 oracle on the
   ranks, which checks the partition, the exchange and the merge against the unsharded solve.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        per_rank = [[0.45, 0.41, 0.47, 0.02], [0.52, 0.40, 0.44, 0.03]][rank]
        got = bench.reduce_over_ranks(per_rank, "cpu", world)
        q.put((rank, got, bench.whole_job_throughput(4096 * 64 * 40, got[0], world)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, thr in out:
        assert got == [0.52, 0.41, 0.47, 0.03]
        assert thr == pytest.approx(2 * 4096 * 64 * 40 / 0.52e-3)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks([1.0, 2.0], "cpu", 1) == [1.0, 2.0]
    assert bench.whole_job_throughput(100, 1.0, 1) == pytest.approx(1e5)


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import numpy as np

        import oracle
        import workload
        p = workload.config0()
        p.K, p.T = 96, 12
        x0, v = workload.random_state(p, 8), workload.random_nominal(p, 8)
        k0, k1 = rank * p.K // world, (rank + 1) * p.K // world
        r = oracle.Oracle(p).solve(x0, v, 21, k_range=(k0, k1))
        part = torch.as_tensor(oracle.lse_partial(r["S"], r["u"], float(np.float32(p.lam)), (k0, k1)))
        parts = [torch.empty_like(part) for _ in range(world)]
        dist.all_gather(parts, part)
        vp, diag = oracle.lse_merge(torch.stack(parts).numpy(), float(np.float32(p.lam)), p.K)
        q.put((rank, vp, diag))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_samples_of_one_solve():
    import numpy as np

    import oracle
    import workload
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    p = workload.config0()
    p.K, p.T = 96, 12
    full = oracle.Oracle(p).solve(workload.random_state(p, 8), workload.random_nominal(p, 8), 21)
    for rank, vp, diag in out:
        np.testing.assert_allclose(vp, full["v_plus"], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(diag, full["diag"], rtol=1e-12)
