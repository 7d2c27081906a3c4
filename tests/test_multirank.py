"""Multi-rank path of the benchmark on CPU: two gloo ranks (replicas, no collective on the data path).

Each rank measures its own controller; the job's time is the slowest rank's, and the job's
throughput is all ranks' units over that time. This checks the aggregation bench.py uses under
torchrun with world size 2, on CPU with the gloo backend.
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
