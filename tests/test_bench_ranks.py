"""Host logic of bench.py's multi-GPU line, run as two gloo ranks on the CPU:
the job time is the slowest rank's, and the value counts every rank's
replica of the workload (weak scaling, no data-path collective)."""
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


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t = bench.max_over_ranks(100.0 + 50.0 * rank, world)
        v = bench.job_mlups(1000, 90, 3, world, t)
        out.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_two_rank_job_time_is_the_max_and_value_counts_all_replicas():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == 150.0
        assert v == pytest.approx(1000 * 90 * 3 * 2 / 0.150 / 1e6)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_mlups(10, 2, 3, 1, 1000.0) == pytest.approx(60 / 1e6)
