"""The N > 1 bench path on CPU: two gloo ranks, each with its own timed
total, agree on the slowest rank's time, and the whole-job throughput counts
every replica's steps within it (replicas only, no data-path collective)."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    totals = [10.0 + 5.0 * rank, 40.0 - rank, 7.0]   # ms: fp32, fp64, gradient
    got = b.max_over_ranks(dist, totals, "cpu")
    dist.barrier()
    q.put((rank, got, b.job_throughput(world, 100, got[0])))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, got, value in res:
        assert got == [15.0, 40.0, 7.0]
        # 2 replicas x 100 steps within the slowest rank's 15 ms
        assert value == round(2 * 1000.0 * 100 / 15.0, 2)


def test_single_rank_is_identity():
    b = _bench()
    assert b.max_over_ranks(None, [1.0, 2.0], "cpu") == [1.0, 2.0]
    assert b.job_throughput(1, 200, 40.0) == 5000.0
