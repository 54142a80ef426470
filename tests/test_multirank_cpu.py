"""The N > 1 path of bench.py on CPU (gloo, world size 2): every rank runs an
independent replica of the workload, the slowest rank's time is the job's,
and the job rate counts every rank's units (weak scaling)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank  # rank 1 is the slower replica
        t = bench.max_over_ranks(ms, dist, device="cpu")
        rate = bench.job_rate(world, 5, 1000, t)
        out.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_rank_reduction_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in got:
        assert t == 150.0                      # the slowest rank's time on every rank
        assert rate == 2 * 5 * 1000 / 0.150    # both ranks' units over that time


def test_single_process_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, None) == 42.0
    assert bench.job_rate(1, 3, 10, 1000.0) == 30.0
