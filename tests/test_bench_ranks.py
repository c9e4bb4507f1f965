"""The replicas path of bench.py on the CPU: two gloo ranks (world size 2, as
torchrun launches them) with different work and different local times report
the same whole-job rate, all ranks' units over the slowest rank's time, and the
single-rank path needs no process group."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rate, s = bench.job_rate(0.010 * (rank + 1), 1000 * (rank + 1), world)  # rank 1: more work, slower
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, rate, s))


def test_job_rate_takes_the_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, s in out:
        assert s == pytest.approx(0.020)
        assert rate == pytest.approx((1000 + 2000) / 0.020)


def test_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    rate, s = bench.job_rate(0.5, 10, 1)
    assert s == 0.5 and rate == pytest.approx(20.0)
