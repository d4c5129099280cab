"""The N > 1 host path of bench.py (replicas: one independent box per rank,
no data-path collective) on CPU with world size 2 over gloo: the job time is
the slowest rank's, and the whole-job rate counts every rank's box."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.5 + rank, dist, device="cpu")   # rank 1 is the slow one
        e = bench.max_over_ranks(10.0 - rank, dist, device="cpu")
        dist.barrier()
        out[rank] = (t, e, bench.whole_job_rate(world, 64, 10, t))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_reduction_and_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    assert res[0] == res[1]
    t, e, rate = res[0]
    assert t == 2.5 and e == 10.0
    assert rate == pytest.approx(2 * 64 ** 3 * 10 / 2.5)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.whole_job_rate(1, 8, 4, 2.0) == 8 ** 3 * 4 / 2.0
