"""Multi-rank host logic of bench.py on CPU: gloo, world size 2.

Each rank measures its own step time; the job's time is the slowest rank's
and the job's value is the sum of the ranks' work over that time.  The ranks
here are processes with the gloo backend (no GPU)."""
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


def _rank_main(rank, world, port, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                     # rank 1 is the slow one
        job_ms = bench.max_over_ranks(ms, world, "cpu")
        dist.barrier()
        q.put((rank, job_ms, bench.job_gflops(1_000_000, world, job_ms)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, job_ms, gf in got:
        assert job_ms == 15.0                     # every rank sees the slowest rank's time
        assert gf == pytest.approx(2 * 2.0 * 1e6 / 15e-3 / 1e9)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_gflops(10**9, 1, 1000.0) == pytest.approx(2.0)
