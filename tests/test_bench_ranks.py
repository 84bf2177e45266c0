"""The bench's multi-rank arithmetic on CPU: two gloo ranks (127.0.0.1), the
job time is the slowest rank's, the rate is all ranks' bytes over it."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], dist, "cpu")
        out.put((rank, t, bench.whole_job_rate(8e9, t, world)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_with_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [0.25, 0.5]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [0.5, 0.5]
    assert all(r[2] == pytest.approx(2 * 8e9 / 0.5 / 1e9) for r in res)


def test_single_rank_helpers_need_no_process_group():
    import bench
    assert bench.max_over_ranks(1.5, None, "cpu") == 1.5
    assert bench.whole_job_rate(4e9, 2.0, 1) == pytest.approx(2.0)
