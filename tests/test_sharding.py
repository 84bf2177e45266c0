"""Row sharding's host side on the CPU: two gloo ranks (127.0.0.1).

The library calls its all-reduce hook once per pass with a device buffer; the
binding's TorchAllReduce answers through torch.distributed.  Here each rank
fills the staging buffer with its own partial sums (FP32 and FP64, as the
library's Z and G) and calls the hook the way the library does; every rank
must then hold the sum over ranks, bit for bit the same on both.  The library
entry point itself is checked for its argument errors (no device needed).
"""
import ctypes
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import paper_2109_03709_gb300 as P
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        red = P.TorchAllReduce(4096, "cpu")
        res = []
        for elem, dt, count in ((4, torch.float32, 300), (8, torch.float64, 129), (8, torch.float64, 1)):
            v = red.staging[: count * elem].view(dt)
            v.copy_(torch.arange(count, dtype=dt) * (rank + 1) + 0.25 * rank)
            st = red._call(red.staging.data_ptr(), count, elem, None, None)
            res.append((st, v.clone().numpy()))
        out.put((rank, res, red.calls, repr(red.error)))
    finally:
        dist.destroy_process_group()


def test_torch_allreduce_hook_sums_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, calls, ncalls, err in res:
        assert ncalls == 3, err
        for (st, v), count in zip(calls, (300, 129, 1)):
            assert st == 0
            np.testing.assert_array_equal(v, np.arange(count) * 3 + 0.25)
    for (st0, v0), (st1, v1) in zip(res[0][1], res[1][1]):
        assert np.array_equal(v0, v1)


def test_hook_reports_a_failed_sum_as_a_status():
    """Without a process group the sum fails inside the callback: the error stays
    on the Python side and the library gets a status, not an exception."""
    import paper_2109_03709_gb300 as P
    red = P.TorchAllReduce(64, "cpu")
    assert red._call(red.staging.data_ptr(), 4, 4, None, None) == P.PPCA_ERR_CUDA
    assert red.error is not None


def test_set_allreduce_argument_errors():
    from paper_2109_03709_gb300 import build as b
    b.build()
    import paper_2109_03709_gb300 as P
    lib = P.load_library()
    assert lib.ppca_set_allreduce(None, None, None, 0, None, 0) == P.PPCA_ERR_INVALID
