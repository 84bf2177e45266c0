"""Row sharding on the GPU: two processes share cuda:0, each holding half the rows.

Each rank creates a handle over its own rows, gives it the binding's
TorchAllReduce (gloo, through host memory: the ranks' kernels never wait on
one another) and runs the same calls.  Checked against one process holding
all the rows, and against the oracle:
* block power (T = 10, Section 2.1) + the pPCA step: both ranks return the same
  E and lambda bit for bit; they match the single-process result (the sums
  differ only in their order: angles <= 1e-5 rad, eigenvalues 1e-6) and the
  oracle's pPCA step on the primed basis (FP32 tolerances: 1e-4 rad, 1e-5);
* EigenGame (10 steps, Section 2.3): the sharded minibatch t is the union of
  each rank's local minibatch t, which a single process reproduces on the rows
  reordered so that its contiguous batches of twice the size are those
  unions; the primed bases agree to 1e-4 rad per direction.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

N, D, K, M, B = 8192, 256, 8, 16, 512


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _data():
    X, _ = synth.gaussian_data(N, D, 0.9 ** np.arange(1, D + 1), seed=77)
    return X.astype(np.float32)


def _prime(P, torch, Xd, method, T, batch, V0, reducer=None, n_total=0):
    h = P.ppca_create(Xd)
    if reducer is not None:
        P.ppca_set_allreduce(h, reducer, n_total)
    prm = P.ppca_prime_params_default(method)
    prm.precision = P.PPCA_PREC_ACCURATE
    if method == P.PPCA_EIGENGAME:
        prm.batch, prm.lr, prm.momentum = batch, 0.05, 0.9
    V0d = torch.from_numpy(np.ascontiguousarray(V0.T, dtype=np.float32)).cuda()
    P.ppca_prime(h, method, M, T, prm, V0=V0d)
    E = torch.empty((K, D), dtype=torch.float32, device="cuda")
    lam = torch.empty(K, dtype=torch.float64, device="cuda")
    P.ppca_finalize(h, K, E, lam)
    V = torch.empty((M, D), dtype=torch.float32, device="cuda")
    P.ppca_get_basis(h, V)
    P.ppca_sync(h)
    return V.double().cpu().numpy().T, E.double().cpu().numpy().T, lam.cpu().numpy()


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import paper_2109_03709_gb300 as P
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P.load_library()
        X = _data()
        half = N // world
        Xd = torch.from_numpy(X[rank * half:(rank + 1) * half].copy()).cuda()
        V0 = synth.initial_basis(D, M, seed=5)
        red = P.TorchAllReduce(D * M * 4, "cuda")
        power = _prime(P, torch, Xd, P.PPCA_POWER, 10, 0, V0, red, N)
        eg = _prime(P, torch, Xd, P.PPCA_EIGENGAME, 10, B, V0, red, N)
        out.put((rank, power, eg, red.calls, repr(red.error)))
    finally:
        dist.destroy_process_group()


def test_row_sharded_priming_and_ppca_step_match_one_process(cuda_device):
    import multiprocessing as mp

    import torch

    import paper_2109_03709_gb300 as P
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=600) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (_, pw0, eg0, calls0, err0), (_, pw1, eg1, _, _) = res
    assert calls0 > 0, err0
    for a, b in zip(pw0 + eg0, pw1 + eg1):           # every rank holds the same result
        assert np.array_equal(a, b)

    P.load_library()
    X = _data()
    V0 = synth.initial_basis(D, M, seed=5)
    _, E1, l1 = _prime(P, torch, torch.from_numpy(X).cuda(), P.PPCA_POWER, 10, 0, V0)
    Vs, Es, ls = pw0
    assert oracle.angles(Es, E1).max() <= 1e-5
    np.testing.assert_allclose(ls, l1, rtol=1e-6)
    Eo, lo = oracle.ppca_finalize(X.astype(np.float64), Vs, K)
    assert oracle.angles(Es, Eo).max() <= 1e-4
    np.testing.assert_allclose(ls, lo, rtol=1e-5)

    # EigenGame: batch t of the reordered rows (size 2B) = rank 0's local batch t + rank 1's
    half = N // 2
    order = np.concatenate([np.r_[j * B:(j + 1) * B, half + j * B:half + (j + 1) * B] for j in range(half // B)])
    Veg, _, _ = _prime(P, torch, torch.from_numpy(X[order].copy()).cuda(), P.PPCA_EIGENGAME, 10, 2 * B, V0)
    assert oracle.angles(eg0[0], Veg).max() <= 1e-4
