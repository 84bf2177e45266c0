"""Large-d EigenGame: the GPU path against the oracle's own EigenGame.

The 50000 x 262144 streaming workload (lambda_i = i^-1.5 + 1e-4, EigenGame
500 steps, minibatch 4096, lr 0.1, Nesterov 0.9, k = l = 32, then the pPCA
step) does not reach a streak of 32 eigenvectors within 1e-2 rad.  This test
decides whether that is the method or the code, on a reduced analogue the
FP64 oracle can run: the same spectrum formula and Hadamard-rotated generator
at d = 4096 (n = 50000, BF16 storage), the same schedule, both sides from the
same V0 over the same minibatches.

* The split-precision GPU EigenGame follows the oracle's trajectory over all
  500 steps: every direction of the primed basis within 1e-3 rad of the
  oracle's (measured: 3.6e-4 rad at most, 1e-7 rad for the leading ones).
* The fast (BF16) GPU EigenGame gives the pPCA step the same quality as the
  oracle's: the same streak at 1e-2 rad (+-1) and a maximum angle within 10 %.
* Both stay short of 32 (measured: 10 for each, maximum angle 0.29 rad): the
  shortfall at this schedule is the method's, and the wider d = 262144 problem,
  with a larger isotropic floor relative to its top eigenvalues, is harder
  still.

The truth is numpy's LAPACK eigh of X^T X formed in FP64 from the stored values
(a library routine used as a test reference; at d = 4096 the oracle's own
cyclic Jacobi would take hours).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_large_d_eigengame_quality_matches_the_oracle(cuda_device):
    import torch

    import paper_2109_03709_gb300 as P
    P.load_library()
    n, d, b, steps, lr, k, m = 50000, 4096, 4096, 500, 0.1, 32, 64
    lam = np.arange(1, d + 1, dtype=np.float64) ** -1.5 + 1e-4
    X, _ = synth.hadamard_rotated_data_torch(n, d, lam, 505, "cuda", torch.bfloat16)
    Xs = X.float().cpu().numpy().astype(np.float64)
    w, U = np.linalg.eigh(Xs.T @ Xs)
    w, U = w[::-1] / n, U[:, ::-1].copy()
    V0 = synth.initial_basis(d, m, seed=7)
    V0d = torch.from_numpy(np.ascontiguousarray(V0.T, dtype=np.float32)).cuda()

    def gpu(prec):
        h = P.ppca_create(X)
        prm = P.ppca_prime_params_default(P.PPCA_EIGENGAME)
        prm.batch, prm.lr, prm.momentum = b, lr, 0.9
        prm.precision = prec
        P.ppca_prime(h, P.PPCA_EIGENGAME, m, steps, prm, V0=V0d)
        E = torch.empty((k, d), dtype=torch.float32, device="cuda")
        lo = torch.empty(k, dtype=torch.float64, device="cuda")
        P.ppca_finalize(h, k, E, lo, P.PPCA_PREC_ACCURATE)
        Vd = torch.empty((m, d), dtype=torch.float32, device="cuda")
        P.ppca_get_basis(h, Vd)
        P.ppca_sync(h)
        return Vd.double().cpu().numpy().T, E.double().cpu().numpy().T

    V_acc, E_acc = gpu(P.PPCA_PREC_ACCURATE)
    V_fast, E_fast = gpu(P.PPCA_PREC_FAST)
    V_or = oracle.eigengame_prime(Xs, V0, b, steps, lr, 0.9)
    E_or, _ = oracle.ppca_finalize(Xs, V_or, k)        # the oracle's pPCA step on its own primed basis

    assert oracle.angles(V_acc, V_or).max() <= 1e-3
    a_or, a_fast, a_acc = (oracle.angles(E, U[:, :k]) for E in (E_or, E_fast, E_acc))
    s_or, s_fast, s_acc = (oracle.lces(a, 1e-2) for a in (a_or, a_fast, a_acc))
    assert s_acc == s_or
    assert abs(s_fast - s_or) <= 1, (s_fast, s_or)
    assert abs(a_fast.max() - a_or.max()) <= 0.1 * a_or.max(), (a_fast.max(), a_or.max())
    assert s_or < k, "the oracle reached the full streak: the large-d shortfall would be the code's"
