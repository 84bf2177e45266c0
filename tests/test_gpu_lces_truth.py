"""The benchmark's time-to-LCES ground truth, pinned to the oracle.

At the benchmark's size (1e6 x 4096) the oracle's cyclic Jacobi is too slow,
so bench.py takes the leading eigenvectors of X^T X from library routines
(FP32 cuBLAS GEMMs over 1024-row chunks summed in FP64, FP64 cuSOLVER eigh).
Here that routine is compared with the oracle's ground truth (FP64 X^T X and
its own Jacobi) on a small case, for FP32 and BF16 storage: angles <= 1e-6 rad
at relative eigengaps of 10%; eigenvalues to 1e-6 relative (FP32 products carry
u = 6e-8 each).  The LCES helper
is checked against the oracle's definition on planted angles.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev_matrix, stored_f64

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_lces_truth_matches_oracle(cuda_device, dtype):
    import bench
    n, d, k = 5000, 256, 16
    lam = 0.9 ** np.arange(1, d + 1)
    X, _ = synth.gaussian_data(n, d, lam, seed=21)
    Xd = dev_matrix(X, dtype)
    E, w = bench.lces_truth(Xd, k)
    Eo, wo = oracle.ground_truth(stored_f64(Xd), k)
    E = E.cpu().numpy()
    assert oracle.angles(E, Eo).max() <= 1e-6
    np.testing.assert_allclose(w.cpu().numpy(), wo, rtol=1e-6)


def test_lces_helper_matches_oracle_definition(cuda_device):
    import torch

    import bench
    d, k = 64, 6
    rng = np.random.default_rng(3)
    T, _ = np.linalg.qr(rng.standard_normal((d, k)))
    planted = np.array([1e-5, 5e-4, 2e-3, 1e-5, 3e-2, 1e-6])
    E = np.empty_like(T)
    for i in range(k):
        # rotate T_i by planted[i] towards a direction orthogonal to all of T
        u = rng.standard_normal(d)
        u -= T @ (T.T @ u)
        u /= np.linalg.norm(u)
        E[:, i] = np.cos(planted[i]) * T[:, i] + np.sin(planted[i]) * u
    Et = torch.from_numpy(np.ascontiguousarray(E.T, dtype=np.float32)).cuda()
    Tt = torch.from_numpy(T).cuda()
    for tol in (1e-3, 1e-4, 1e-1):
        streak, ang = bench.lces_of(Et, Tt, tol)
        assert streak == oracle.lces(oracle.angles(E.astype(np.float32).astype(np.float64), T), tol)
        np.testing.assert_allclose(ang, planted, rtol=1e-3, atol=2e-7)
